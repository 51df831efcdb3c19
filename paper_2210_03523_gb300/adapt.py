"""The paper's two p-adaptation strategies (Sec. 3.2) over the libdg C ABI.

Dynamic (Fig. 1): initialise, then repeat { advance dt_e; stop at the final
time; estimate the error; adapt }.  Static (Fig. 2): initialise, then repeat
{ advance dt_e; leave at the final estimation time; estimate the error and
keep it }, adapt once from the kept estimates, advance to the final time.

Every step runs in the library: dg_advance (CFL-adaptive RK3 to the stage
time, replayed as CUDA graphs), dg_tau_estimate, dg_tau_extrapolate (with
F_max accumulation on the device), dg_select_orders and dg_set_orders.
This module only sequences the calls and reads the time back once per stage.

Readings: stage k ends at t0 + k dt_e (a physical time, Sec. 3); estimates
follow only stages that did not reach the final (estimation) time; a stage's
estimate is the map of the chosen form (new, Eq. TEtildedef, or traditional,
Eq. TEdef) over the sweep, extrapolated to the target list when one is
given (approach 2, Sec. 2.4); the static total map is their F_max; the RK
register restarts at zero after an adaptation.  NDOF is the node count per
variable (dg_count_nodes); NDOF_dyn, the mean NDOF over the time steps of
the run (Sec. 3.3), weights each stage's NDOF by the steps it took.
"""
from __future__ import annotations

import numpy as np

from . import dg


def _to_device(q, device):
    import torch
    if isinstance(q, torch.Tensor):
        return q.to(device=device, dtype=torch.float64).contiguous().clone()
    return torch.from_numpy(np.ascontiguousarray(q, dtype=np.float64)).to(device)


class _Stage:
    """Per-stage estimate with device buffers reused across stages."""

    def __init__(self, form, isolated, fp32, targets, n_fit, decoupled, tau_floor):
        self.form, self.isolated, self.fp32 = form, isolated, fp32
        self.targets = None if targets is None else np.ascontiguousarray(np.asarray(targets, np.int32).reshape(-1, 3))
        self.n_fit, self.decoupled, self.tau_floor = n_fit, decoupled, tau_floor

    def map(self, m, q, sweep, into=None):
        """The stage map (accumulated by max into `into` when given); returns
        (map, the list it is over)."""
        new = self.form == "new"
        if self.targets is None:
            tn, tt = m.tau_estimate(q, sweep, isolated=self.isolated, fp32=self.fp32, accumulate=into is not None,
                                    map_new=into if new else None, map_trad=None if new else into,
                                    want=(new, not new))
            return (tn if new else tt), np.asarray(sweep, np.int32).reshape(-1, 3)
        tn, tt = m.tau_estimate(q, sweep, isolated=self.isolated, fp32=self.fp32, want=(new, not new))
        mp = tn if new else tt
        out = m.tau_extrapolate(mp, sweep, self.targets, n_fit=self.n_fit, tau_floor=self.tau_floor,
                                decoupled=self.decoupled, out=into, accumulate=into is not None)
        return out, self.targets


def static_adaptation(mi, q0, *, t0, t_est, dt_e, t_final, cfl, sweep, tau_max, n_min, n_max, jump_rule=0,
                      form="new", isolated=True, fp32=False, targets=None, n_fit=0, decoupled=False, tau_floor=0.0,
                      stream=None, keep_estimation_state=False):
    """Fig. 2 on the GPU.  mi: a MeshInput; q0: the initial state (host or
    device).  Returns a dict: orders (host), q (device), t, total (device F_max
    map or None), n_estimates, steps (before, after adaptation), ndof (of the
    adapted orders), ndof_dyn (the step-weighted mean over the run), mesh;
    with keep_estimation_state, q_est: a copy of the state at the initial
    orders when the estimation phase ended (at t_est_state), before the
    projection."""
    import torch
    m = dg.Mesh(mi, stream=stream)
    q = _to_device(q0, m.device)
    g = torch.zeros_like(q)
    t = torch.full((1,), float(t0), dtype=torch.float64, device=m.device)
    st = _Stage(form, isolated, fp32, targets, n_fit, decoupled, tau_floor)
    total, lst, n_est, steps, k = None, None, 0, 0, 1
    nd0 = dg.dg_count_nodes(np.asarray(mi.orders, np.int32).reshape(-1, 3))
    while True:
        steps += m.advance(q, g, t, min(t0 + k * dt_e, t_est), cfl, count=True)
        if float(t.item()) >= t_est:
            break
        total, lst = st.map(m, q, sweep, into=total)
        n_est += 1
        k += 1
    if total is None:
        orders = np.array(mi.orders, dtype=np.int32).reshape(-1, 3)
    else:
        orders = m.select_orders(total, lst, tau_max, n_min, n_max, jump_rule)
    t_est_state = float(t.item())
    q_est = q.clone() if keep_estimation_state else None
    q = m.set_orders(orders, q)
    g = torch.zeros_like(q)
    n2 = m.advance(q, g, t, t_final, cfl, count=True)
    nd = dg.dg_count_nodes(orders)
    ndyn = (steps * nd0 + n2 * nd) / (steps + n2) if steps + n2 else float(nd)
    return dict(orders=orders, q=q, t=float(t.item()), total=total, n_estimates=n_est, steps=(steps, n2), ndof=nd,
                ndof_dyn=ndyn, mesh=m, q_est=q_est, t_est_state=t_est_state)


def dynamic_adaptation(mi, q0, *, t0, dt_e, t_final, cfl, sweep, tau_max, n_min, n_max, jump_rule=0,
                       max_decrease=-1, form="new", isolated=True, fp32=False, targets=None, n_fit=0,
                       decoupled=False, tau_floor=0.0, stream=None):
    """Fig. 1 on the GPU.  sweep: a fixed list, or a callable orders -> list.
    Returns a dict: orders, q, t, history (orders after every adaptation),
    steps, ndof (of the final orders), ndof_dyn (the mean NDOF over the time
    steps), mesh, and timing: host wall seconds per stage of the time
    integration (advance_s), of the estimate and the order selection
    (estimate_select_s; the selection is a synchronous call that waits for
    the estimate) and of the mesh rebuild with the projection of the state
    (rebuild_s: dg_set_orders, synchronous, on the host)."""
    import time
    import torch
    m = dg.Mesh(mi, stream=stream)
    q = _to_device(q0, m.device)
    g = torch.zeros_like(q)
    t = torch.full((1,), float(t0), dtype=torch.float64, device=m.device)
    st = _Stage(form, isolated, fp32, targets, n_fit, decoupled, tau_floor)
    orders = np.array(mi.orders, dtype=np.int32).reshape(-1, 3)
    steps, k, hist, nd_sum = 0, 1, [], 0
    timing = {"advance_s": [], "estimate_select_s": [], "rebuild_s": []}
    while True:
        ta = time.perf_counter()
        n = m.advance(q, g, t, min(t0 + k * dt_e, t_final), cfl, count=True)
        timing["advance_s"].append(time.perf_counter() - ta)
        steps += n
        nd_sum += n * dg.dg_count_nodes(orders)
        if float(t.item()) >= t_final:
            break
        sw = sweep(orders) if callable(sweep) else sweep
        tb = time.perf_counter()
        mp, lst = st.map(m, q, sw)
        orders = m.select_orders(mp, lst, tau_max, n_min, n_max, jump_rule, max_decrease=max_decrease)
        tc = time.perf_counter()
        q = m.set_orders(orders, q)
        g = torch.zeros_like(q)
        timing["estimate_select_s"].append(tc - tb)
        timing["rebuild_s"].append(time.perf_counter() - tc)
        hist.append(orders)
        k += 1
    nd = dg.dg_count_nodes(orders)
    return dict(orders=orders, q=q, t=float(t.item()), history=hist, steps=steps, ndof=nd,
                ndof_dyn=nd_sum / steps if steps else float(nd), mesh=m, timing=timing)
