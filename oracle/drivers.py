"""Oracle versions of the paper's two p-adaptation strategies (Sec. 3.2).

TEST INFRASTRUCTURE ONLY: the tests compare the library's drivers
(paper_2210_03523_gb300.adapt) with these loops.  Every step is an oracle
call (dg_oracle.c); this file only sequences them as the flowcharts do.

Dynamic (Fig. 1): initialise, then repeat { advance dt_e; if the final time
is reached stop; estimate the error; adapt }.
Static (Fig. 2): initialise, then repeat { advance dt_e; if the final
estimation time is reached leave the loop; estimate the error and keep it },
adapt once from the kept estimates, advance to the final time.

Readings, stated once: stage k ends at t0 + k dt_e (a physical time, as in
the paper's runs, Sec. 3) and the time step is shortened to land on it; the
flowcharts estimate only after a stage that did not reach the final
(estimation) time; the estimate of a stage is the tau map of the chosen form
over the sweep, extrapolated to the target list when one is given (approach
2 needs the extrapolated map, Sec. 2.4); the static total map is the F_max
of the stage maps; the RK register restarts at zero after an adaptation
(Williamson's first stage discards it anyway).
"""
from __future__ import annotations

import numpy as np

from . import Mesh, select_orders, tau_extrapolate


def ndof(orders):
    """degrees of freedom per variable of a discretisation: sum of the element
    node counts (N1+1)(N2+1)(N3+1)"""
    o = np.asarray(orders, dtype=np.int64).reshape(-1, 3)
    return int(np.prod(o + 1, axis=1).sum())


def _stage_map(m, q, sweep, form, isolated, targets, n_fit, decoupled, tau_floor):
    tn, tt = m.tau(q, sweep, isolated=isolated)
    mp = tn if form == "new" else tt
    if targets is None:
        return mp, np.asarray(sweep, dtype=np.int32).reshape(-1, 3)
    return tau_extrapolate(mp, m.orders, sweep, targets, n_fit, decoupled, tau_floor=tau_floor), np.asarray(targets, np.int32).reshape(-1, 3)


def static_adaptation(mi, q0, *, t0, t_est, dt_e, t_final, cfl, sweep, tau_max, n_min, n_max, jump_rule=0,
                      form="new", isolated=True, targets=None, n_fit=0, decoupled=False, tau_floor=0.0):
    """Fig. 2.  Returns a dict: orders, q (final state), t, total (the F_max
    map or None), n_estimates, steps (before, after adaptation), ndof (of the
    adapted orders), ndof_dyn (the step-weighted mean over the whole run)."""
    m = Mesh(mi)
    q = np.array(q0, dtype=np.float64)
    G = np.zeros_like(q)
    t, total, n_est, steps, k = float(t0), None, 0, 0, 1
    lst = None
    nd0 = ndof(m.orders)
    while True:
        t, n = m.advance(q, G, cfl, t, min(t0 + k * dt_e, t_est))
        steps += n
        if t >= t_est:
            break
        mp, lst = _stage_map(m, q, sweep, form, isolated, targets, n_fit, decoupled, tau_floor)
        total = mp.copy() if total is None else np.maximum(total, mp)
        n_est += 1
        k += 1
    if total is None:
        orders = np.array(m.orders, dtype=np.int32)
    else:
        orders = select_orders(total, lst, tau_max, n_min, n_max, jump_rule, mi.neighbors)
    q = m.set_orders(orders, q)
    m2 = Mesh(mi.with_orders(orders))
    G = np.zeros_like(q)
    t, n2 = m2.advance(q, G, cfl, t, t_final)
    nd = ndof(orders)
    ndyn = (steps * nd0 + n2 * nd) / (steps + n2) if steps + n2 else float(nd)
    return dict(orders=orders, q=q, t=t, total=total, n_estimates=n_est, steps=(steps, n2), ndof=nd, ndof_dyn=ndyn)


def dynamic_adaptation(mi, q0, *, t0, dt_e, t_final, cfl, sweep, tau_max, n_min, n_max, jump_rule=0,
                       max_decrease=-1, form="new", isolated=True, targets=None, n_fit=0, decoupled=False, tau_floor=0.0):
    """Fig. 1.  sweep: a fixed list, or a callable orders -> list (the orders
    change between stages).  Returns a dict: orders, q, t, history (orders
    after every adaptation), steps, ndof (of the final orders), ndof_dyn
    (the mean NDOF over the time steps)."""
    m = Mesh(mi)
    q = np.array(q0, dtype=np.float64)
    G = np.zeros_like(q)
    t, steps, k, hist, nd_sum = float(t0), 0, 1, [], 0
    while True:
        t, n = m.advance(q, G, cfl, t, min(t0 + k * dt_e, t_final))
        steps += n
        nd_sum += n * ndof(m.orders)
        if t >= t_final:
            break
        sw = sweep(m.orders) if callable(sweep) else sweep
        mp, lst = _stage_map(m, q, sw, form, isolated, targets, n_fit, decoupled, tau_floor)
        orders = select_orders(mp, lst, tau_max, n_min, n_max, jump_rule, mi.neighbors, prev=m.orders,
                               max_decrease=max_decrease)
        q = m.set_orders(orders, q)
        m = Mesh(mi.with_orders(orders))
        G = np.zeros_like(q)
        hist.append(orders)
        k += 1
    nd = ndof(m.orders)
    return dict(orders=np.array(m.orders, dtype=np.int32), q=q, t=t, history=hist, steps=steps, ndof=nd,
                ndof_dyn=nd_sum / steps if steps else float(nd))
