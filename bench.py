"""Benchmark of the DGSEM hot path on GB300.

Workload (default ``pulse48mixed``): the Euler density pulse on 48^3
periodic straight hexes. Each element's orders (N1,N2,N3) are drawn i.i.d.
from {2..8} (seed 2210), so faces are p-nonconforming; 2.4e7 nodes, a state
of 0.96 GB. One *step* is one pass of the whole hot path:

  * 50 explicit RK3 steps in FP64 through dg_advance (batches of steps
    replayed as CUDA graphs). Each RK step is one CFL reduction and three
    stages of face flux + volume residual with the fused RK update.
  * then one FP32 isolated tau-estimation sweep over every anisotropic
    order N <= P_e of every element, both forms, max-accumulated.

The timed region runs the steps as a user would, without per-kernel events.
A second timed region runs up to PROFILE_STEPS of the same steps with CUDA
events around every kernel (launched one by one); the per-kernel shares and
the roofline come from it.  On the 48^3 mixed-order mesh the same step is
then timed on the uniform-order partner (P = (5,5,5), the same expected
nodes per element) and reported under ``vs_uniform``.

The metric is DOF-residuals/s: NDOF x residual evaluations per step / step
time, summed over ranks. tau-estimated elements/s is reported next to it.

``--impl reference`` times the CPU oracle (FP64 C, OpenMP over elements) on
a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DOF-residuals/s and tau-estimated elements/s at stated error; % of HBM roofline"
UNIT = "DOF-residuals/s"
CFL = 0.5
RK_PER_STEP = 50
DEFAULT_WORKLOAD = "pulse48mixed"
UNIFORM_PARTNER = {"pulse48mixed": "pulse48uniform"}   # the uniform-order FP64 path at the same nodes per element
PROFILE_STEPS = 5          # steps of the profiled region, the e2e region and the uniform partner (at most K)
TAU_FP32_BOUND = ("<= 8 (eps32 S_dev + eps64 S_full) per element, S = (sum_i ||D^(P_i)||) F max|Ja| / min J, F the "
                  "largest flux-deviation term (deviations from the element's first-node state) or, for the FP64 "
                  "reference's own rounding, the largest flux term")
L2_FLUSH_BYTES = 256 << 20
FP64_FMA_PER_CLK_PER_SM = 2        # GB300: 64 FP64 lanes per 32 clocks per SM (measured 1.20 TFLOP/s)
FP32_FMA_PER_CLK_PER_SM = 128
N_SM = 152


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def workload_desc(name):
    return {
        "pulse16mixed": "Euler density pulse, 16^3 periodic straight hexes, orders iid U{1..6} per element and "
                        "direction (seed 2210), Roe, gamma=1.4, Mach 0.1; step = 50 RK3 steps at CFL 0.5 (FP64) "
                        "+ 1 FP32 isolated tau sweep over all N <= P_e",
        "pulse32mixed": "Euler density pulse, 32^3 periodic straight hexes, orders iid U{1..6} (seed 2210); "
                        "step = 50 RK3 steps + 1 FP32 tau sweep",
        "pulse4": "Euler density pulse, 4^3 periodic straight hexes, P=(4,4,4); step = 50 RK3 steps + 1 FP32 tau sweep",
        "pulse48mixed": "Euler density pulse, 48^3 periodic straight hexes, orders iid U{2..8} (seed 2210); "
                        "step = 50 RK3 steps + 1 FP32 tau sweep",
        "pulse48uniform": "Euler density pulse, 48^3 periodic straight hexes, P=(5,5,5); step = 50 RK3 steps + 1 "
                          "FP32 tau sweep",
        "pulse24mixed": "Euler density pulse, 24^3 periodic straight hexes, orders iid U{2..8} (seed 2210); step = "
                        "50 RK3 steps + 1 FP32 tau sweep",
        "cylinder": "Navier-Stokes flow past a cylinder, Re=100, Ma=0.2, Pr=0.72, 40x24x1 curved O-grid (geometry "
                    "order 3), P=(6,6,1), BR1, no-slip adiabatic wall; step = 50 RK3 steps + 1 FP32 tau sweep",
    }[name]


def initial_state(workload, mi, xyz):
    """The density pulse for the pulse workloads; the free stream, slowed near
    the wall with a seeded small perturbation, for the cylinder."""
    from paper_2210_03523_gb300 import inputs as I
    if workload != "cylinder":
        return I.pulse_state_fast(xyz, mi.orders, mi.phys)
    ph = mi.phys
    p_inf = (ph.gamma - 1) * (ph.qinf[4] - 0.5)

    def fn(x, y, z):
        r2 = x * x + y * y
        damp = 1.0 - np.exp(-(r2 - 0.25) * 8.0)
        u = damp * (1.0 + 0.02 * np.sin(2.0 * y))
        v = 0.02 * damp * np.exp(-((x - 1.5) ** 2 + y * y))
        rho = np.ones_like(x)
        return np.stack([rho, rho * u, rho * v, 0 * x, p_inf / (ph.gamma - 1) + 0.5 * rho * (u * u + v * v)])
    return I.pointwise_state(xyz, mi.orders, fn)


def full_sweep_for(orders):
    from paper_2210_03523_gb300 import inputs as I
    return I.full_sweep(np.asarray(orders).max(0))


# DRAM bytes per RK stage (the launches of one stage summed; the volume
# kernel the mean of a step's three stages, the mortar kernel a stage that
# reads the face traces, as all but the first of a replayed batch of steps
# do) from ncu captures of these kernels as they stand; the commands and the
# per-launch figures are in profiles/traffic_mortar_volume_pulse24mixed_pulse48mixed.md
MEASURED_TRAFFIC = {
    ("pulse48mixed", "mortar"): 2033.6e6, ("pulse48mixed", "volume"): 5362.5e6,
}
TRAFFIC_SOURCE = ("ncu dram__bytes_read.sum + dram__bytes_write.sum, "
                  "profiles/traffic_mortar_volume_pulse24mixed_pulse48mixed.md")


# ------------------------------------------------------------ algorithmic counts
def is_axis_aligned(mi):
    """Every element an axis-aligned box (its lattice edges parallel to the axes)."""
    if mi.geom_order != 1:
        return False
    g = np.asarray(mi.geom).reshape(mi.n_elem, 8, 3)
    for d, (a, b) in enumerate(((0, 1), (0, 2), (0, 4))):
        e = g[:, b] - g[:, a]
        off = np.delete(np.abs(e), d, axis=1)
        if np.any(off > 1e-12 * np.abs(e[:, d:d + 1])):
            return False
    return True


def volume_counts(orders, rk=True, axis_aligned=False, traces=True):
    """Algorithmic FP64 flops and HBM bytes of one volume-kernel launch (Euler,
    straight elements, fused RK stage).  Per node: primitive variables 12,
    Cartesian fluxes 16, contravariant fluxes 75, sum-factorised derivative
    10*sum_i(N_i+1), 1/J scaling 6, RK update 25 (axis_aligned: the
    contravariant fluxes are 15, the metric being diagonal); per face node of the
    element's own six faces: lift 15.  Bytes per node: q read 40, G read and
    write 80, q write 40 (RK) or R write 40; per face node 40 (F* read) and,
    in an RK stage with traces, 40 (the new state's face trace written for
    the next stage's mortars); per element 80 (metrics)."""
    o = np.asarray(orders, dtype=np.int64).reshape(-1, 3) + 1
    n = o.prod(1)
    faces = 2 * (o[:, 1] * o[:, 2] + o[:, 0] * o[:, 2] + o[:, 0] * o[:, 1])
    flops = (n * (134 + 10 * o.sum(1)) + 15 * faces).sum() - (0 if rk else (n * 25).sum())
    if axis_aligned:      # diagonal J a^i: the contravariant fluxes take 15 instead of 75
        flops -= (60 * n).sum()
    bytes_ = ((160 if rk else 80) * n + (80 if rk and traces else 40) * faces + 80).sum()
    return float(flops), float(bytes_)


# one Roe flux per mortar node (roe_t), counted operation by operation:
# through an axis-aligned unit normal e_d (every face of an axis-aligned box):
# 1/rho and sqrt(rho) from two rsqrt and four products 6, velocities 6,
# pressures 16, rho H and H 4, Roe weights 4, averaged velocity 9, averaged H
# 3, averaged rho 1, sound speed (|u~|^2 5, c~^2 3, rsqrt and three products
# 4) 12, jumps 3, wave strengths 8, eigenvalue products and sums 10, the
# tangential jump and u~ . du~ 5, mass flux 5, momentum fluxes 34, energy flux
# 14, the face-area factor 1/2 |J a| 1: 141.  Through a general unit normal
# the normal velocities and momenta (17), the full tangential jump (9 more)
# and the normal projections of the momentum flux (12 more) add 38: 179.
ROE_FLOPS_AXIS = 141
ROE_FLOPS_GENERAL = 179


def mortar_counts(mi, axis_aligned=False):
    """Algorithmic FP64 flops and HBM bytes of one mortar-kernel launch.

    For every interior face in the launch (on straight-sided Euler meshes the
    conforming faces too, with no interpolation) with la x lb and ra x rb
    nodes and mortar Ma x Mb = max per direction: interpolation of the 5
    trace variables up to the mortar, per side and tangential direction where
    the side is coarser (2 * 5 * taps flops per output node), one Roe flux per
    mortar node (ROE_FLOPS_AXIS on an axis-aligned box, else
    ROE_FLOPS_GENERAL), and the L2 projection back in the same passes
    reversed.  Bytes: each element-face node reads its 5-variable trace and
    writes 5 values of F*, 80 B."""
    roe = ROE_FLOPS_AXIS if axis_aligned else ROE_FLOPS_GENERAL
    o = np.asarray(mi.orders, dtype=np.int64).reshape(-1, 3) + 1
    nb = np.asarray(mi.neighbors).reshape(-1, 6)
    flops = bytes_ = 0.0
    for d in range(3):
        t0, t1 = (1, 2) if d == 0 else ((0, 2) if d == 1 else (0, 1))
        L = np.flatnonzero(nb[:, 2 * d + 1] >= 0)
        R = nb[L, 2 * d + 1]
        la, lb, ra, rb = o[L, t0], o[L, t1], o[R, t0], o[R, t1]
        Ma, Mb = np.maximum(la, ra), np.maximum(lb, rb)
        for a, b in ((la, lb), (ra, rb)):
            up_a, up_b = a != Ma, b != Mb
            # interpolation up (xi_a then xi_b) and projection down (the reverse)
            flops += (2 * 2 * 5 * a * Ma * b * up_a).sum() + (2 * 2 * 5 * b * Ma * Mb * up_b).sum()
            bytes_ += (80 * a * b).sum()
        flops += (roe * Ma * Mb).sum()
    return float(flops), float(bytes_)


# FP32 operations of the deviation-form Euler flux at one node of the tau
# sweep (tau_flux_nm): primitives rho, 1/rho, u' (12), u (3), u_f.u' and
# |u'|^2 (12), p' (9) = 38; flux deviations: momentum 27 + 3, energy 9 + 1 = 40.
TAU_FLUX_FLOPS = 78


def tau_counts(orders, sweep, axis_aligned=False):
    """Algorithmic FP32 flops of one isolated tau sweep (Euler): per element,
    the isolated R^P (per node: the flux deviations TAU_FLUX_FLOPS, the
    contravariant fluxes 75, or 15 on an axis-aligned box, the derivative
    10 sum(P_i+1), the 1/J scaling 6), then per applicable entry N:
    restriction of 10 fields in xi3, xi2, xi1 (2*10*(P_i+1) per output node of
    each pass; the xi3 / xi2 passes only when N3 / (N2,N3) change), the coarse
    isolated residual (as R^P) and the two norms (tau~ 5, |.| and max 10, J w
    and its products 3 + 5, max 5)."""
    o = np.asarray(orders, dtype=np.int64).reshape(-1, 3)
    sw = np.asarray(sweep, dtype=np.int64).reshape(-1, 3)
    node = TAU_FLUX_FLOPS + (15 if axis_aligned else 75) + 6
    total = 0.0
    for P in {tuple(r) for r in o}:
        cnt = int((o == P).all(1).sum())
        P1, P2, P3 = P
        nP = (P1 + 1) * (P2 + 1) * (P3 + 1)
        f = nP * (node + 10 * (P1 + P2 + P3 + 3))
        cur3 = cur2 = None
        for N1, N2, N3 in sw:
            if N1 > P1 or N2 > P2 or N3 > P3:
                continue
            if N3 != cur3:
                f += 20 * (P3 + 1) * (P1 + 1) * (P2 + 1) * (N3 + 1)
                cur3, cur2 = N3, None
            if N2 != cur2:
                f += 20 * (P2 + 1) * (P1 + 1) * (N2 + 1) * (N3 + 1)
                cur2 = N2
            nN = (N1 + 1) * (N2 + 1) * (N3 + 1)
            f += 20 * (P1 + 1) * nN
            f += nN * (node + 10 * (N1 + N2 + N3 + 3) + 28)
        total += cnt * f
    return total


# ------------------------------------------------------------ multi-rank
def max_over_ranks(x: float, world: int) -> float:
    """Largest value over all ranks (the job's time is its slowest rank's)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world: int, ndof: int, res_per_step: int, ms_per_step: float) -> float:
    """Whole-job DOF-residuals/s: every rank runs a replica of the workload, so
    the job processes world * ndof * res_per_step DOF-residuals per step."""
    return world * ndof * res_per_step / (ms_per_step * 1e-3)


# ------------------------------------------------------------ clocks sampling
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, nm in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def fp32_tau_check(m, q, sweep):
    """The FP32 sweep against the FP64 sweep on the same state (outside the
    timed regions): the largest |tau32 - tau64|, the FP32 value where FP64 is
    exactly zero (the FP32 noise floor), and the fraction of elements whose
    selection (approach 2, no jump rule) changes at each tau_max of the
    paper's range (Sec. 3.1)."""
    from paper_2210_03523_gb300 import dg
    try:
        m64, _ = m.tau_estimate(q, sweep, isolated=True, fp32=False, want=(True, False))
    except dg.DGError as e:       # FP64 tiles above the shared-memory limit (orders 8)
        return {"unavailable": str(e)}
    m32, _ = m.tau_estimate(q, sweep, isolated=True, fp32=True, want=(True, False))
    a64, a32 = m64.cpu().numpy(), m32.double().cpu().numpy()
    valid = a64 >= 0
    err = np.abs(a32 - a64)[valid]
    zero = valid & (a64 == 0.0)      # exact zeros in FP64 (elements the pulse has not reached)
    changed = {}
    for tm in (1e-3, 1e-2, 1e-1, 1.0):
        s64 = m.select_orders(m64, sweep, tm, 1, 8, 0)
        s32 = m.select_orders(m32, sweep, tm, 1, 8, 0)
        changed[f"{tm:g}"] = float((s64 != s32).any(axis=1).mean())
    return {"max_abs_err": float(err.max()), "map_max": float(a64[valid].max()),
            "max_abs_err_over_map_max": float(err.max() / a64[valid].max()),
            "fp32_noise_floor": float(a32[zero].max()) if zero.any() else None,
            "selection_changed_fraction": changed, "eps32": 2.0 ** -23}


def tau_sweep_timing(m, q, P, reps=5):
    """The isolated sweep over S = {N : 1 <= N_i <= P_i} and over the interior
    set {1..P_i - 1}^3, each in FP32 and FP64 (outside the timed regions; CUDA
    events over reps sweeps after one warm-up)."""
    import torch
    from paper_2210_03523_gb300 import dg, inputs as I
    P = np.asarray(P)
    out = {}
    for name, sw in (("full", I.full_sweep(P)), ("interior", I.full_sweep(np.maximum(P - 1, 1)))):
        for fp32 in (True, False):
            key = f"{name}_{'fp32' if fp32 else 'fp64'}"
            try:
                mn, mt = m.tau_estimate(q, sw, isolated=True, fp32=fp32)
            except dg.DGError as e:       # FP64 tiles above the shared-memory limit (orders 8)
                out[key] = {"unavailable": str(e)}
                continue
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(reps):
                m.tau_estimate(q, sw, isolated=True, fp32=fp32, map_new=mn, map_trad=mt)
            b.record()
            torch.cuda.synchronize()
            ms = a.elapsed_time(b) / reps
            out[key] = {"entries": int(len(sw)), "ms": ms, "elements_per_s": m.n_elem / (ms * 1e-3)}
    return out


def adjoint_timing(m, q, dt_adj, reps=10):
    """The adjoint on the bench mesh (outside the timed regions): one residual
    VJP and one RK3-step VJP (which recomputes the stage states), CUDA events
    over reps calls each, against the forward residual."""
    import torch
    from paper_2210_03523_gb300 import dg
    v = torch.randn(q.shape, dtype=torch.float64, device=q.device, generator=torch.Generator(q.device).manual_seed(1))
    out = torch.empty_like(q)
    lam = v.clone()
    r = torch.empty_like(q)

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps
    try:
        fwd = timed(lambda: m.residual(q, r))
        vjp = timed(lambda: m.residual_vjp(q, v, out))
        step = timed(lambda: m.rk_step_vjp(q, dt_adj, lam))
    except dg.DGError as e:
        return {"unavailable": str(e)}
    ndof = m.n_nodes
    return {"residual_ms": fwd, "residual_vjp_ms": vjp, "rk_step_vjp_ms": step,
            "vjp_over_residual": vjp / fwd, "vjp_dof_per_s": ndof / (vjp * 1e-3),
            "note": "dg_residual_vjp and dg_rk_step_vjp (FP64; Roe by a hand-written reverse sweep, the volume fluxes by Dual numbers)"}


# ------------------------------------------------------------ our arm
def measure(workload, args, steps, warmup, world, sample_clocks=True):
    """Set up one workload and time `steps` bench steps after `warmup` untimed
    ones (the timed region: no per-kernel events), then min(steps,
    PROFILE_STEPS) steps with CUDA events around every kernel (the profiled
    region: per-kernel shares and the rooflines).  Returns a dict of the
    mesh, its buffers and the timings."""
    import torch
    from paper_2210_03523_gb300 import dg, inputs as I

    dev = torch.cuda.current_device()
    stream = torch.cuda.current_stream()
    mi = I.workload(workload)
    m = dg.Mesh(mi)
    ndof = m.n_nodes
    xyz = m.coords().cpu().numpy()
    q0_h = initial_state(workload, mi, xyz)
    del xyz
    q0 = torch.from_numpy(q0_h).cuda()
    q = q0.clone()
    g = torch.zeros_like(q)
    # tile shapes per size class, timed on this mesh (setup, outside the timed regions)
    t_tune = time.perf_counter()
    tiles = m.tiles() if args.no_autotune else m.autotune(q0, reps=3)
    tune_s = time.perf_counter() - t_tune
    sweep = full_sweep_for(mi.orders)
    ns = sweep.shape[0]
    map_new = torch.zeros((m.n_elem, ns), dtype=torch.float32, device="cuda")
    map_trad = torch.zeros_like(map_new)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    ev = lambda: torch.cuda.Event(enable_timing=True)
    t_dev = torch.zeros(1, dtype=torch.float64, device="cuda")

    def advance():
        # the user-facing time loop: dg_advance runs the CFL steps as replays of cached CUDA graphs
        m.advance(q, g, t_dev, math.inf, CFL, max_steps=args.rk_per_step)

    def sweep_tau():
        m.tau_estimate(q, sweep, isolated=True, fp32=True, accumulate=True, map_new=map_new, map_trad=map_trad)

    def reset():
        q.copy_(q0)
        g.zero_()
        flush.fill_(1.0)       # evict the working set from L2 between timed steps

    for _ in range(warmup):
        reset()
        advance()
        sweep_tau()
    assert m.get_error() == 0, "non-physical state during warm-up"
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()

    # timed region: K steps, no per-kernel events
    clocks = ClockSampler(dev) if sample_clocks else None
    if clocks:
        clocks.start()
    launches0 = m.launch_count()
    starts, mids, ends = [ev() for _ in range(steps)], [ev() for _ in range(steps)], [ev() for _ in range(steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    for k in range(steps):
        reset()
        starts[k].record(stream)
        advance()
        mids[k].record(stream)
        sweep_tau()
        ends[k].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    launches = m.launch_count() - launches0
    clk = clocks.stop() if clocks else None
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    rk_ms = [s.elapsed_time(e) for s, e in zip(starts, mids)]
    tau_ms = [s.elapsed_time(e) for s, e in zip(mids, ends)]

    # profiled region: the same steps with CUDA events around every kernel
    # (launched one by one) for the per-kernel shares and the roofline
    psteps = min(steps, PROFILE_STEPS)
    m.profile_enable(True)
    prof_s, prof_e = [ev() for _ in range(psteps)], [ev() for _ in range(psteps)]
    for k in range(psteps):
        reset()
        prof_s[k].record(stream)
        advance()
        sweep_tau()
        prof_e[k].record(stream)
    torch.cuda.synchronize()
    prof_ms = statistics.mean(s.elapsed_time(e) for s, e in zip(prof_s, prof_e))
    kern = {name: m.profile_read(kid) for name, kid in dg.KERNELS.items()}
    m.profile_enable(False)
    err = m.get_error()
    assert err == 0, f"device error {err}"
    total_ms = max_over_ranks(float(sum(step_ms)), world)
    return {"mi": mi, "m": m, "q": q, "g": g, "q0_h": q0_h, "flush": flush, "t_dev": t_dev, "sweep": sweep,
            "map_new": map_new, "map_trad": map_trad, "advance": advance, "sweep_tau": sweep_tau,
            "ndof": ndof, "steps": steps, "ms_per_step": total_ms / steps, "rk_ms": rk_ms, "tau_ms": tau_ms,
            "prof_ms": prof_ms, "psteps": psteps, "kern": kern, "clk": clk, "launches": launches,
            "tiles": tiles, "tune_s": tune_s}


def rooflines(workload, r, sm_mhz):
    """The rooflines of a measured workload: the volume and mortar kernels
    against the FP64 peak (algorithmic flops of the mesh at hand: on an
    axis-aligned box the diagonal-metric volume count and the axis-normal Roe
    count, the general counts beside them), the tau kernel against the FP32
    peak, and every kernel kind's share of the profiled step."""
    mi, kern = r["mi"], r["kern"]
    fp64_peak = N_SM * FP64_FMA_PER_CLK_PER_SM * 2 * sm_mhz * 1e6 / 1e12
    hbm_peak, hbm_src = _peaks()
    axis = is_axis_aligned(mi)
    stages = r["psteps"] * r["rk_steps"] * 3        # both kernels launch once per size class: time per RK stage
    vol_ms, _ = kern["volume"]
    vflops, vbytes = volume_counts(mi.orders, rk=True, axis_aligned=axis)
    vflops_gen, _ = volume_counts(mi.orders, rk=True, axis_aligned=False)
    vol_avg_s = vol_ms / stages * 1e-3
    mor_ms, mor_n = kern["mortar"]
    mflops, mbytes = mortar_counts(mi, axis_aligned=axis)
    mflops_gen, _ = mortar_counts(mi, axis_aligned=False)
    mor_avg_s = (mor_ms / stages * 1e-3) if mor_n else None

    def fp64_roofline(name, flops, flops_gen, bytes_, avg_s, kind):
        traffic = MEASURED_TRAFFIC.get((workload, kind))
        return {"kernel": name, "bound": "alu", "achieved": flops / avg_s / 1e12, "peak": fp64_peak,
                "unit": "TFLOP/s", "frac": flops / avg_s / 1e12 / fp64_peak,
                "peak_source": f"FP64: {N_SM} SMs x {FP64_FMA_PER_CLK_PER_SM} DFMA/clk x 2 x median SM clock "
                               f"{sm_mhz:.0f} MHz (recipe nominal 1.25 TFLOP/s at 2070 MHz)",
                "flop_count": ("axis-aligned box: the operations the kernel performs there (diagonal metric, "
                               "axis-normal Roe without the tangential normal projection)" if axis else
                               "general affine count"),
                "frac_general_count": flops_gen / avg_s / 1e12 / fp64_peak,
                "traffic": traffic, "traffic_source": TRAFFIC_SOURCE if traffic else None,
                "algorithmic_flops_per_stage": flops, "algorithmic_bytes_per_stage": bytes_,
                "traffic_over_algorithmic_bytes": traffic / bytes_ if traffic else None,
                "time_from": "CUDA events around each launch, profiled region; the launches of one RK stage "
                             "(one per tile-size class) summed",
                "avg_stage_ms": avg_s * 1e3, "hbm_achieved_gbs": bytes_ / avg_s / 1e9, "hbm_peak_gbs": hbm_peak,
                "hbm_frac": bytes_ / avg_s / 1e9 / hbm_peak, "hbm_peak_source": hbm_src}

    vol_roof = fp64_roofline("volume_kernel (FP64 residual + fused RK3 stage)", vflops, vflops_gen, vbytes,
                             vol_avg_s, "volume")
    mor_roof = fp64_roofline("mortar_kernel (p-nonconforming and conforming interior faces)", mflops, mflops_gen,
                             mbytes, mor_avg_s, "mortar") if mor_n else None
    dominant = mor_roof if (mor_roof and mor_ms > vol_ms) else vol_roof
    others = [x for x in (vol_roof, mor_roof) if x is not None and x is not dominant]
    kernels_json = {k: {"launches": n, "total_ms": round(ms, 3), "share": None} for k, (ms, n) in kern.items() if n}
    kernels_json["_region"] = {"ms_per_step": r["prof_ms"], "steps": r["psteps"],
                               "note": "a second timed region of the same steps, kernels launched one by one with "
                                       "CUDA events around each"}
    ktot = sum(v["total_ms"] for k, v in kernels_json.items() if not k.startswith("_"))
    for k, v in kernels_json.items():
        if not k.startswith("_"):
            v["share"] = round(v["total_ms"] / ktot, 4) if ktot else None
    tau_k_ms, tau_k_n = kern["tau"]
    tflops = tau_counts(mi.orders, r["sweep"], axis_aligned=axis)
    tflops_gen = tau_counts(mi.orders, r["sweep"], axis_aligned=False)
    fp32_peak = N_SM * FP32_FMA_PER_CLK_PER_SM * 2 * sm_mhz * 1e6 / 1e12
    tau_s = tau_k_ms / r["psteps"] * 1e-3 if tau_k_n else None      # one sweep per step
    tau_roof = {"kernel": "tau_euler_kernel<float> + tau_euler_prologue_kernel" if mi.phys.eqs == 0 else
                          "tau_kernel<float> + tau_prologue_kernel (Navier-Stokes)", "bound": "alu",
                "achieved": tflops / tau_s / 1e12 if tau_s else None, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": tflops / tau_s / 1e12 / fp32_peak if tau_s else None, "sweep_ms": tau_s * 1e3 if tau_s else None,
                "algorithmic_flops_per_sweep": tflops,
                "frac_general_count": tflops_gen / tau_s / 1e12 / fp32_peak if tau_s else None,
                "flop_count": ("axis-aligned box: diagonal contravariant fluxes" if axis else "general affine count")
                              + "; FP32 deviation-form fluxes",
                "peak_source": f"FP32: {N_SM} SMs x {FP32_FMA_PER_CLK_PER_SM} FFMA/clk x 2 x {sm_mhz:.0f} MHz"}
    return dominant, others, tau_roof, kernels_json


def run_gb300(args, rank, world):
    import torch
    from paper_2210_03523_gb300 import dg

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)
    r = measure(args.workload, args, args.steps, args.warmup, world)
    r["rk_steps"] = args.rk_per_step
    m, q, g, mi, sweep = r["m"], r["q"], r["g"], r["mi"], r["sweep"]
    map_new, map_trad, flush = r["map_new"], r["map_trad"], r["flush"]
    ndof, ms_per_step = r["ndof"], r["ms_per_step"]
    res_per_step = 3 * args.rk_per_step
    value = job_value(world, ndof, res_per_step, ms_per_step)
    clk = r["clk"]
    sm_mhz = (clk or {}).get("sm_mhz") or 2070.0
    dominant, others, tau_roof, kernels_json = rooflines(args.workload, r, sm_mhz)

    # end to end through the C ABI with host buffers (dg_step_host): every
    # step copies the initial state from page-locked host memory, advances
    # it, runs the FP32 sweep and reads the state and both maps back, all
    # inside the library call
    esteps = min(args.steps, PROFILE_STEPS)
    q_pin = torch.from_numpy(r["q0_h"]).pin_memory()
    out_q = torch.empty(q.numel(), dtype=torch.float64).pin_memory()
    out_mn = torch.empty(map_new.shape, dtype=torch.float32).pin_memory()
    out_mt = torch.empty(map_trad.shape, dtype=torch.float32).pin_memory()
    sweep = r["sweep"]

    def step_host():
        m.step_host(q_pin, out_q, 0.0, math.inf, CFL, args.rk_per_step, sweep, isolated=True, fp32=True,
                    accumulate=True, map_new=out_mn, map_trad=out_mt)
    step_host()   # the library's device copies and their CUDA graphs are made here, outside the timed region
    e2e_s, e2e_e = [ev() for _ in range(esteps)], [ev() for _ in range(esteps)]
    torch.cuda.synchronize()
    for k in range(esteps):
        flush.fill_(1.0)
        e2e_s[k].record(stream)
        step_host()
        e2e_e[k].record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(sum(s.elapsed_time(e) for s, e in zip(e2e_s, e2e_e)) / esteps, world)
    h2d = q.numel() * 8
    d2h = q.numel() * 8 + 2 * map_new.numel() * 4
    del q_pin, out_q, out_mn, out_mt

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "description": workload_desc(args.workload), "n_elem": m.n_elem,
                   "ndof": ndof, "scalar_dof": 5 * ndof, "rk_steps_per_step": args.rk_per_step,
                   "residual_evals_per_step": res_per_step, "tau_sweep": {"entries": int(len(sweep)), "dtype": "f32",
                                                                         "form": "isolated, new + traditional"},
                   "l2": "flushed between timed steps (256 MiB write)", "parallelism": f"replicas x{world}"},
        "tau_elements_per_s": world * m.n_elem / (statistics.mean(r["tau_ms"]) * 1e-3),
        "rk_dof_residuals_per_s": world * ndof * res_per_step / (statistics.mean(r["rk_ms"]) * 1e-3),
        "stated_error": {"residual_rk_fp64_rel": 1e-12, "tau_fp32_abs": TAU_FP32_BOUND,
                         "checked_by": "tests/test_gpu_parity.py, tests/test_gpu_tau_production.py"},
        "roofline": dominant,
        "roofline_other_kernels": others,
        "tau_roofline": tau_roof,
        "kernels": kernels_json,
        "e2e": {"value": job_value(world, ndof, res_per_step, e2e_ms), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms, "steps": esteps,
                "path": "dg_step_host (C ABI, host buffers): page-locked host state -> device -> dg_advance "
                        "(CUDA-graph step batches) -> dg_tau_estimate -> page-locked host state and maps"},
        "gpu_launches": int(r["launches"]),
        "clocks": clk,
        "autotune": {"enabled": not args.no_autotune, "seconds": r["tune_s"], "vol_budget": r["tiles"]["vol_budget"],
                     "mortar_budget": r["tiles"]["mortar_budget"],
                     "volume_launch_ms_after_class": r["tiles"]["vol_ms"],
                     "volume_launch_ms_before_class": r["tiles"]["vol_ms_default"],
                     "face_launch_ms_after_class": r["tiles"]["mortar_ms"],
                     "face_launch_ms_before_class": r["tiles"]["mortar_ms_default"],
                     "method": "coordinate descent over size classes, whole production launch timed",
                     "classes": "elements of <= 27 / 125 / 343 / more nodes; mortars of <= 9 / 25 / 49 / more nodes"},
    }
    if not args.no_extras:
        # static p-adaptation selection on the accumulated map (Sec. 2.4, approach 2,
        # jump condition (b)); timed once, outside the step
        t0 = time.perf_counter()
        sel = m.select_orders(map_new, sweep, 1.0, 1, 8, 2)
        line["select_orders"] = {"ms": (time.perf_counter() - t0) * 1e3, "tau_max": 1.0, "jump_rule": "N_i >= N_j - 1",
                                 "mean_order_after": float(np.mean(sel)), "synchronous_host_call": True}
        line["fp32_tau_check"] = fp32_tau_check(m, q, sweep)
        line["tau_sweep_timing"] = tau_sweep_timing(m, q, np.asarray(mi.orders).reshape(-1, 3).max(0))
        line["adjoint"] = adjoint_timing(m, q, dt_adj=m.max_dt(q, CFL))

    partner = UNIFORM_PARTNER.get(args.workload)
    if partner and not args.no_uniform:
        # the plain uniform-order FP64 path at the same expected nodes per element, same step
        mixed_tau_eps = line["tau_elements_per_s"]
        m.close()
        del r, m, q, g, map_new, map_trad
        torch.cuda.empty_cache()
        u = measure(partner, args, min(args.steps, PROFILE_STEPS), 3, world, sample_clocks=False)
        u["rk_steps"] = args.rk_per_step
        udom, uoth, utau, ukern = rooflines(partner, u, sm_mhz)
        uval = job_value(world, u["ndof"], res_per_step, u["ms_per_step"])
        pick = lambda roofs, key: next((x for x in roofs if x and x["kernel"].startswith(key)), None)
        line["vs_uniform"] = {
            "workload": partner, "description": workload_desc(partner), "ndof": u["ndof"], "steps": u["steps"],
            "dof_residuals_per_s": uval,
            "rk_dof_residuals_per_s": world * u["ndof"] * res_per_step / (statistics.mean(u["rk_ms"]) * 1e-3),
            "tau_elements_per_s": world * u["m"].n_elem / (statistics.mean(u["tau_ms"]) * 1e-3),
            "tau_sweep_entries": int(len(u["sweep"])),
            "mixed_over_uniform": {"dof_residuals_per_s": value / uval,
                                   "tau_elements_per_s": mixed_tau_eps / (
                                       world * u["m"].n_elem / (statistics.mean(u["tau_ms"]) * 1e-3))},
            "dominant_kernel": {"kernel": udom["kernel"], "frac": udom["frac"]},
            "volume_frac": (pick([udom] + uoth, "volume") or {}).get("frac"),
            "mortar_frac": (pick([udom] + uoth, "mortar") or {}).get("frac"),
            "mixed_dominant_kernel": {"kernel": dominant["kernel"], "frac": dominant["frac"]},
            "mixed_volume_frac": (pick([dominant] + others, "volume") or {}).get("frac"),
            "mixed_mortar_frac": (pick([dominant] + others, "mortar") or {}).get("frac"),
            "kernels": ukern, "tau_roofline_frac": utau["frac"],
            "note": "same step (RK3 steps at CFL 0.5 + one FP32 isolated tau sweep over its own S), timed after the "
                    "mixed-order run on the same GPU",
        }
        u["m"].close()
    return line


# ------------------------------------------------------------ the oracle
def _oracle_setup(workload):
    import oracle
    from paper_2210_03523_gb300 import inputs as I
    mi = I.workload(workload)
    om = oracle.Mesh(mi)
    q = initial_state(workload, mi, om.coords())
    return mi, om, q


def _tau_sample_mesh(workload, mi, n=8):
    """The isolated tau sweep is element-local: a sample of the workload's
    elements is an n^3 block of them (same element size, orders and state
    recipe), as its own mesh."""
    from paper_2210_03523_gb300 import inputs as I
    import oracle
    if workload in ("pulse4", "cylinder"):
        return None
    nx = round(mi.n_elem ** (1 / 3))
    if nx <= n:
        return None
    o = np.asarray(mi.orders).reshape(nx, nx, nx, 3)[:n, :n, :n].reshape(-1, 3)   # e = i + nx (j + nx k)
    o = np.ascontiguousarray(o)
    sub = I.box_mesh(n, lo=-1.0, hi=-1.0 + n * 2.0 / nx, orders=o, phys=mi.phys)
    om = oracle.Mesh(sub)
    return sub, om, initial_state(workload, sub, om.coords())


def cpu_baseline(workload):
    """The oracle (as it stands) on the host cores, on a bounded sample of the
    workload: residual evaluations of the full mesh (2 for meshes above 1e7
    nodes, else 4 RK3 steps), and one FP64 isolated tau sweep over the full
    set S (of an 8^3 block of the elements when the mesh is larger)."""
    mi, om, q = _oracle_setup(workload)
    big = om.n_nodes > 10_000_000
    t0 = time.perf_counter()
    if big:
        n_res = 2
        for _ in range(n_res):
            om.residual(q)
        what = f"{n_res} FP64 residuals of the full mesh"
    else:
        n_res = 12
        G = np.zeros_like(q)
        dt = om.max_dt(q, CFL)
        for _ in range(4):
            om.rk_step(q, G, dt)
        what = "4 RK3 steps (12 FP64 residuals) of the full mesh"
    rk_s = time.perf_counter() - t0
    ndof = om.n_nodes
    sample = _tau_sample_mesh(workload, mi) if big else None
    if sample is not None:
        _, omt, qt = sample
        tau_what = f"one FP64 isolated tau sweep over S of an 8^3 block ({omt.n_elem} elements)"
    else:
        omt, qt = om, q
        tau_what = "one FP64 isolated tau sweep over S of the full mesh"
    sweep = full_sweep_for(np.asarray(mi.orders))
    t2 = time.perf_counter()
    omt.tau(qt, sweep)
    tau_s = time.perf_counter() - t2
    return {"value": ndof * n_res / rk_s, "unit": UNIT, "cores": int(os.environ.get("OMP_NUM_THREADS", os.cpu_count())),
            "kind": "oracle", "sample": f"{workload}: {what} + {tau_what}; OpenMP over elements (schedule guided)",
            "tau_elements_per_s": omt.n_elem / tau_s, "seconds": rk_s + tau_s}


def run_reference(args):
    """The reference arm: the oracle on the host cores, each step a bounded
    sample of the workload (FP64 residuals of the full mesh: 1 per step above
    1e7 nodes, else 2 RK3 steps), timed on the host clock."""
    mi, om, q0 = _oracle_setup(args.workload)
    big = om.n_nodes > 10_000_000
    steps_ms = []
    for k in range(args.warmup + args.steps):
        q = q0.copy()
        t0 = time.perf_counter()
        if big:
            om.residual(q)
            n_res = 1
        else:
            G = np.zeros_like(q)
            dt = om.max_dt(q, CFL)
            for _ in range(2):
                om.rk_step(q, G, dt)
            n_res = 6
        if k >= args.warmup:
            steps_ms.append((time.perf_counter() - t0) * 1e3)
    ndof = om.n_nodes
    ms = statistics.mean(steps_ms)
    value = ndof * n_res / (ms * 1e-3)
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count()))
    sample = (f"{args.workload}: each step = {n_res} FP64 residual{'s' if n_res > 1 else ''} of the full mesh"
              + ("" if big else " (2 RK3 steps)"))
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": args.workload, "description": workload_desc(args.workload), "ndof": ndof},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def developed_cylinder(args, mi):
    """A developed shedding flow on the cylinder mesh at the orders of mi: from
    the free stream slowed near the wall plus an off-axis vortex (it breaks the
    symmetry), advanced at the lower orders (develop_order, develop_order, 1)
    to t = develop (shedding is established by t ~ 45 at Re 100), raised to
    mi's orders (dg_set_orders: interpolation) and settled for `settle` time
    units.  Returns (mesh at mi's orders, device state, time, wall seconds)."""
    import torch
    from paper_2210_03523_gb300 import dg, inputs as I
    t_wall = time.perf_counter()
    ph = mi.phys
    lo = np.tile(np.array([args.develop_order, args.develop_order, 1], dtype=np.int32), (mi.n_elem, 1))
    m = dg.Mesh(mi.with_orders(lo))
    xyz = m.coords().cpu().numpy()
    p_inf = (ph.gamma - 1) * (ph.qinf[4] - 0.5)

    def fn(x, y, z):
        r2 = x * x + y * y
        damp = 1.0 - np.exp(-(r2 - 0.25) * 8.0)
        g = 0.5 * np.exp(-((x - 1.5) ** 2 + (y - 0.4) ** 2) / 0.25)
        u = damp * (1.0 - g * (y - 0.4) / 0.5)
        v = damp * g * (x - 1.5) / 0.5
        rho = np.ones_like(x)
        return np.stack([rho, rho * u, rho * v, 0 * x, p_inf / (ph.gamma - 1) + 0.5 * rho * (u * u + v * v)])
    q = torch.from_numpy(I.pointwise_state(xyz, lo, fn)).cuda()
    g = torch.zeros_like(q)
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    m.advance(q, g, t, args.develop, CFL)
    q = m.set_orders(np.asarray(mi.orders, dtype=np.int32).reshape(-1, 3), q)
    g = torch.zeros_like(q)
    m.advance(q, g, t, args.develop + args.settle, CFL)
    torch.cuda.synchronize()
    assert m.get_error() == 0
    return m, q, float(t.item()), time.perf_counter() - t_wall


def run_static_cylinder(args):
    """The paper's second case end to end on the GPU (Fig. 2, Sec. 3.3): the
    cylinder mesh at uniform P = (6,6,1) is advanced for t_est with 10
    estimation stages (FP32 isolated tau, new form, F_max), the orders are
    selected among N <= P (approach 2, jump condition N_i >= N_j - 1; the
    single spanwise element at N_3 = 1 leaves nothing to extrapolate from in
    that direction), the state projected, and the adapted mesh
    (p-nonconforming faces on a curved Navier-Stokes mesh) advanced for
    t_post.  The uniform-order run continues from the same state over the
    same interval and gives the reference drag and time.  With --develop T the
    run starts from a developed shedding flow (developed_cylinder) at t = T +
    settle, else from the bench's initial field at t = 0.  Timed with CUDA
    events; the drag is sampled 20 times over the post interval."""
    import torch
    from paper_2210_03523_gb300 import adapt, dg, inputs as I
    mi = I.workload("cylinder")
    dev_s = None
    if args.develop > 0:
        mu, q_start, t0, dev_s = developed_cylinder(args, mi)
        if args.save_state:
            mu.save_state(args.save_state, q_start, t0)
        qh = q_start
    else:
        mu = dg.Mesh(mi)
        qh = initial_state("cylinder", mi, mu.coords().cpu().numpy())
        t0 = 0.0
    P = np.asarray(mi.orders).reshape(-1, 3).max(0)
    sweep = I.full_sweep(P)
    dt_e = args.t_est / 10.5                  # ten estimation stages end before t0 + t_est
    n_samples = 20

    def events():
        return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def segment(m, q, ta, tb):
        g = torch.zeros_like(q)
        t = torch.full((1,), ta, dtype=torch.float64, device=q.device)
        drags, steps = [], 0
        a, b = events()
        torch.cuda.synchronize()
        a.record()
        for k in range(1, n_samples + 1):
            steps += m.advance(q, g, t, ta + (tb - ta) * k / n_samples, CFL, count=True)
            drags.append(m.wall_force(q)[0].clone())
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b), steps, torch.stack(drags).cpu().numpy()

    ndof_u = int(mu.n_nodes)
    # static adaptation: estimation stages, selection, projection (timed as a whole)
    a, b = events()
    torch.cuda.synchronize()
    a.record()
    res = adapt.static_adaptation(mi, qh, t0=t0, t_est=t0 + args.t_est, dt_e=dt_e, t_final=t0 + args.t_est, cfl=CFL,
                                  sweep=sweep, tau_max=args.tau_max, n_min=1, n_max=int(P.max()), jump_rule=2,
                                  form="new", isolated=True, fp32=True, keep_estimation_state=True)
    b.record()
    torch.cuda.synchronize()
    est_ms = a.elapsed_time(b)
    ma, qa = res["mesh"], res["q"]
    t1 = res["t"]
    # the uniform reference continues from the state the estimation ended with
    ref_ms, ref_steps, ref_drag = segment(mu, res["q_est"], t1, t1 + args.t_post)
    ad_ms, ad_steps, ad_drag = segment(ma, qa, t1, t1 + args.t_post)
    assert ma.get_error() == 0 and mu.get_error() == 0
    ndof_a = int(ma.n_nodes)
    # NDOF the same accumulated map gives at other thresholds
    ndof_at = {}
    for tm in (1e2, 10.0, 1.0, 0.1, 0.01):
        o = ma.select_orders(res["total"], sweep, tm, 1, int(P.max()), 2)
        ndof_at[f"{tm:g}"] = int(np.prod(o + 1, axis=1).sum())
    o = res["orders"]
    dref = np.abs(ref_drag).mean()
    value = ndof_a * 3 * ad_steps / (ad_ms * 1e-3)
    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": ad_steps, "warmup": 0,
        "ms_per_step": ad_ms / max(ad_steps, 1), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": "cylinder_static",
                   "description": "static p-adaptation of the cylinder (Re=100, Ma=0.2, 40x24x1 curved O-grid, "
                                  "P=(6,6,1)): 10 FP32 tau estimations over t_est, selection, projection, then "
                                  "t_post on the adapted mesh against the uniform mesh",
                   "start": (f"developed shedding flow: P=({args.develop_order},{args.develop_order},1) to "
                             f"t={args.develop:g}, raised to P=(6,6,1), settled to t={t0:g}") if args.develop > 0
                   else "the bench's initial field at t=0",
                   "t0": t0, "t_est": args.t_est, "dt_e": dt_e, "t_post": args.t_post,
                   "tau_max_new_form": args.tau_max, "sweep_entries": int(len(sweep)), "selection": "among the sweep, N <= P"},
        "static_adaptation": {
            "development_s": dev_s,
            "n_estimates": res["n_estimates"], "estimation_and_adaptation_ms": est_ms,
            "estimation_rk_steps": res["steps"][0],
            "ndof_uniform": ndof_u, "ndof_adapted": ndof_a, "ndof_ratio": ndof_a / ndof_u,
            "ndof_at_tau_max": ndof_at,
            "orders_histogram": {f"{i}": int(c) for i, c in enumerate(np.bincount(o[:, :2].ravel(), minlength=9))},
            "post_interval": {"uniform_ms": ref_ms, "adapted_ms": ad_ms, "speedup": ref_ms / ad_ms,
                              "uniform_steps": ref_steps, "adapted_steps": ad_steps,
                              "uniform_dof_residuals_per_s": ndof_u * 3 * ref_steps / (ref_ms * 1e-3),
                              "adapted_dof_residuals_per_s": value},
            "drag": {"uniform_mean": float(ref_drag.mean()), "adapted_mean": float(ad_drag.mean()),
                     "mean_rel_diff": float(abs(ad_drag.mean() - ref_drag.mean()) / dref),
                     "max_rel_diff": float(np.abs(ad_drag - ref_drag).max() / dref),
                     "uniform_range": [float(ref_drag.min()), float(ref_drag.max())]},
        },
    }


def run_dynamic_cylinder(args):
    """The dynamic strategy (Fig. 1) on the cylinder: from uniform P = (6,6,1)
    every dt_e the state is re-estimated (FP32 isolated tau, new form, over
    every N <= the current maximum orders), re-selected (approach 2, N_i >=
    N_j - 1, orders fall by at most one per stage, Sec. 3.3) and projected,
    up to t_final; NDOF_dyn is the step-weighted mean NDOF (Sec. 3.3).  A
    uniform-order run over the same interval gives the reference time and the
    final drag."""
    import torch
    from paper_2210_03523_gb300 import adapt, dg, inputs as I
    mi = I.workload("cylinder")
    mu = dg.Mesh(mi)
    qh = initial_state("cylinder", mi, mu.coords().cpu().numpy())
    P = int(np.asarray(mi.orders).reshape(-1, 3).max())
    T, dt_e = args.t_final, args.t_final / args.stages

    def events():
        return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    qu = torch.from_numpy(qh).cuda()
    g = torch.zeros_like(qu)
    t = torch.zeros(1, dtype=torch.float64, device=qu.device)
    a, b = events()
    torch.cuda.synchronize()
    a.record()
    steps_u = mu.advance(qu, g, t, T, CFL, count=True)
    b.record()
    torch.cuda.synchronize()
    uni_ms = a.elapsed_time(b)
    drag_u = float(mu.wall_force(qu)[0])
    a, b = events()
    torch.cuda.synchronize()
    a.record()
    res = adapt.dynamic_adaptation(mi, qh, t0=0.0, dt_e=dt_e, t_final=T, cfl=CFL,
                                   sweep=lambda o: I.full_sweep(np.asarray(o).reshape(-1, 3).max(0)),
                                   tau_max=args.tau_max, n_min=1, n_max=P, jump_rule=2, max_decrease=1, form="new",
                                   isolated=True, fp32=True)
    b.record()
    torch.cuda.synchronize()
    dyn_ms = a.elapsed_time(b)
    ma = res["mesh"]
    drag_a = float(ma.wall_force(res["q"])[0])
    assert ma.get_error() == 0 and mu.get_error() == 0
    hist = [int(np.prod(h + 1, axis=1).sum()) for h in res["history"]]
    value = res["ndof_dyn"] * 3 * res["steps"] / (dyn_ms * 1e-3)
    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": res["steps"], "warmup": 0,
        "ms_per_step": dyn_ms / max(res["steps"], 1), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "cylinder_dynamic",
                   "description": "dynamic p-adaptation of the cylinder (Re=100, Ma=0.2, 40x24x1 curved O-grid, "
                                  "from P=(6,6,1)): re-estimated and re-adapted every dt_e up to t_final, against "
                                  "the uniform mesh",
                   "t_final": T, "dt_e": dt_e, "tau_max_new_form": args.tau_max, "max_decrease": 1},
        "dynamic_adaptation": {
            "stages": len(res["history"]), "ndof_uniform": int(mu.n_nodes), "ndof_dyn": res["ndof_dyn"],
            "ndof_final": res["ndof"], "ndof_after_each_adaptation": hist,
            "uniform_ms": uni_ms, "dynamic_ms": dyn_ms, "speedup": uni_ms / dyn_ms,
            "uniform_steps": steps_u, "dynamic_steps": res["steps"],
            "final_drag": {"uniform": drag_u, "dynamic": drag_a, "rel_diff": abs(drag_a - drag_u) / abs(drag_u)},
            "timing_note": "the dynamic time includes every estimation, selection, projection and mesh rebuild",
            "stage_timing_s": {k: [round(x, 5) for x in v] for k, v in res["timing"].items()},
            "rebuild_share": sum(res["timing"]["rebuild_s"]) / (dyn_ms * 1e-3),
            "estimate_select_share": sum(res["timing"]["estimate_select_s"]) / (dyn_ms * 1e-3),
            "rebuild_note": "dg_set_orders (synchronous, once per stage): the projection, the offsets, the curved "
                            "metrics at the new orders, the order buckets and the face classification and shape "
                            "sort on the device; the host tiles the sorted buckets and shape groups into work items "
                            "and batches",
        },
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD,
                    choices=["pulse16mixed", "pulse4", "pulse32mixed", "pulse48mixed", "pulse48uniform", "pulse24mixed",
                             "cylinder", "cylinder_static", "cylinder_dynamic"])
    ap.add_argument("--t-est", type=float, default=0.3, help="cylinder_static: estimation time")
    ap.add_argument("--t-post", type=float, default=0.3, help="cylinder_static: time advanced after adaptation")
    ap.add_argument("--develop", type=float, default=0.0,
                    help="cylinder_static: start from a shedding flow developed to this time (0: the initial field)")
    ap.add_argument("--develop-order", type=int, default=4, help="cylinder_static: orders of the development run")
    ap.add_argument("--settle", type=float, default=1.0, help="cylinder_static: time at P after raising the orders")
    ap.add_argument("--save-state", default="", help="cylinder_static: write the developed state (dg_state_write)")
    ap.add_argument("--tau-max", type=float, default=1.0, help="cylinder_static/_dynamic: threshold, new-form map")
    ap.add_argument("--t-final", type=float, default=0.6, help="cylinder_dynamic: end time")
    ap.add_argument("--stages", type=int, default=10, help="cylinder_dynamic: adaptation stages up to t_final")
    ap.add_argument("--rk-per-step", type=int, default=RK_PER_STEP)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default 256-node tiles")
    ap.add_argument("--no-uniform", action="store_true", help="skip the uniform-order partner run")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the e2e-independent extras (FP32 check, sweep timings, adjoint, selection)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return 0
        print(json.dumps(run_reference(args)), flush=True)
        return 0

    if args.workload in ("cylinder_static", "cylinder_dynamic"):     # one GPU; end-to-end adaptation runs
        if rank == 0:
            run = run_static_cylinder if args.workload == "cylinder_static" else run_dynamic_cylinder
            print(json.dumps(run(args)), flush=True)
        return 0
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    line = run_gb300(args, rank, world)
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(args.workload)
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
