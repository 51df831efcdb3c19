"""The p-adaptation support through the C ABI against the oracle:
dg_advance (CFL-adaptive RK3 to a given time, CUDA-graph batches),
dg_tau_extrapolate (Sec. 2.3-2.4), dg_select_orders with the bounded
decrease (Sec. 3.3), and the static / dynamic drivers (Figs. 2 and 1)."""
import math

import numpy as np
import pytest

from paper_2210_03523_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_03523_gb300 import build
    build.build()
    return torch


def _case(nx=3, lo=2, hi=5, seed=3, width=0.35):
    import oracle
    ph = I.pulse_physics(mach=0.4)
    mi = I.box_mesh(nx, orders=I.random_orders(nx ** 3, lo, hi, seed), phys=ph)
    om = oracle.Mesh(mi)
    q = I.pulse_state(om.coords(), mi.orders, ph, width=width, center=(-0.2, -0.3, 0.1))
    return mi, om, q


def _close(a, b, orders, tol):
    """per variable: max |a - b| <= tol * the state scale of that variable"""
    from oracle_helpers import state_scale
    a, b = np.asarray(a), np.asarray(b)
    off = I.node_offsets(orders)
    sc = state_scale(b, off)
    for e in range(len(off) - 1):
        n = off[e + 1] - off[e]
        d = np.abs(a[5 * off[e]:5 * off[e + 1]] - b[5 * off[e]:5 * off[e + 1]]).reshape(5, n).max(1)
        if np.any(d > tol * sc):
            return False
    return True


def test_advance_infinite_end_equals_the_step_loop(torch_cuda):
    """t_end = inf: max_steps plain CFL steps, bitwise the dg_max_dt +
    dg_rk_step loop; graph replay bitwise the eager launches."""
    torch = torch_cuda
    from paper_2210_03523_gb300 import dg
    mi, om, q0 = _case()
    m = dg.Mesh(mi)
    qa = torch.from_numpy(q0).cuda()
    ga = torch.zeros_like(qa)
    dt = torch.empty(1, dtype=torch.float64, device="cuda")
    for _ in range(37):
        m.max_dt(qa, 0.5, dt)
        m.rk_step(qa, ga, dt)
    for eager in (True, False):
        qb = torch.from_numpy(q0).cuda()
        gb = torch.zeros_like(qb)
        t = torch.zeros(1, dtype=torch.float64, device="cuda")
        n = m.advance(qb, gb, t, math.inf, 0.5, max_steps=37, eager=eager, count=True)
        assert n == 37
        assert torch.equal(qa, qb), eager
    assert m.get_error() == 0


def test_advance_to_time_matches_oracle(torch_cuda):
    torch = torch_cuda
    from paper_2210_03523_gb300 import dg
    mi, om, q0 = _case()
    m = dg.Mesh(mi)
    q = torch.from_numpy(q0).cuda()
    g = torch.zeros_like(q)
    t = torch.full((1,), 0.05, dtype=torch.float64, device="cuda")
    n = m.advance(q, g, t, 0.0975, 0.6, count=True)
    qo, Go = q0.copy(), np.zeros_like(q0)
    to, no = om.advance(qo, Go, 0.6, 0.05, 0.0975)
    assert t.item() == 0.0975 == to and n == no > 3
    assert _close(q.cpu().numpy(), qo, mi.orders, 1e-12)
    # already there: nothing happens
    q_before = q.clone()
    assert m.advance(q, g, t, 0.0975, 0.6, count=True) == 0 and torch.equal(q, q_before)
    # max_steps stops early
    t2 = torch.zeros(1, dtype=torch.float64, device="cuda")
    assert m.advance(q, g, t2, 10.0, 0.6, max_steps=5, count=True) == 5 and 0 < t2.item() < 10.0


def test_advance_launch_count_and_graph_reuse(torch_cuda):
    torch = torch_cuda
    from paper_2210_03523_gb300 import dg
    mi, om, q0 = _case()
    m = dg.Mesh(mi)
    q = torch.from_numpy(q0).cuda()
    g = torch.zeros_like(q)
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    m.advance(q, g, t, math.inf, 0.5, max_steps=1)      # eager warm-up step
    l0 = m.launch_count()
    m.advance(q, g, t, math.inf, 0.5, max_steps=1, eager=True)
    per_step = m.launch_count() - l0
    l1 = m.launch_count()
    m.advance(q, g, t, math.inf, 0.5, max_steps=64)     # two replays of a 32-step graph
    assert m.launch_count() - l1 == 64 * per_step


@pytest.mark.parametrize("fp32", [False, True])
@pytest.mark.parametrize("decoupled", [False, True])
def test_extrapolation_matches_oracle(torch_cuda, fp32, decoupled):
    torch = torch_cuda
    import oracle
    from paper_2210_03523_gb300 import dg
    mi, om, q0 = _case(nx=3, lo=1, hi=6, seed=9, width=0.5)
    m = dg.Mesh(mi)
    sweep = I.full_sweep((6, 6, 6))
    tn, _ = m.tau_estimate(torch.from_numpy(q0).cuda(), sweep, fp32=fp32, want=(True, False))
    targets = np.array([(a, b, c) for c in range(1, 9) for b in range(1, 9) for a in range(1, 9)], np.int32)
    for n_fit, floor in ((0, 0.0), (2, 1e-9)):
        got = m.tau_extrapolate(tn, sweep, targets, n_fit=n_fit, tau_floor=floor, decoupled=decoupled)
        ref = oracle.tau_extrapolate(tn.double().cpu().numpy(), mi.orders, sweep, targets, n_fit=n_fit,
                                     decoupled=decoupled, tau_floor=floor)
        g = got.double().cpu().numpy()
        assert np.array_equal(np.isinf(g), np.isinf(ref)) and np.array_equal(g < 0, ref < 0)
        fin = np.isfinite(ref) & (ref >= 0)
        if fp32:
            np.testing.assert_allclose(g[fin], ref[fin].astype(np.float32), rtol=2 ** -22, atol=0)
        else:
            np.testing.assert_allclose(g[fin], ref[fin], rtol=1e-13, atol=0)
        assert np.isinf(ref).any() and fin.sum() > ref.size // 8
    # F_max accumulation on the device
    acc = m.tau_extrapolate(tn, sweep, targets)
    gen = torch.Generator(device="cuda").manual_seed(5)
    f = torch.rand(tn.shape, generator=gen, device="cuda", dtype=tn.dtype) + 0.5
    tn2 = torch.where(tn >= 0, tn * f, tn)
    m.tau_extrapolate(tn2, sweep, targets, out=acc, accumulate=True)
    want = torch.maximum(m.tau_extrapolate(tn, sweep, targets), m.tau_extrapolate(tn2, sweep, targets))
    assert torch.equal(acc, want)


def test_select_max_decrease_matches_oracle(torch_cuda):
    torch = torch_cuda
    import oracle
    from paper_2210_03523_gb300 import dg
    mi = I.box_mesh(5, orders=I.random_orders(125, 3, 8, 4), phys=I.pulse_physics())
    m = dg.Mesh(mi)
    rng = np.random.default_rng(8)
    sweep = np.array([(a, b, c) for c in range(1, 9) for b in range(1, 9) for a in range(1, 9)], dtype=np.int32)
    mp = rng.uniform(0.0, 1.0, size=(mi.n_elem, len(sweep))) * (sweep.prod(1) ** -1.5)[None, :] * 50
    for rule in (0, 2):
        for dec in (-1, 0, 1, 2):
            ref = oracle.select_orders(mp, sweep, 0.1, 2, 7, rule, mi.neighbors, prev=mi.orders, max_decrease=dec)
            got = m.select_orders(torch.from_numpy(mp).cuda(), sweep, 0.1, 2, 7, rule, max_decrease=dec)
            assert np.array_equal(got, ref), (rule, dec)


def _margin_ok(total, tau_max):
    v = np.asarray(total)
    v = v[np.isfinite(v) & (v >= 0)]
    return np.min(np.abs(v / tau_max - 1.0)) > 1e-9


def test_static_driver_matches_oracle(torch_cuda):
    from oracle import drivers as od
    from paper_2210_03523_gb300 import adapt
    mi, om, q0 = _case(nx=2, lo=3, hi=3, width=0.35)
    targets = np.array([(a, b, c) for c in range(1, 6) for b in range(1, 6) for a in range(1, 6)], np.int32)
    kw = dict(t0=0.0, t_est=0.06, dt_e=0.02, t_final=0.08, cfl=0.5, sweep=I.full_sweep((3, 3, 3)), tau_max=1e-2,
              n_min=1, n_max=5, targets=targets, tau_floor=1e-10)
    ref = od.static_adaptation(mi, q0, **kw)
    got = adapt.static_adaptation(mi, q0, **kw)
    assert _margin_ok(ref["total"], 1e-2)
    assert got["n_estimates"] == ref["n_estimates"] == 2 and got["t"] == ref["t"] == 0.08
    assert got["steps"] == ref["steps"]
    # tau is a difference of O(R) terms: measure the map error against its largest finite entry
    fin = ref["total"][np.isfinite(ref["total"])]
    np.testing.assert_allclose(got["total"].cpu().numpy(), ref["total"], rtol=0, atol=1e-11 * np.abs(fin).max())
    assert np.array_equal(got["orders"], ref["orders"])
    assert got["ndof"] == ref["ndof"] and got["ndof_dyn"] == ref["ndof_dyn"]
    assert _close(got["q"].cpu().numpy(), ref["q"], got["orders"], 1e-11)


@pytest.mark.parametrize("rule", [1, 2])
def test_dynamic_driver_matches_oracle(torch_cuda, rule):
    from oracle import drivers as od
    from paper_2210_03523_gb300 import adapt
    mi, om, q0 = _case(nx=3, lo=4, hi=4, width=0.3)
    targets = np.array([(a, b, c) for c in range(3, 8) for b in range(3, 8) for a in range(3, 8)], np.int32)
    kw = dict(t0=0.0, dt_e=0.02, t_final=0.1, cfl=0.5, sweep=lambda P: I.full_sweep(np.asarray(P).max(0)),
              tau_max=3e-3, n_min=3, n_max=7, jump_rule=rule, max_decrease=1, targets=targets, tau_floor=1e-10)
    ref = od.dynamic_adaptation(mi, q0, **kw)
    got = adapt.dynamic_adaptation(mi, q0, **kw)
    assert len(got["history"]) == len(ref["history"]) == 4 and got["t"] == ref["t"] == 0.1
    for a, b in zip(got["history"], ref["history"]):
        assert np.array_equal(a, b)
    assert got["steps"] == ref["steps"]
    assert got["ndof"] == ref["ndof"] and got["ndof_dyn"] == ref["ndof_dyn"]
    assert _close(got["q"].cpu().numpy(), ref["q"], got["orders"], 1e-11)


@pytest.mark.parametrize("fp32", [False, True])
def test_dual_time_stepping_tau_matches_oracle(torch_cuda, fp32):
    """The dual time-stepping estimate (Sec. 2.3, item 2) through the C ABI:
    r_p = BDF2 time derivative of three states of an RK trajectory."""
    torch = torch_cuda
    import oracle
    from paper_2210_03523_gb300 import dg
    mi, om, q0 = _case(nx=2, lo=2, hi=4, seed=12, width=0.4)
    m = dg.Mesh(mi)
    dt = 2e-3
    qs = [q0.copy()]
    q, G = q0.copy(), np.zeros_like(q0)
    for _ in range(2):
        om.rk_step(q, G, dt)
        qs.append(q.copy())
    bdf2 = (3.0 * qs[2] - 4.0 * qs[1] + qs[0]) / (2.0 * dt)
    sweep = I.full_sweep((4, 4, 4))
    ref, _ = om.tau(qs[2], sweep, rP=bdf2)
    got, _ = m.tau_estimate(torch.from_numpy(qs[2]).cuda(), sweep, fp32=fp32, r_p=torch.from_numpy(bdf2).cuda(),
                            want=(True, False))
    from test_gpu_parity import _fp32_scale, _tau_tol
    g = got.double().cpu().numpy()
    assert np.array_equal(g < 0, ref < 0)
    ok = ref >= 0
    if fp32:      # the FP32 bound of the sweep: 8 (eps32 S_dev + eps64 S_full) per element
        from oracle_helpers import fp32_tau_ratio
        assert fp32_tau_ratio(g, ref, _fp32_scale(om, qs[2], mi)) <= 8
    else:
        assert np.abs(g - ref)[ok].max() <= _tau_tol(ref, mi, qs[2], om)


def test_resume_from_checkpoint_is_bitwise(torch_cuda, tmp_path):
    """A run checkpointed half way (after an order change) and resumed on a
    fresh mesh ends bitwise where the uninterrupted run ends: the low-storage
    RK3 register restarts at zero every step, so the state, the orders and
    the time are the whole solution."""
    torch = torch_cuda
    from paper_2210_03523_gb300 import dg
    mi, om, q0 = _case()
    new_orders = I.random_orders(mi.n_elem, 1, 6, 77)

    def run(m, q, t, n):
        g = torch.zeros_like(q)
        assert m.advance(q, g, t, math.inf, 0.5, max_steps=n, count=True) == n
        return q

    m = dg.Mesh(mi)
    q = torch.from_numpy(q0).cuda()
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    run(m, q, t, 10)
    q = m.set_orders(new_orders, q)
    run(m, q, t, 5)
    m.save_state(tmp_path / "half.dgs", q, t.item())
    run(m, q, t, 12)
    m2 = dg.Mesh(mi)                   # the original orders: load_state switches them
    q2, t2 = m2.load_state(tmp_path / "half.dgs")
    assert np.array_equal(m2.orders(), new_orders)
    run(m2, q2, t2, 12)
    assert torch.equal(q, q2) and t.item() == t2.item()
    assert m.get_error() == 0 and m2.get_error() == 0


def test_static_driver_on_a_curved_navier_stokes_ogrid_matches_oracle(torch_cuda):
    """The static driver on a small curved O-grid around a cylinder
    (Navier-Stokes, walls and far field, uniform P = (4,4,1)): estimation,
    selection among N <= P and the run after adaptation, whose mixed orders put
    p-nonconforming faces on a curved Navier-Stokes mesh.  tau_max sits midway
    between two well separated values of the oracle's accumulated map, so that
    no selection hinges on rounding."""
    from oracle import drivers as od
    from paper_2210_03523_gb300 import adapt
    import oracle
    p0 = 10.0
    ph = I.Physics(1, 1.4, 0.05, 0.72, p0, (1.0, 0.5, 0.1, 0.0, p0 / 0.4 + 0.5 * 0.26))
    mi = I.ogrid_mesh(n_theta=8, n_r=3, ratio=4.0, orders=(4, 4, 1), phys=ph)
    om = oracle.Mesh(mi)

    def fn(x, y, z):
        r2 = x * x + y * y
        damp = 1.0 - np.exp(-(r2 - 0.25) * 4.0)
        rho = 1.0 + 0.05 * np.sin(1.3 * x + 0.2) * np.cos(0.9 * y)
        u, v = damp * (0.5 + 0.05 * np.cos(y)), damp * (0.1 + 0.04 * np.sin(0.7 * x))
        p = p0 * (1.0 + 0.02 * np.cos(x + 0.5 * y + 0.7))
        return np.stack([rho, rho * u, rho * v, 0 * x, p / 0.4 + 0.5 * rho * (u * u + v * v)])
    q0 = I.pointwise_state(om.coords(), mi.orders, fn)
    dt = om.max_dt(q0, 0.5)
    kw = dict(t0=0.0, t_est=3.5 * 4 * dt, dt_e=4 * dt, cfl=0.5, sweep=I.full_sweep((4, 4, 1)), n_min=1, n_max=4,
              jump_rule=2)
    est = od.static_adaptation(mi, q0, t_final=kw["t_est"], tau_max=1.0, **kw)
    v = np.sort(est["total"][np.isfinite(est["total"]) & (est["total"] > 0)].ravel())
    gaps = v[1:] / v[:-1]
    mid = len(v) // 2
    k = mid + int(np.argmax(gaps[mid: mid + len(v) // 4]))       # a wide gap above the median
    tau_max = float(np.sqrt(v[k] * v[k + 1]))
    kw.update(t_final=kw["t_est"] + 40 * dt, tau_max=tau_max)
    ref = od.static_adaptation(mi, q0, **kw)
    got = adapt.static_adaptation(mi, q0, **kw)
    assert _margin_ok(ref["total"], tau_max)
    assert len({tuple(o) for o in ref["orders"]}) > 1               # mixed orders after adaptation
    assert got["n_estimates"] == ref["n_estimates"] == 3 and got["steps"] == ref["steps"]
    assert np.array_equal(got["orders"], ref["orders"])
    assert got["ndof"] == ref["ndof"] and got["ndof_dyn"] == ref["ndof_dyn"]
    assert _close(got["q"].cpu().numpy(), ref["q"], got["orders"], 1e-11)
    assert got["mesh"].get_error() == 0
