"""Pins of the oracle's time integration to a given time and of its
dynamic (Fig. 1) and static (Fig. 2) p-adaptation drivers (Sec. 3.2), with
the bounds of Sec. 3.3 (N_min, N_max, an order falls by at most one per
adaptation stage) and the jump conditions of Sec. 3.1."""
import numpy as np
import pytest

from paper_2210_03523_gb300 import inputs as I


def test_advance_lands_on_t_end_with_constant_dt(orc):
    """Uniform flow: the CFL step is constant, so reaching T takes
    ceil(T/dt) steps, the last one shortened, and the state stays uniform
    (free stream)."""
    ph = I.pulse_physics(mach=0.4)
    mi = I.box_mesh(2, orders=(3, 2, 4), phys=ph)
    m = orc.Mesh(mi)
    q = I.uniform_state(mi.orders, ph.qinf)
    dt = m.max_dt(q, 0.5)
    T = 7.3 * dt
    G = np.zeros_like(q)
    t, n = m.advance(q, G, 0.5, 0.0, T)
    assert t == T and n == 8
    np.testing.assert_allclose(q, I.uniform_state(mi.orders, ph.qinf), rtol=1e-13, atol=1e-13 * abs(ph.qinf[4]))
    t2, n2 = m.advance(q, G, 0.5, t, T)
    assert (t2, n2) == (T, 0)


def test_advance_equals_explicit_steps(orc):
    ph = I.pulse_physics(mach=0.3)
    mi = I.box_mesh(2, orders=I.random_orders(8, 2, 4, 7), phys=ph)
    m = orc.Mesh(mi)
    q0 = I.pulse_state(m.coords(), mi.orders, ph, width=0.4)
    q, G = q0.copy(), np.zeros_like(q0)
    t, n = m.advance(q, G, 0.6, 0.1, 0.13)
    # the same by hand: CFL steps, the last one cut at t_end
    q2, G2, tt, k = q0.copy(), np.zeros_like(q0), 0.1, 0
    while tt < 0.13:
        dt = m.max_dt(q2, 0.6)
        dt = min(dt, 0.13 - tt)
        m.rk_step(q2, G2, dt)
        tt = 0.13 if tt + dt >= 0.13 else tt + dt
        k += 1
    assert t == 0.13 and n == k
    np.testing.assert_array_equal(q, q2)


def _pulse_case(nx=2, P=3, width=0.35):
    ph = I.pulse_physics(mach=0.5)
    mi = I.box_mesh(nx, orders=(P, P, P), phys=ph)
    q0 = I.pulse_state(_coords(mi), mi.orders, ph, width=width, center=(-0.3, -0.3, 0.0))
    return mi, q0


def _coords(mi):
    import oracle
    return oracle.Mesh(mi).coords()


def test_static_driver_is_fmax_of_the_stage_maps(orc):
    from oracle import drivers
    mi, q0 = _pulse_case()
    sweep = I.full_sweep((3, 3, 3))
    targets = np.array([(a, b, c) for c in range(1, 6) for b in range(1, 6) for a in range(1, 6)], np.int32)
    kw = dict(cfl=0.5, sweep=sweep, tau_max=1e-2, n_min=1, n_max=5, targets=targets, tau_floor=1e-10)
    res = drivers.static_adaptation(mi, q0, t0=0.0, t_est=0.06, dt_e=0.02, t_final=0.08, **kw)
    assert res["n_estimates"] == 2 and res["t"] == 0.08
    # by hand: the maps at t = 0.02 and 0.04, extrapolated, F_max, selection
    m = orc.Mesh(mi)
    q, G = q0.copy(), np.zeros_like(q0)
    total = None
    t = 0.0
    for te in (0.02, 0.04):
        t, _ = m.advance(q, G, 0.5, t, te)
        mp = orc.tau_extrapolate(m.tau(q, sweep)[0], mi.orders, sweep, targets, tau_floor=1e-10)
        total = mp if total is None else np.maximum(total, mp)
    np.testing.assert_array_equal(res["total"], total)
    np.testing.assert_array_equal(res["orders"], orc.select_orders(total, targets, 1e-2, 1, 5, 0, mi.neighbors))
    assert not np.array_equal(res["orders"], mi.orders)


def test_static_driver_without_estimate_keeps_orders(orc):
    from oracle import drivers
    mi, q0 = _pulse_case()
    res = drivers.static_adaptation(mi, q0, t0=0.0, t_est=0.01, dt_e=0.05, t_final=0.02, cfl=0.5,
                                    sweep=I.full_sweep((3, 3, 3)), tau_max=1e-2, n_min=1, n_max=5)
    assert res["n_estimates"] == 0 and res["total"] is None
    np.testing.assert_array_equal(res["orders"], mi.orders)
    m = orc.Mesh(mi)
    q, G = q0.copy(), np.zeros_like(q0)
    t, _ = m.advance(q, G, 0.5, 0.0, 0.01)
    m.advance(q, G, 0.5, t, 0.02)
    np.testing.assert_array_equal(res["q"], q)


@pytest.mark.parametrize("rule", [1, 2])
def test_dynamic_driver_bounds_and_jumps(orc, rule):
    from oracle import drivers
    mi, q0 = _pulse_case(nx=3, P=4, width=0.3)
    targets = np.array([(a, b, c) for c in range(3, 8) for b in range(3, 8) for a in range(3, 8)], np.int32)
    res = drivers.dynamic_adaptation(mi, q0, t0=0.0, dt_e=0.02, t_final=0.1, cfl=0.5,
                                     sweep=lambda P: I.full_sweep(P.max(0)), tau_max=3e-3, n_min=3, n_max=7,
                                     jump_rule=rule, max_decrease=1, targets=targets, tau_floor=1e-10)
    hist = [np.asarray(mi.orders)] + res["history"]
    assert len(res["history"]) == 4 and res["t"] == 0.1
    nb = mi.neighbors
    for prev, cur in zip(hist[:-1], hist[1:]):
        assert cur.min() >= 3 and cur.max() <= 7
        assert np.all(cur >= prev - 1)
        for e in range(mi.n_elem):
            for j in nb[e][nb[e] >= 0]:
                lim = (2 * cur[j]) // 3 if rule == 1 else cur[j] - 1
                assert np.all(cur[e] >= lim)
    assert any(not np.array_equal(h, hist[0]) for h in hist[1:])


@pytest.mark.slow
def test_static_adaptation_follows_the_pulse(orc):
    """The elements the pulse crosses during the estimation time end with
    more degrees of freedom than the elements it never reaches (Sec. 3.3:
    the adapted orders concentrate where the flow feature travels)."""
    from oracle import drivers
    ph = I.pulse_physics(mach=0.5)
    mi = I.box_mesh(4, orders=(3, 3, 3), phys=ph)
    xyz = orc.Mesh(mi).coords()
    q0 = I.pulse_state(xyz, mi.orders, ph, width=0.2, center=(-0.5, -0.5, 0.0))
    targets = np.array([(a, b, c) for c in range(1, 7) for b in range(1, 7) for a in range(1, 7)], np.int32)
    # u = (1, 1, 0): by t = 0.5 the pulse centre moves from (-0.5, -0.5, 0) to the origin
    res = drivers.static_adaptation(mi, q0, t0=0.0, t_est=0.5, dt_e=0.125, t_final=0.5, cfl=0.5,
                                    sweep=I.full_sweep((3, 3, 3)), tau_max=1e-3, n_min=1, n_max=6,
                                    targets=targets, tau_floor=1e-10)
    nd = np.prod(res["orders"] + 1, axis=1)
    cen = np.array([[xyz[3 * 64 * e + d * 64: 3 * 64 * e + (d + 1) * 64].mean() for d in range(3)]
                    for e in range(mi.n_elem)])
    near = np.abs(cen[:, 2]) < 0.5
    assert nd[near].mean() > 1.5 * nd[~near].mean(), (nd[near].mean(), nd[~near].mean())


def test_ndof_counts_the_nodes(orc):
    """NDOF = sum over elements of (N1+1)(N2+1)(N3+1): the number of nodes the
    oracle mesh places (three coordinates each), for mixed anisotropic orders."""
    from oracle import drivers
    mi = I.box_mesh(3, orders=I.random_orders(27, 1, 7, 19), phys=I.pulse_physics())
    assert drivers.ndof(mi.orders) * 3 == orc.Mesh(mi).coords().size
    assert drivers.ndof([(3, 3, 1)]) == 32 and drivers.ndof([(1, 3, 1), (3, 1, 1)]) == 32


def test_ndof_dyn_weights_each_step(orc):
    """NDOF_dyn is the mean NDOF over the time steps (Sec. 3.3).  With a huge
    tau_max every element drops to N_min at the first adaptation and stays
    there (max_decrease off), so NDOF_dyn = (n1 NDOF_0 + (S - n1) NDOF_min) / S
    with n1 the steps of the first stage, counted by a separate advance."""
    from oracle import drivers
    mi, q0 = _pulse_case(nx=2, P=4, width=0.3)
    res = drivers.dynamic_adaptation(mi, q0, t0=0.0, dt_e=0.02, t_final=0.07, cfl=0.5,
                                     sweep=I.full_sweep((4, 4, 4)), tau_max=1e30, n_min=2, n_max=4)
    assert len(res["history"]) == 3
    assert all(np.array_equal(h, np.full((8, 3), 2)) for h in res["history"])
    m = orc.Mesh(mi)
    q, G = q0.copy(), np.zeros_like(q0)
    _, n1 = m.advance(q, G, 0.5, 0.0, 0.02)
    S = res["steps"]
    nd0, ndmin = 8 * 125, 8 * 27
    assert 0 < n1 < S and res["ndof"] == ndmin
    assert res["ndof_dyn"] == pytest.approx((n1 * nd0 + (S - n1) * ndmin) / S, rel=1e-15)
    # without an adaptation stage the mean is the constant NDOF
    res0 = drivers.dynamic_adaptation(mi, q0, t0=0.0, dt_e=0.05, t_final=0.02, cfl=0.5,
                                      sweep=I.full_sweep((4, 4, 4)), tau_max=1e30, n_min=2, n_max=4)
    assert res0["history"] == [] and res0["ndof_dyn"] == nd0 == res0["ndof"]
    # static: the estimation phase at the initial orders, the rest at the adapted ones
    st = drivers.static_adaptation(mi, q0, t0=0.0, t_est=0.03, dt_e=0.02, t_final=0.05, cfl=0.5,
                                   sweep=I.full_sweep((4, 4, 4)), tau_max=1e30, n_min=2, n_max=4)
    a, b = st["steps"]
    assert st["ndof"] == ndmin and st["ndof_dyn"] == pytest.approx((a * nd0 + b * ndmin) / (a + b), rel=1e-15)
