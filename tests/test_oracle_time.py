"""Pins of the oracle's Williamson low-storage RK3 (Sec. 3), its CFL time
step, and design-order convergence of the advected density pulse
(Sec. 3.1) against the closed-form translation rho(x - u t)."""
import math

import numpy as np
import pytest

from paper_2210_03523_gb300 import inputs as I
from oracle_helpers import tensor_weights


def test_williamson_rk3_order_conditions(orc):
    """Turn the 2N-storage (A, B) pairs into a Butcher tableau and check the
    four third-order conditions exactly."""
    A, B = orc.rk_coeffs()
    s = 3
    # G_k = A_k G_{k-1} + dt R_{k-1};  Q_k = Q_{k-1} + B_k G_k; track coefficients of dt R_j
    Gc = np.zeros(s)
    Qc = np.zeros(s)
    a = np.zeros((s, s))     # a[k] = coefficients of stage k's input state
    for k in range(s):
        a[k] = Qc
        Gc = A[k] * Gc
        Gc[k] += 1.0
        Qc = Qc + B[k] * Gc
    b = Qc
    c = a.sum(1)
    assert abs(b.sum() - 1) < 1e-15
    assert abs(b @ c - 0.5) < 1e-15
    assert abs(b @ c ** 2 - 1 / 3) < 1e-15
    assert abs(b @ (a @ c) - 1 / 6) < 1e-15
    np.testing.assert_allclose(c, [0.0, 1 / 3, 3 / 4], atol=1e-15)


def test_rk3_step_is_third_order_taylor_on_linear_operator(orc):
    """On the density-pulse family the residual is linear in rho:
    R_rho(c + phi) = L phi.  One RK3 step must equal
    (I + dt L + dt^2 L^2/2 + dt^3 L^3/6) applied to rho."""
    ph = I.pulse_physics(mach=0.5, velocity=(0.6, 0.3, -0.2))
    mi = I.box_mesh(2, orders=I.random_orders(8, 1, 4, 3), phys=ph)
    m = orc.Mesh(mi)
    xyz = m.coords()
    q0 = I.pulse_state(xyz, m.orders, ph, width=0.4)
    u = np.asarray(ph.qinf[1:4])
    p0 = (ph.gamma - 1) * (ph.qinf[4] - 0.5 * u @ u)
    off = m.off

    def state_of(rho):
        q = np.empty(5 * off[-1])
        for e in range(m.n_elem):
            blk = q[5 * off[e]:5 * off[e + 1]].reshape(5, -1)
            r = rho[off[e]:off[e + 1]]
            blk[0] = r
            blk[1:4] = r[None] * u[:, None]
            blk[4] = p0 / (ph.gamma - 1) + 0.5 * r * (u @ u)
        return q

    def rho_of(q):
        return np.concatenate([m.elem(q, e)[0] for e in range(m.n_elem)])

    def L(phi):
        c = 10.0 * (1.0 + np.abs(phi).max())
        return rho_of(m.residual(state_of(c + phi)))

    rho = rho_of(q0)
    dt = 0.02
    L1 = L(rho)
    L2 = L(L1)
    L3 = L(L2)
    expect = rho + dt * L1 + dt ** 2 / 2 * L2 + dt ** 3 / 6 * L3
    q = q0.copy()
    G = np.zeros_like(q)
    m.rk_step(q, G, dt)
    np.testing.assert_allclose(rho_of(q), expect, atol=1e-13)


def test_max_dt_closed_form(orc):
    """uniform state on an axis-aligned box of size h: J = h^3/8, J a^i = h^2/4 e_i"""
    ph = I.pulse_physics(mach=0.3, velocity=(1.0, 0.5, 0.0))
    mi = I.box_mesh(4, orders=(3, 2, 5), phys=ph)
    m = orc.Mesh(mi)
    q = I.uniform_state(m.orders, ph.qinf)
    h = 0.5
    u = np.array([1.0, 0.5, 0.0])
    p = (ph.gamma - 1) * (ph.qinf[4] - 0.5 * u @ u)
    c = math.sqrt(ph.gamma * p)
    J, a = h ** 3 / 8, h ** 2 / 4
    s = sum((N + 1) ** 2 * (a * abs(u[i]) + c * a) / (2 * J) for i, N in enumerate((3, 2, 5)))
    assert abs(m.max_dt(q, 0.5) - 0.5 / s) < 1e-14 * (0.5 / s)


def _ns_rest(mu, Pr, p0=3.0, rho=1.7):
    return I.Physics(1, 1.4, mu, Pr, 1.0, (rho, 0.0, 0.0, 0.0, p0 / 0.4))


def _dt(orc, mi, cfl=0.5):
    m = orc.Mesh(mi)
    return m.max_dt(I.uniform_state(m.orders, mi.phys.qinf), cfl)


def test_max_dt_viscous_term(orc):
    """The viscous term of the CFL step (Navier-Stokes), pinned without its
    formula: a fluid at rest (no advective speed but sound) with a large mu
    is in the viscous regime, where the step must scale as h^2 (mesh scaled
    by 2: dt x 4) and as 1/mu, take max(1, gamma/Pr) (Pr = 2.8 against 0.35:
    ratio 4), and be invariant under a rotation of a sheared mesh (a
    transposed metric index is not); at small mu the sound speed decides
    (dt x 2 under the same scaling) and mu drops out."""
    orders = (3, 2, 4)
    A = np.array([[1.0, 0.3, 0.0], [0.0, 1.0, 0.2], [0.1, 0.0, 1.0]])
    th = 0.7
    R = np.array([[math.cos(th), -math.sin(th), 0.0], [math.sin(th), math.cos(th), 0.0], [0.0, 0.0, 1.0]])
    R = R @ np.array([[1.0, 0.0, 0.0], [0.0, math.cos(0.4), -math.sin(0.4)], [0.0, math.sin(0.4), math.cos(0.4)]])

    def mesh(mu, Pr=2.8, M=A):
        return I.box_mesh(2, orders=orders, phys=_ns_rest(mu, Pr), mapping=I.affine_map(M))
    big, small = 50.0, 1e-6
    dv = _dt(orc, mesh(big))
    assert _dt(orc, mesh(big, M=2 * A)) == pytest.approx(4 * dv, rel=1e-13)
    assert _dt(orc, mesh(2 * big)) == pytest.approx(dv / 2, rel=1e-13)
    assert _dt(orc, mesh(big, Pr=0.35)) == pytest.approx(dv / 4, rel=1e-13)
    assert _dt(orc, mesh(big, M=R @ A)) == pytest.approx(dv, rel=1e-12)
    da = _dt(orc, mesh(small))
    assert da < dv / 1e-3   # the sound speed now decides ...
    assert _dt(orc, mesh(small, M=2 * A)) == pytest.approx(2 * da, rel=1e-13)
    assert _dt(orc, mesh(2 * small)) == pytest.approx(da, rel=1e-13)
    assert _dt(orc, mesh(small, M=R @ A)) == pytest.approx(da, rel=1e-12)
    # ... and the axis-aligned closed form of the viscous term, h = 1 per element:
    # |J a^i|^2 / (4 J^2) = 1 / h^2, nu = mu / rho
    dbox = _dt(orc, I.box_mesh(2, orders=orders, phys=_ns_rest(big, 2.8)))
    s_v = sum((N + 1) ** 4 for N in orders) * big / 1.7
    assert dbox == pytest.approx(0.5 / s_v, rel=1e-14)


def test_pulse_centroid_moves_with_the_flow(orc):
    """No dispersion of the pulse's position (Sec. 3.1, the advected pulse):
    the discrete first moment M1 = sum w J x (rho - 1) of the density
    perturbation obeys dM1/dt = u M0 exactly, because every face flux is
    single-valued, x is continuous and linear (the mortars' L2 projection
    keeps it) and the GL derivative is summation-by-parts.  So the residual's
    first moment is u M0, and one RK3 step (linear in the moments) moves the
    centroid by u dt, to roundoff, on mixed orders with mortars.  The identity
    needs the perturbation to stay off the periodic seam, where x jumps: the
    pulse family's Roe flux is pure upwinding (the acoustic waves vanish up to
    roundoff), so the support grows by one element per stage downstream, and
    the pulse starts four elements upstream of the seam."""
    u = np.array([1.0, 0.5, -0.25])
    ph = I.pulse_physics(mach=0.3, velocity=tuple(u))
    mi = I.box_mesh(8, orders=I.random_orders(512, 2, 5, 31), phys=ph)
    m = orc.Mesh(mi)
    xyz = m.coords()
    q = I.pulse_state(xyz, m.orders, ph, amp=4.0, width=0.05, center=(-0.6, -0.6, 0.6), images=0)

    def last_layer_clean(q):   # the elements at the downstream seams hold rho = 1 to roundoff
        dev = 0.0
        for e in range(m.n_elem):
            x = m.elem(xyz, e, 3)
            if x[0].min() > 0.7 or x[1].min() > 0.7 or x[2].max() < -0.7:
                dev = max(dev, np.abs(m.elem(q, e)[0] - 1.0).max())
        return dev <= 1e-14

    def moments(a, q0=True):   # M0, M1 and the size of their terms (the roundoff scale)
        M0, M1, S = 0.0, np.zeros(3), 0.0
        for e in range(m.n_elem):
            _, _, J = m.metrics(e)
            wr = tensor_weights(m.orders[e]) * J * (m.elem(a, e)[0] - (1.0 if q0 else 0.0))
            M0 += wr.sum()
            M1 += m.elem(xyz, e, 3) @ wr
            S += np.abs(wr).sum()
        return M0, M1, S
    assert last_layer_clean(q)
    M0, M1, _ = moments(q)
    dM0, dM1, S = moments(m.residual(q), q0=False)
    assert abs(dM0) <= 1e-13 * S
    assert np.abs(dM1 - u * M0).max() <= 1e-13 * S, (dM1 / M0, u)
    assert np.abs(u * M0).max() > 1e-3 * S        # ... which is not small against the terms
    dt = m.max_dt(q, 0.5)
    G = np.zeros_like(q)
    m.rk_step(q, G, dt)
    assert last_layer_clean(q)
    M0t, M1t, _ = moments(q)
    assert abs(M0t - M0) <= 1e-15 * 8.0             # roundoff of the nodal values over the box's volume
    shift = M1t / M0t - M1 / M0
    assert np.abs(shift - u * dt).max() <= 1e-10 * np.abs(u * dt).max(), (shift, u * dt)


def _l2_error(m, q, ph, t, width, center):
    xyz = m.coords()
    u = np.asarray(ph.qinf[1:4])
    err = 0.0
    for e in range(m.n_elem):
        x = m.elem(xyz, e, 3)
        exact = I.pulse_primitive(x[0] - u[0] * t, x[1] - u[1] * t, x[2] - u[2] * t, width=width, center=center,
                                  images=1)
        _, _, J = m.metrics(e)
        err += ((m.elem(q, e)[0] - exact) ** 2 * tensor_weights(m.orders[e]) * J).sum()
    return math.sqrt(err)


@pytest.mark.parametrize("N", [2, 3])
def test_design_order_convergence(orc, N):
    """L2 error of the advected pulse against rho(x - u t) (periodic-image
    sum) decays like h^(N+1) on 2^3, 4^3, 8^3 meshes (observed 2.7 for N=2,
    4.0 for N=3 at t=0.2; shorter times are dominated by the O(h^N)
    pointwise residual truncation error)."""
    ph = I.pulse_physics(mach=0.5, velocity=(1.0, 1.0, 0.0))
    width, center, T = 0.6, (0.1, -0.05, 0.0), 0.2
    errs = []
    for nx in (2, 4, 8):
        mi = I.box_mesh(nx, orders=(N, N, N), phys=ph)
        m = orc.Mesh(mi)
        q = I.pulse_state(m.coords(), m.orders, ph, width=width, center=center, images=1)
        G = np.zeros_like(q)
        dt0 = m.max_dt(q, 0.4)
        nsteps = int(math.ceil(T / dt0))
        dt = T / nsteps
        for _ in range(nsteps):
            m.rk_step(q, G, dt)
        errs.append(_l2_error(m, q, ph, T, width, center))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert rates[-1] > N + 1 - 0.6, (errs, rates)


def test_rk3_temporal_convergence_order(orc):
    """At a fixed spatial discretisation (N = 6), the time-integration error of
    Williamson's RK3 falls by 2^3 per halving of dt (Sec. 3: a third-order
    scheme); the reference is the same run at dt/16."""
    ph = I.pulse_physics(mach=0.5, velocity=(0.6, 0.3, -0.2))
    mi = I.box_mesh(2, orders=(6, 6, 6), phys=ph)
    m = orc.Mesh(mi)
    q0 = I.pulse_state(m.coords(), m.orders, ph, width=0.45, images=2)
    T = 0.08
    dt0 = m.max_dt(q0, 1.0)

    def run(n):
        q, G = q0.copy(), np.zeros_like(q0)
        for _ in range(n):
            m.rk_step(q, G, T / n)
        return q
    n0 = int(math.ceil(T / dt0))
    ref = run(16 * n0)
    err = [np.abs(run(k * n0) - ref).max() for k in (1, 2, 4)]
    rates = [err[i] / err[i + 1] for i in range(2)]
    assert all(6.5 < r < 9.5 for r in rates), (err, rates)
