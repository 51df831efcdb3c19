"""Pins of the oracle's brute-force discrete adjoint (the reference of the
adjoint kernels): every Jacobian column by fourth-order central differences,
then J^T v.  On the density-pulse family (uniform velocity and pressure) the
Euler residual and one RK3 step are exactly affine in the density (Sec. 3.1
pulse problem; the pin of the residual against scalar upwind advection), so
along a direction w of that family J w = F(q + w) - F(q) exactly, and
<J^T v, w> must equal <v, F(q + w) - F(q)> for any v: a transposed index, a
wrong sign or a dropped column fails it."""
import numpy as np
import pytest

from paper_2210_03523_gb300 import inputs as I

VEL = (0.9, -0.6, 0.3)    # no velocity component is zero: Roe's |u.n| stays away from its kink


def _family(ph, coords, orders, fn):
    qi = np.asarray(ph.qinf)
    u = qi[1:4] / qi[0]
    p0 = (ph.gamma - 1) * (qi[4] - 0.5 * qi[0] * u @ u)

    def state(x, y, z):
        rho = fn(x, y, z)
        return np.stack([rho, rho * u[0], rho * u[1], rho * u[2], p0 / (ph.gamma - 1) + 0.5 * rho * (u @ u)])

    def direction(x, y, z):
        phi = np.sin(np.pi * x + 0.3) * np.cos(np.pi * y) * (1.0 + 0.2 * z)
        return 1e-2 * np.stack([phi, phi * u[0], phi * u[1], phi * u[2], 0.5 * phi * (u @ u)])
    return I.pointwise_state(coords, orders, state), I.pointwise_state(coords, orders, direction)


@pytest.mark.parametrize("periodic", [True, False])
def test_residual_adjoint_along_the_pulse_family(orc, periodic):
    ph = I.pulse_physics(mach=0.4, velocity=VEL)
    kw = {} if periodic else dict(periodic=(False, False, False))
    mi = I.box_mesh(2, orders=I.random_orders(8, 1, 3, 31), phys=ph, **kw)
    m = orc.Mesh(mi)
    q, w = _family(ph, m.coords(), m.orders, lambda x, y, z: 1.0 + 0.3 * np.exp(-((x + 0.2) ** 2 + y ** 2)))
    v = np.random.default_rng(5).standard_normal(q.size)
    lhs = m.residual_vjp_fd(q, v) @ w
    rhs = v @ (m.residual(q + w) - m.residual(q))
    assert abs(lhs - rhs) <= 1e-9 * np.abs(v).sum() * np.abs(m.residual(q + w) - m.residual(q)).max()


def test_rk_step_adjoint_along_the_pulse_family(orc):
    ph = I.pulse_physics(mach=0.4, velocity=VEL)
    mi = I.box_mesh(2, orders=I.random_orders(8, 1, 3, 32), phys=ph)
    m = orc.Mesh(mi)
    q, w = _family(ph, m.coords(), m.orders, lambda x, y, z: 1.0 + 0.3 * np.cos(np.pi * x) * np.sin(np.pi * z))
    dt = 0.5 * m.max_dt(q, 1.0)
    lam = np.random.default_rng(6).standard_normal(q.size)

    def step(x):
        x = x.copy()
        m.rk_step(x, np.zeros_like(x), dt)
        return x
    lhs = m.rk_step_vjp_fd(q, dt, lam) @ w
    d = step(q + w) - step(q)
    rhs = lam @ d
    assert abs(lhs - rhs) <= 1e-9 * np.abs(lam).sum() * np.abs(d).max()


def test_residual_adjoint_is_not_the_jacobian(orc):
    """The Jacobian of the residual is not symmetric: J^T v differs from J v
    (taken by one central difference), so the pin above tells them apart."""
    ph = I.pulse_physics(mach=0.4, velocity=VEL)
    mi = I.box_mesh(2, orders=(2, 2, 2), phys=ph)
    m = orc.Mesh(mi)
    q = I.pulse_state(m.coords(), m.orders, ph, width=0.5)
    v = np.random.default_rng(7).standard_normal(q.size) * 1e-3
    jt = m.residual_vjp_fd(q, v)
    jv = (m.residual(q + v) - m.residual(q - v)) / 2.0
    assert np.abs(jt - jv).max() > 1e-3 * np.abs(jt).max()
