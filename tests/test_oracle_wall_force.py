"""Pins of the oracle's wall force (drag and lift of the cylinder case,
Sec. 3.3): zero on a closed body in a fluid at rest at constant pressure,
the divergence theorem for a linear pressure field, and the shear drag of a
linear velocity profile over a no-slip plate."""
import math

import numpy as np
import pytest

from paper_2210_03523_gb300 import inputs as I


def _rest(ph, p_fn, u_fn=None):
    def fn(x, y, z):
        rho = np.ones_like(x)
        u = u_fn(x, y, z) if u_fn else (0 * x, 0 * x, 0 * x)
        p = p_fn(x, y, z)
        return np.stack([rho, rho * u[0], rho * u[1], rho * u[2],
                         p / (ph.gamma - 1) + 0.5 * rho * (u[0] ** 2 + u[1] ** 2 + u[2] ** 2)])
    return fn


@pytest.mark.parametrize("eqs", [0, 1])
def test_closed_body_at_rest_has_no_force(orc, eqs):
    ph = I.Physics(eqs, 1.4, 0.01 * eqs, 0.72, 10.0, (1.0, 0.0, 0.0, 0.0, 25.0))
    mi = I.ogrid_mesh(n_theta=12, n_r=2, ratio=4.0, orders=(3, 3, 1), phys=ph)
    m = orc.Mesh(mi)
    q = I.pointwise_state(m.coords(), mi.orders, _rest(ph, lambda x, y, z: 10.0 + 0 * x))
    F = m.wall_force(q)
    assert np.abs(F).max() <= 1e-12 * 10.0 * math.pi


def test_linear_pressure_gives_the_divergence_theorem(orc):
    """p = p0 + a x at rest: F = sum p n_fluid dS = -a V_body e_x (n_fluid
    points into the body).  V_body: the cylinder of radius 0.5, length 1, as
    the degree-3 geometry approximates it (within 1e-5 at 16 elements)."""
    a = 0.7
    ph = I.Physics(0, 1.4, 0.0, 0.72, 10.0, (1.0, 0.0, 0.0, 0.0, 25.0))
    mi = I.ogrid_mesh(n_theta=16, n_r=2, ratio=4.0, orders=(4, 4, 1), phys=ph)
    m = orc.Mesh(mi)
    q = I.pointwise_state(m.coords(), mi.orders, _rest(ph, lambda x, y, z: 10.0 + a * x))
    F = m.wall_force(q)
    assert F[0] == pytest.approx(-a * math.pi * 0.25, rel=1e-5)
    assert abs(F[1]) <= 1e-10 and abs(F[2]) <= 1e-10


def test_shear_drag_on_a_plate(orc):
    """u = alpha (y + 1) e_x over a no-slip wall at y = -1 (box periodic in x
    and z, far field at y = 1 with the state there): the wall sees the shear
    stress mu alpha and the pressure p0, so F = (mu alpha A, -p0 A, 0) with
    A = 4 (BR1 is exact for the linear profile: q-hat equals the trace on
    both boundaries)."""
    mu, alpha, p0 = 0.03, 0.2, 5.0
    E_top = p0 / 0.4 + 0.5 * (2 * alpha) ** 2
    ph = I.Physics(1, 1.4, mu, 0.72, 5.0, (1.0, 2 * alpha, 0.0, 0.0, E_top))
    mi = I.box_mesh(2, orders=(2, 2, 2), phys=ph, periodic=(True, False, True),
                    tags=(I.FAR_FIELD, I.FAR_FIELD, I.WALL, I.FAR_FIELD, I.FAR_FIELD, I.FAR_FIELD))
    m = orc.Mesh(mi)
    q = I.pointwise_state(m.coords(), mi.orders,
                          _rest(ph, lambda x, y, z: p0 + 0 * x, lambda x, y, z: (alpha * (y + 1), 0 * x, 0 * x)))
    F = m.wall_force(q)
    np.testing.assert_allclose(F, [mu * alpha * 4.0, -p0 * 4.0, 0.0], rtol=1e-12, atol=1e-12)
