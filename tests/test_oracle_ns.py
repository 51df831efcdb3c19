"""Pins of the oracle's Navier-Stokes residual with BR1 (Sec. 2.1, Eq.
(SystemAdvDiff), (DGSEMsystem:2); Sec. 3): exact BR1 gradient of linear
states, exact viscous residual of a shear flow, free-stream preservation
with walls and far field, and the pulse-free cylinder case."""
import numpy as np
import pytest

from paper_2210_03523_gb300 import inputs as I


def _ns_phys(mu=0.05):
    return I.Physics(1, 1.4, mu, 0.72, 2.0, (1.0, 0.4, -0.2, 0.1, 8.0))


def _interior(nx):
    return [ix + nx * (iy + nx * iz) for iz in range(1, nx - 1) for iy in range(1, nx - 1)
            for ix in range(1, nx - 1)]


def test_br1_gradient_exact_for_linear_state(orc):
    A = [[1.0, 0.2, 0.0], [0.1, 1.0, 0.15], [0.0, -0.1, 0.9]]
    nx = 4
    mi = I.box_mesh(nx, mapping=I.affine_map(A), orders=I.random_orders(nx ** 3, 1, 4, 31), phys=_ns_phys())
    m = orc.Mesh(mi)
    xyz = m.coords()
    C = np.array([[1.0, 0.1, -0.2, 0.05], [0.3, 0.2, 0.1, -0.1], [-0.1, 0.05, 0.3, 0.2], [0.2, -0.1, 0.0, 0.1],
                  [8.0, 0.5, -0.3, 0.2]])      # q_v = C[v,0] + C[v,1:] . x
    q = I.pointwise_state(xyz, m.orders, lambda x, y, z: C[:, :1] + C[:, 1:] @ np.stack([x, y, z]))
    g = m.gradient(q)
    for e in _interior(nx):
        n = m.off[e + 1] - m.off[e]
        ge = g[15 * m.off[e]:15 * m.off[e + 1]].reshape(3, 5, n)
        for c in range(3):
            np.testing.assert_allclose(ge[c], np.repeat(C[:, 1 + c][:, None], n, 1), atol=1e-12)
    # isolated gradient is exact on every element (no faces involved)
    gi = m.gradient(q, isolated=True)
    for e in range(m.n_elem):
        n = m.off[e + 1] - m.off[e]
        ge = gi[15 * m.off[e]:15 * m.off[e + 1]].reshape(3, 5, n)
        for c in range(3):
            np.testing.assert_allclose(ge[c], np.repeat(C[:, 1 + c][:, None], n, 1), atol=1e-12)


@pytest.mark.parametrize("mixed", [False, True])
def test_shear_flow_viscous_residual(orc, mixed):
    """u = (a y, 0, 0), rho and p constant: the advective residual vanishes and
    the viscous one is R_rhoE = mu a^2 (viscous heating), R_mom = 0.  Mixed:
    orders 3..4 per element and direction, so that the BR1 and Roe fluxes
    cross mortars; the energy flux (E + p) u is cubic in y, which every
    order >= 3 holds exactly, so the mortar's projection changes nothing."""
    nx, a, mu = 4, 0.8, 0.07
    ph = _ns_phys(mu)
    mi = I.box_mesh(nx, orders=I.random_orders(nx ** 3, 3, 4, 33) if mixed else (2, 3, 2), phys=ph)
    if mixed:   # p-nonconforming faces among the interior elements' faces
        o = np.asarray(mi.orders).reshape(-1, 3)
        assert len({tuple(o[e]) for e in _interior(nx)}) > 1
    m = orc.Mesh(mi)
    rho, p = 1.3, 5.0
    q = I.pointwise_state(m.coords(), m.orders, lambda x, y, z: np.stack(
        [rho + 0 * x, rho * a * y, 0 * x, 0 * x, p / 0.4 + 0.5 * rho * (a * y) ** 2]))
    r = m.residual(q)
    for e in _interior(nx):
        R = m.elem(r, e)
        np.testing.assert_allclose(R[:4], 0.0, atol=1e-11)
        np.testing.assert_allclose(R[4], mu * a * a, atol=1e-11)


def test_isolated_shear_flow_every_element(orc):
    """The isolated residual (element-local BR1 gradient, inner fluxes on the
    faces; Sec. 2.2) sees each element's polynomial alone, so the shear flow
    u = (a y, 0, 0) gives R_rhoE = mu a^2 and R_mom = 0 on every element,
    the ones on the periodic seam included, and on a sheared mesh too."""
    nx, a, mu = 3, 0.8, 0.07
    A = [[1.0, 0.2, 0.0], [0.1, 1.0, 0.15], [0.0, -0.1, 0.9]]
    mi = I.box_mesh(nx, mapping=I.affine_map(A), orders=I.random_orders(nx ** 3, 3, 4, 34), phys=_ns_phys(mu))
    m = orc.Mesh(mi)
    rho, p = 1.3, 5.0
    q = I.pointwise_state(m.coords(), m.orders, lambda x, y, z: np.stack(
        [rho + 0 * x, rho * a * y, 0 * x, 0 * x, p / 0.4 + 0.5 * rho * (a * y) ** 2]))
    r = m.residual(q, isolated=True)
    for e in range(m.n_elem):
        R = m.elem(r, e)
        np.testing.assert_allclose(R[:4], 0.0, atol=1e-11)
        np.testing.assert_allclose(R[4], mu * a * a, atol=1e-11)
    assert np.abs(m.residual(q)).max() > 1.0      # the full residual does see the seam's jump


@pytest.mark.parametrize("case", ["wavy_moving", "ogrid_rest"])
def test_ns_free_stream(orc, case):
    if case == "wavy_moving":
        mi = I.box_mesh(3, geom_order=3, mapping=I.wavy_map(0.08), orders=I.random_orders(27, 1, 4, 32),
                        phys=_ns_phys())
        qc = mi.phys.qinf
    else:
        ph = I.Physics(1, 1.4, 0.01, 0.72, 17.857142857142858, (1.0, 0.0, 0.0, 0.0, 44.642857142857146))
        mi = I.ogrid_mesh(n_theta=12, n_r=4, orders=(4, 4, 1), phys=ph)
        qc = ph.qinf
    m = orc.Mesh(mi)
    q = I.uniform_state(m.orders, qc)
    assert np.abs(m.residual(q)).max() < 1e-10 * qc[4]
    assert np.abs(m.residual(q, isolated=True)).max() < 1e-10 * qc[4]


def test_cylinder_wall_has_no_mass_flux(orc):
    """A swirl with tangential velocity, uniform density and pressure, and a
    far-field state of the same density and pressure: no mass crosses the
    far field (no normal velocity, no jump in rho or p) nor the wall (the
    reflected ghost makes Roe's mass flux vanish), so the J w-weighted mass
    residual sums to zero while the flow along the wall is non-trivial."""
    p0 = 17.857142857142858
    ph = I.Physics(1, 1.4, 0.01, 0.72, p0, (1.0, 0.0, 0.0, 0.0, p0 / 0.4))
    mi = I.ogrid_mesh(n_theta=16, n_r=6, ratio=4.0, orders=(3, 3, 1), phys=ph)
    m = orc.Mesh(mi)
    # swirl at rest far away: u = omega(r) (-y, x) with omega -> 0 beyond r = 1.5
    def fn(x, y, z):
        r2 = x * x + y * y
        om = 0.3 * np.exp(-(r2 - 0.25) * 3.0)
        u, v = -om * y, om * x
        rho = 1.0 + 0 * x
        p = p0
        return np.stack([rho, rho * u, rho * v, 0 * x, p / 0.4 + 0.5 * rho * (u * u + v * v)])
    q = I.pointwise_state(m.coords(), m.orders, fn)
    r = m.residual(q)
    from oracle_helpers import tensor_weights
    tot = 0.0
    for e in range(m.n_elem):
        _, _, J = m.metrics(e)
        tot += (m.elem(r, e)[0] * tensor_weights(m.orders[e]) * J).sum()
    assert abs(tot) < 1e-12 * np.abs(r).max()
