"""Pins of the oracle's DGSEM residual R = -(M^N)^{-1} F^N(Q), Sec. 2.1,
Eqs. (DGSEMsystem), (DGMassMatrixRight): free-stream preservation, the
density-pulse family's exact reduction to scalar upwind advection,
polynomial exactness across p-nonconforming mortars, discrete
conservation, metric identities."""
import math

import numpy as np
import pytest

from paper_2210_03523_gb300 import inputs as I
from oracle_helpers import np_gl, np_lagrange_deriv_matrix, tensor_weights


def _mesh(orc, mi):
    return orc.Mesh(mi)


def _flux_scale(phys):
    qi = np.asarray(phys.qinf)
    p = (phys.gamma - 1) * (qi[4] - 0.5 * (qi[1:4] @ qi[1:4]) / qi[0])
    return qi[4] + p + qi[0]


@pytest.mark.parametrize("case", ["affine_mixed", "sheared_mixed", "wavy_uniform", "wavy_mixed", "ogrid_rest"])
def test_free_stream_preservation(orc, case):
    ph = I.pulse_physics(mach=0.5)
    if case == "affine_mixed":
        mi = I.box_mesh(3, orders=I.random_orders(27, 1, 6, 7), phys=ph)
    elif case == "sheared_mixed":
        A = [[1.0, 0.3, 0.1], [0.0, 0.9, -0.2], [0.1, 0.0, 1.2]]
        mi = I.box_mesh(3, mapping=I.affine_map(A), orders=I.random_orders(27, 1, 5, 8), phys=ph)
    elif case == "wavy_uniform":
        mi = I.box_mesh(3, geom_order=3, mapping=I.wavy_map(0.08), orders=(4, 3, 5), phys=ph)
    elif case == "wavy_mixed":
        mi = I.box_mesh(3, geom_order=3, mapping=I.wavy_map(0.08), orders=I.random_orders(27, 1, 5, 9), phys=ph)
    else:
        ph = I.Physics(0, 1.4, 0.0, 0.72, 1.0, (1.0, 0.0, 0.0, 0.0, 2.5))
        mi = I.ogrid_mesh(n_theta=12, n_r=4, orders=(3, 3, 1), phys=ph)
    m = _mesh(orc, mi)
    q = I.uniform_state(mi.orders, mi.phys.qinf)
    r = m.residual(q)
    h = 2.0 / 3.0
    # round-off only: relative to the flux scale over the element size
    assert np.abs(r).max() < 1e-12 * _flux_scale(mi.phys) / h * 10
    # and the isolated residual too
    assert np.abs(m.residual(q, isolated=True)).max() < 1e-12 * _flux_scale(mi.phys) / h * 10


def test_curl_form_metric_identities(orc):
    """sum_i D^(i) (J a^i)_n = 0 node by node (Kopriva's conservative curl
    form), on a 3D curved element where the cross-product form fails."""
    mi = I.box_mesh(2, geom_order=3, mapping=I.wavy_map(0.1), orders=(3, 4, 2))
    m = _mesh(orc, mi)
    for e in range(m.n_elem):
        N = m.orders[e]
        X, Ja, J = m.metrics(e)
        ext = (N[2] + 1, N[1] + 1, N[0] + 1)
        Ds = [np_lagrange_deriv_matrix(np_gl(int(N[d]))[0]) for d in range(3)]
        for n in range(3):
            s = np.einsum("im,kjm->kji", Ds[0], Ja[0, n].reshape(ext)) + \
                np.einsum("jm,kmi->kji", Ds[1], Ja[1, n].reshape(ext)) + \
                np.einsum("km,mji->kji", Ds[2], Ja[2, n].reshape(ext))
            assert np.abs(s).max() < 1e-13


def test_ogrid_volume(orc):
    """sum J w over the O-grid = annulus volume up to the degree-3 geometry
    interpolation error of the arcs (relative ~ (dtheta)^4)."""
    mi = I.ogrid_mesh()
    m = _mesh(orc, mi)
    vol = 0.0
    for e in range(m.n_elem):
        _, _, J = m.metrics(e)
        vol += (J * tensor_weights(m.orders[e])).sum()
    exact = math.pi * (40.0 ** 2 - 0.5 ** 2) * 1.0
    assert abs(vol - exact) / exact < 1e-5
    assert min(m.metrics(e)[2].min() for e in range(m.n_elem)) > 0.0     # right-handed


def test_affine_metrics_closed_form(orc):
    A = np.array([[1.0, 0.3, 0.1], [0.0, 0.9, -0.2], [0.1, 0.0, 1.2]])
    mi = I.box_mesh(2, mapping=I.affine_map(A), orders=(2, 3, 1))
    m = _mesh(orc, mi)
    X, Ja, J = m.metrics(3)
    h = 1.0                                        # 2 elements on [-1,1]
    Jm = A * (h / 2)                               # dX/dxi
    np.testing.assert_allclose(J, np.linalg.det(Jm), rtol=1e-14)
    cof = np.linalg.det(Jm) * np.linalg.inv(Jm)    # rows: J a^i = J grad(xi_i)
    for i in range(3):
        for d in range(3):
            np.testing.assert_allclose(Ja[i, d], cof[i, d], atol=1e-14)


def _pulse_poly_state(coords, orders, phys, coef):
    """pulse family: rho = 1 + polynomial(x), uniform velocity and pressure"""
    qi = np.asarray(phys.qinf)
    u = qi[1:4] / qi[0]
    p0 = (phys.gamma - 1) * (qi[4] - 0.5 * qi[0] * u @ u)

    def fn(x, y, z):
        rho = 2.0 + coef(x, y, z)
        return np.stack([rho, rho * u[0], rho * u[1], rho * u[2], p0 / (phys.gamma - 1) + 0.5 * rho * (u @ u)])
    return I.pointwise_state(coords, orders, fn), u


def _interior(nx):
    """elements of a periodic nx^3 box none of whose faces lies on the seam"""
    out = []
    for iz in range(1, nx - 1):
        for iy in range(1, nx - 1):
            for ix in range(1, nx - 1):
                out.append(ix + nx * (iy + nx * iz))
    return out


@pytest.mark.parametrize("mixed", [False, True])
def test_pulse_family_polynomial_exactness(orc, mixed):
    """rho of degree d_i <= N_i in direction i (all elements), constant u and p:
    R_rho = -u . grad rho exactly at every node of elements away from the
    periodic seam, including across p-nonconforming mortars; momentum and
    energy residuals follow as u R_rho and |u|^2/2 R_rho."""
    ph = I.pulse_physics(mach=0.3, velocity=(0.7, -0.4, 0.25))
    A = [[1.0, 0.2, 0.0], [0.1, 1.0, 0.15], [0.0, -0.1, 0.9]]
    nx = 4
    orders = I.random_orders(nx ** 3, 2, 5, 11) if mixed else (3, 3, 4)
    mi = I.box_mesh(nx, mapping=I.affine_map(A), orders=orders, phys=ph)
    m = _mesh(orc, mi)
    # degree 2 in x, 1 in y, 2 in z (<= the minimum orders 2)
    poly = lambda x, y, z: 0.3 * x * x - 0.2 * x * y + 0.5 * z + 0.1 * z * z * x / 3 + 0.05 * y * z
    dpoly = lambda x, y, z: (0.6 * x - 0.2 * y + 0.1 * z * z / 3, -0.2 * x + 0.05 * z,
                             0.5 + 0.2 * z * x / 3 + 0.05 * y)
    # the state's degree along each reference direction of the sheared affine map is the
    # total degree (2 for x^2, 3 for z^2 x): keep the orders >= 3 when mixed
    if mixed:
        mi = mi.with_orders(np.maximum(mi.orders, 3))
        m = _mesh(orc, mi)
    xyz = m.coords()
    q, u = _pulse_poly_state(xyz, m.orders, ph, poly)
    r = m.residual(q)
    for e in _interior(nx):
        x = m.elem(xyz, e, 3)
        g = np.stack(dpoly(*x))
        R = m.elem(r, e)
        exact = -(u @ g)
        np.testing.assert_allclose(R[0], exact, atol=1e-11)
        for c in range(3):
            np.testing.assert_allclose(R[1 + c], u[c] * exact, atol=1e-10)
        np.testing.assert_allclose(R[4], 0.5 * (u @ u) * exact, atol=1e-10)


def _textbook_upwind_dg(N, nx, u, rho_nodes, h):
    """Scalar linear advection rho_t + u.grad rho = 0 on a periodic nx^3 box of
    axis-aligned cubes of size h, DGSEM strong form with upwind flux, built
    from numpy's Legendre nodes; rho_nodes[e, k, j, i]."""
    x, w = np_gl(N)
    D = np_lagrange_deriv_matrix(x)
    out = np.empty_like(rho_nodes)
    n1 = N + 1
    for e in range(nx ** 3):
        ix, iy, iz = e % nx, (e // nx) % nx, e // (nx * nx)
        r = rho_nodes[e]
        du = (np.einsum("im,kjm->kji", D, r) * u[0] + np.einsum("jm,kmi->kji", D, r) * u[1] +
              np.einsum("km,mji->kji", D, r) * u[2]) * (2.0 / h)
        res = -du
        for d, (ax, uc) in enumerate(zip((2, 1, 0), u)):
            for side in (0, 1):
                step = 1 if side else -1
                j = [ix, iy, iz]
                j[d] = (j[d] + step) % nx
                nb = j[0] + nx * (j[1] + nx * j[2])
                own = np.take(r, N if side else 0, axis=ax)
                oth = np.take(rho_nodes[nb], 0 if side else N, axis=ax)
                # upwind numerical flux through the face in the +x_d direction
                left, right = (own, oth) if side else (oth, own)
                fstar = uc * (left if uc > 0 else right)
                fin = uc * own
                lift = (fstar - fin) * (2.0 / h) / w[-1 if side else 0]
                sl = [slice(None)] * 3
                sl[ax] = N if side else 0
                res[tuple(sl)] += -lift if side else lift
        out[e] = res
    return out


def test_euler_pulse_equals_textbook_scalar_upwind(orc):
    """The Euler operator on the pulse family is scalar upwind DGSEM advection
    of rho (Roe's contact-wave reduction), checked against an independent
    textbook scalar DGSEM, for the residual and for 5 RK3 steps."""
    N, nx = 3, 3
    ph = I.pulse_physics(mach=0.4, velocity=(0.8, -0.5, 0.3))
    mi = I.box_mesh(nx, orders=(N, N, N), phys=ph)
    m = _mesh(orc, mi)
    xyz = m.coords()
    q = I.pulse_state(xyz, m.orders, ph, width=0.35, center=(0.1, -0.2, 0.05))
    u = np.asarray(ph.qinf[1:4])
    h = 2.0 / nx
    rho = np.stack([m.elem(q, e)[0].reshape(N + 1, N + 1, N + 1) for e in range(m.n_elem)])
    ref = _textbook_upwind_dg(N, nx, u, rho, h)
    r = m.residual(q)
    got = np.stack([m.elem(r, e)[0].reshape(N + 1, N + 1, N + 1) for e in range(m.n_elem)])
    np.testing.assert_allclose(got, ref, atol=2e-12 * np.abs(ref).max())
    # five RK3 steps of both
    A, B = orc.rk_coeffs()
    dt = 0.01
    G = np.zeros_like(q)
    qq = q.copy()
    gr = np.zeros_like(rho)
    rr = rho.copy()
    for _ in range(5):
        m.rk_step(qq, G, dt)
        for k in range(3):
            gr = A[k] * gr + dt * _textbook_upwind_dg(N, nx, u, rr, h)
            rr = rr + B[k] * gr
    got = np.stack([m.elem(qq, e)[0].reshape(N + 1, N + 1, N + 1) for e in range(m.n_elem)])
    np.testing.assert_allclose(got, rr, atol=1e-13)


@pytest.mark.parametrize("eqs", [0, 1])
def test_discrete_conservation(orc, eqs):
    """sum_e sum_j w_j J_j R_j = 0 on a periodic mesh (every face flux is
    single-valued, mortars included), for a generic smooth state."""
    ph = I.pulse_physics(mach=0.3) if eqs == 0 else I.Physics(1, 1.4, 0.05, 0.72, 2.0, (1.0, 0.3, 0.1, 0.0, 6.0))
    A = [[1.0, 0.2, 0.0], [0.1, 1.0, 0.15], [0.0, -0.1, 0.9]]
    mi = I.box_mesh(3, mapping=I.affine_map(A), orders=I.random_orders(27, 1, 5, 12), phys=ph)
    m = _mesh(orc, mi)
    xyz = m.coords()

    def fn(x, y, z):
        rho = 1.0 + 0.2 * np.sin(np.pi * x) * np.cos(np.pi * y)
        uu = np.stack([0.3 + 0.1 * np.sin(np.pi * z), 0.1 * np.cos(np.pi * x), 0.05 * np.sin(np.pi * y)])
        p = 2.0 + 0.1 * np.cos(np.pi * (x + z))
        return np.stack([rho, *(rho * uu), p / 0.4 + 0.5 * rho * (uu * uu).sum(0)])
    q = I.pointwise_state(xyz, m.orders, fn)
    r = m.residual(q)
    tot = np.zeros(5)
    for e in range(m.n_elem):
        _, _, J = m.metrics(e)
        tot += (m.elem(r, e) * (tensor_weights(m.orders[e]) * J)[None]).sum(1)
    scale = max(np.abs(r).max(), 1.0)
    assert np.abs(tot).max() < 1e-13 * scale * 27
    assert np.abs(r).max() > 1e-3                      # the state is not trivial
