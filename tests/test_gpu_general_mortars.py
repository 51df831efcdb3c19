"""Mortars on curved and Navier-Stokes meshes (the general mortar kernels)
against the oracle, element by element: each side's flux from both traces on
the mortar grid with its own J a^dir, BR1 q-hat and viscous-flux averages on
the mortar, L2 projection back to each side.  Residuals (face-coupled), RK3
steps and the non-isolated tau sweep, on curved Euler, affine and curved
Navier-Stokes boxes with mixed orders, and on an O-grid around a cylinder
with walls and far field.  The adjoint through these mortars is checked with
the other adjoint kernels against the oracle's finite-difference Jacobian."""
import numpy as np
import pytest

from paper_2210_03523_gb300 import inputs as I
from oracle_helpers import rel_err, scale_per_var, state_scale

pytestmark = pytest.mark.gpu

RTOL = 1e-12
NS = I.Physics(1, 1.4, 0.05, 0.72, 2.0, (1.0, 0.4, -0.3, 0.2, 8.0))


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_03523_gb300 import build
    build.build()
    return torch


def _ogrid_mixed(seed):
    p0 = 10.0
    ph = I.Physics(1, 1.4, 0.05, 0.72, p0, (1.0, 0.5, 0.1, 0.0, p0 / 0.4 + 0.5 * 0.26))
    mi = I.ogrid_mesh(n_theta=8, n_r=3, ratio=4.0, orders=(3, 3, 1), phys=ph)
    orders = I.random_orders(mi.n_elem, 2, 5, seed)
    orders[:, 2] = 1
    return mi.with_orders(orders)


def _cases():
    return {
        "curved_euler": I.box_mesh(3, geom_order=3, mapping=I.wavy_map(0.08), orders=I.random_orders(27, 1, 5, 61),
                                   phys=I.pulse_physics(mach=0.3)),
        "ns_affine_periodic": I.box_mesh(3, orders=I.random_orders(27, 1, 4, 62), phys=NS),
        "ns_curved_walls": I.box_mesh(3, geom_order=2, mapping=I.wavy_map(0.05), orders=I.random_orders(27, 1, 4, 63),
                                      phys=NS, periodic=(True, False, True),
                                      tags=(I.FAR_FIELD, I.FAR_FIELD, I.WALL, I.WALL, I.FAR_FIELD, I.FAR_FIELD)),
        "ogrid_ns_mixed": _ogrid_mixed(64),
    }


CASES = _cases()


def _state(mi, om):
    if mi.phys.eqs == 0:
        return I.pulse_state(om.coords(), mi.orders, mi.phys, width=0.3)
    qi = np.asarray(mi.phys.qinf)
    u0 = qi[1:4] / qi[0]
    p0 = 0.4 * (qi[4] - 0.5 * qi[0] * u0 @ u0)

    def fn(x, y, z):
        rho = qi[0] * (1.0 + 0.05 * np.sin(1.3 * x + 0.2) * np.cos(0.9 * y))
        u = [u0[0] + 0.05 * np.cos(y + 0.4 * z), u0[1] + 0.04 * np.sin(0.7 * x), u0[2] + 0.03 * np.cos(x - y)]
        p = p0 * (1.0 + 0.02 * np.cos(x + 0.5 * y))
        return np.stack([rho, rho * u[0], rho * u[1], rho * u[2], p / 0.4 + 0.5 * rho * (u[0] ** 2 + u[1] ** 2 + u[2] ** 2)])
    return I.pointwise_state(om.coords(), mi.orders, fn)


def _setup(name):
    import oracle
    mi = CASES[name]
    om = oracle.Mesh(mi)
    return mi, om, _state(mi, om)


def _h(mi):
    return 2.0 / max(np.cbrt(mi.n_elem), 1.0)


@pytest.mark.parametrize("name", list(CASES))
def test_residual_parity(torch_cuda, name):
    torch = torch_cuda
    from paper_2210_03523_gb300 import dg
    mi, om, q = _setup(name)
    orders = np.asarray(mi.orders).reshape(-1, 3)
    assert len({tuple(o) for o in orders}) > 1     # mixed orders: p-nonconforming faces
    m = dg.Mesh(mi)
    r = m.residual(torch.from_numpy(q).cuda()).cpu().numpy()
    ro = om.residual(q)
    assert np.isfinite(r).all()
    err = rel_err(r, ro, om.off, scale_per_var(q, mi.phys, _h(mi)))
    assert err.max() < RTOL, err
    assert m.get_error() == 0


@pytest.mark.parametrize("name", ["curved_euler", "ns_curved_walls", "ogrid_ns_mixed"])
def test_rk3_parity(torch_cuda, name):
    torch = torch_cuda
    from paper_2210_03523_gb300 import dg
    mi, om, q = _setup(name)
    m = dg.Mesh(mi)
    dt = om.max_dt(q, 0.5)
    qg = torch.from_numpy(q).cuda()
    gg = torch.zeros_like(qg)
    dtd = torch.tensor([dt], dtype=torch.float64, device="cuda")
    qo, go = q.copy(), np.zeros_like(q)
    for _ in range(5):
        m.rk_step(qg, gg, dtd)
        om.rk_step(qo, go, dt)
    err = rel_err(qg.cpu().numpy(), qo, om.off, state_scale(qo, om.off))
    assert err.max() < RTOL, err
    assert m.get_error() == 0


@pytest.mark.parametrize("name", ["curved_euler", "ns_affine_periodic"])
def test_tau_non_isolated_parity(torch_cuda, name):
    """non-isolated tau: full residuals of the coarse discretisations, whose
    mortars on these meshes run the general kernels"""
    torch = torch_cuda
    from paper_2210_03523_gb300 import dg
    mi, om, q = _setup(name)
    m = dg.Mesh(mi)
    sweep = np.array([(1, 1, 1), (2, 1, 1), (1, 2, 2), (2, 2, 2), (3, 2, 1)], dtype=np.int32)
    tn, tt = m.tau_estimate(torch.from_numpy(q).cuda(), sweep, isolated=False)
    on, ot = om.tau(q, sweep, isolated=False)
    tn, tt = tn.cpu().numpy(), tt.cpu().numpy()
    assert np.array_equal(tn < 0, on < 0)
    s = scale_per_var(q, mi.phys, _h(mi)).max()
    Jmax = max(om.metrics(e)[2].max() for e in range(om.n_elem))
    assert np.abs(tn - on).max() <= RTOL * max(np.abs(on).max(), s)
    assert np.abs(tt - ot).max() <= RTOL * max(np.abs(ot).max(), s * Jmax)
