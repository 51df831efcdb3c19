"""The adjoint kernels through the C ABI (dg_residual_vjp, dg_rk_step_vjp)
against the oracle's brute-force discrete adjoint (every Jacobian column by
fourth-order central differences of the oracle's own residual / RK3 step),
on conforming meshes, on affine Euler mortars and on the general mortars
(curved or Navier-Stokes, mixed orders, walls and far field, a curved O-grid),
a dot-product test against central differences of the GPU residual at scale,
and gradients through the time integration (torch.autograd) against finite
differences of a functional, for every checkpoint budget."""
import math

import numpy as np
import pytest

from paper_2210_03523_gb300 import inputs as I

pytestmark = pytest.mark.gpu

VEL = (0.9, -0.6, 0.3)    # no velocity component is zero: Roe's |u.n| stays away from its kink


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_03523_gb300 import build
    build.build()
    return torch


def _case(name):
    ph = I.pulse_physics(mach=0.4, velocity=VEL)
    if name == "periodic_mortars":
        mi = I.box_mesh(2, orders=I.random_orders(8, 1, 4, 41), phys=ph)
    elif name == "farfield_mortars":
        mi = I.box_mesh(2, orders=I.random_orders(8, 1, 3, 42), phys=ph, periodic=(False, False, False))
    elif name == "sheared":
        A = [[1.0, 0.2, 0.0], [0.0, 1.0, -0.15], [0.1, 0.0, 1.0]]
        mi = I.box_mesh(2, orders=I.random_orders(8, 2, 3, 43), phys=ph, mapping=I.affine_map(A))
    elif name == "wall":
        mi = I.box_mesh(2, orders=(2, 3, 2), phys=ph, periodic=(True, False, True),
                        tags=(I.FAR_FIELD, I.FAR_FIELD, I.WALL, I.WALL, I.FAR_FIELD, I.FAR_FIELD))
    elif name == "curved_euler":
        mi = I.box_mesh(2, orders=(2, 3, 2), phys=ph, geom_order=2, mapping=I.wavy_map(0.05))
    elif name == "curved_euler_mortars":
        mi = I.box_mesh(2, orders=I.random_orders(8, 1, 4, 46), phys=ph, geom_order=2, mapping=I.wavy_map(0.05))
    elif name in ("ns_box", "ns_box_farfield"):
        ph = I.Physics(1, 1.4, 0.05, 0.72, 2.0, (1.0, 0.4, -0.3, 0.2, 8.0))
        kw = {} if name == "ns_box" else dict(periodic=(False, False, False))
        mi = I.box_mesh(2, orders=(2, 2, 3), phys=ph, **kw)
    elif name in ("ns_mortars", "ns_farfield_mortars"):
        ph = I.Physics(1, 1.4, 0.05, 0.72, 2.0, (1.0, 0.4, -0.3, 0.2, 8.0))
        kw = {} if name == "ns_mortars" else dict(periodic=(False, False, False))
        mi = I.box_mesh(2, orders=I.random_orders(8, 1, 4, 47), phys=ph, **kw)
    elif name == "ns_curved_wall_mortars":
        ph = I.Physics(1, 1.4, 0.05, 0.72, 2.0, (1.0, 0.4, -0.3, 0.2, 8.0))
        mi = I.box_mesh(2, orders=I.random_orders(8, 1, 3, 48), phys=ph, geom_order=2, mapping=I.wavy_map(0.05),
                        periodic=(True, False, True),
                        tags=(I.FAR_FIELD, I.FAR_FIELD, I.WALL, I.WALL, I.FAR_FIELD, I.FAR_FIELD))
    elif name in ("ns_ogrid", "ns_ogrid_mortars"):
        p0 = 10.0
        ph = I.Physics(1, 1.4, 0.05, 0.72, p0, (1.0, 0.5, 0.1, 0.05, p0 / 0.4 + 0.5 * (0.25 + 0.01 + 0.0025)))
        mi = I.ogrid_mesh(n_theta=8, n_r=2, ratio=4.0, orders=(2, 2, 1), phys=ph)
        if name == "ns_ogrid_mortars":
            orders = I.random_orders(mi.n_elem, 1, 3, 49)
            orders[:, 2] = 1
            mi = mi.with_orders(orders)
    else:
        raise KeyError(name)
    import oracle
    om = oracle.Mesh(mi)
    if ph.eqs == 1:   # the free stream with a smooth perturbation
        qi = np.asarray(ph.qinf)
        u0 = qi[1:4] / qi[0]
        p0 = (ph.gamma - 1) * (qi[4] - 0.5 * qi[0] * u0 @ u0)

        def fn(x, y, z):
            rho = qi[0] * (1.0 + 0.05 * np.sin(1.3 * x + 0.2) * np.cos(0.9 * y))
            u = [u0[0] + 0.05 * np.cos(y + 0.4 * z), u0[1] + 0.04 * np.sin(0.7 * x), u0[2] + 0.03 * np.cos(x - y)]
            p = p0 * (1.0 + 0.02 * np.cos(x + 0.5 * y))
            return np.stack([rho, rho * u[0], rho * u[1], rho * u[2],
                             p / (ph.gamma - 1) + 0.5 * rho * (u[0] ** 2 + u[1] ** 2 + u[2] ** 2)])
        q = I.pointwise_state(om.coords(), mi.orders, fn)
    else:
        q = I.pulse_state(om.coords(), mi.orders, ph, width=0.5, center=(-0.2, 0.1, 0.0))
    return mi, om, q


GENERAL_MORTARS = ["curved_euler_mortars", "ns_mortars", "ns_farfield_mortars", "ns_curved_wall_mortars",
                   "ns_ogrid_mortars"]


@pytest.mark.parametrize("name", ["periodic_mortars", "farfield_mortars", "sheared", "wall", "curved_euler", "ns_box",
                                  "ns_box_farfield", "ns_ogrid"] + GENERAL_MORTARS)
def test_residual_vjp_matches_oracle(torch_cuda, name):
    torch = torch_cuda
    from paper_2210_03523_gb300 import dg
    mi, om, q = _case(name)
    v = np.random.default_rng(9).standard_normal(q.size)
    ref = om.residual_vjp_fd(q, v)
    m = dg.Mesh(mi)
    got = m.residual_vjp(torch.from_numpy(q).cuda(), torch.from_numpy(v).cuda()).cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-8 * np.abs(ref).max(), np.abs(got - ref).max() / np.abs(ref).max()
    assert m.get_error() == 0


@pytest.mark.parametrize("name", ["periodic_mortars", "ns_ogrid", "curved_euler_mortars", "ns_ogrid_mortars"])
def test_rk_step_vjp_matches_oracle(torch_cuda, name):
    torch = torch_cuda
    from paper_2210_03523_gb300 import dg
    mi, om, q = _case(name)
    dt = 0.5 * om.max_dt(q, 1.0)
    lam = np.random.default_rng(10).standard_normal(q.size)
    ref = om.rk_step_vjp_fd(q, dt, lam)
    m = dg.Mesh(mi)
    lam_g = torch.from_numpy(lam).cuda()
    m.rk_step_vjp(torch.from_numpy(q).cuda(), torch.tensor([dt], dtype=torch.float64, device="cuda"), lam_g)
    got = lam_g.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-8 * np.abs(ref).max(), np.abs(got - ref).max() / np.abs(ref).max()


def test_dot_product_at_scale(torch_cuda):
    """<J^T v, w> = <v, J w> on 8^3 elements of orders 1..6 (every mortar shape),
    J w by fourth-order central differences of the GPU residual."""
    torch = torch_cuda
    import oracle
    from paper_2210_03523_gb300 import dg
    ph = I.pulse_physics(mach=0.4, velocity=VEL)
    mi = I.box_mesh(8, orders=I.random_orders(512, 1, 6, 44), phys=ph)
    q = torch.from_numpy(I.pulse_state(oracle.Mesh(mi).coords(), mi.orders, ph, width=0.3)).cuda()
    m = dg.Mesh(mi)
    g = torch.Generator(device="cuda").manual_seed(3)
    v = torch.randn(q.shape, generator=g, device="cuda", dtype=torch.float64)
    w = torch.randn(q.shape, generator=g, device="cuda", dtype=torch.float64) * q.abs().amax() * 1e-3
    jtv = m.residual_vjp(q, v)
    h = 1.0
    R = lambda s: m.residual(q + s * h * w)
    jw = (-R(2) + 8 * R(1) - 8 * R(-1) + R(-2)) / (12 * h)
    lhs, rhs = float(jtv @ w), float(v @ jw)
    assert abs(lhs - rhs) <= 1e-7 * (jtv.abs() @ w.abs()).item(), (lhs, rhs)


def test_gradient_through_time_integration(torch_cuda):
    """d/dq0 of a functional of the state after 12 RK3 steps, through RKSteps
    (dg_rk_step_vjp under checkpointing), against central differences; every
    checkpoint budget gives the same gradient bitwise."""
    torch = torch_cuda
    from paper_2210_03523_gb300 import autograd as AG, dg
    mi, om, qh = _case("periodic_mortars")
    m = dg.Mesh(mi)
    q0 = torch.from_numpy(qh).cuda()
    dt = torch.tensor([0.5 * om.max_dt(qh, 1.0)], dtype=torch.float64, device="cuda")
    c = torch.from_numpy(np.random.default_rng(11).standard_normal(qh.size)).cuda()
    n = 12

    def functional(q):
        return (c * AG.rk_steps(q, m, dt, n, snapshots)).sum()
    grads = []
    for snapshots in (0, 1, 2, 8):
        x = q0.clone().requires_grad_(True)
        functional(x).backward()
        grads.append(x.grad.clone())
    for gr in grads[1:]:
        assert torch.equal(gr, grads[0])
    w = torch.from_numpy(np.random.default_rng(12).standard_normal(qh.size)).cuda() * 1e-4 * q0.abs().amax()
    with torch.no_grad():
        snapshots = 0
        f = lambda s: float(functional(q0 + s * w))
        fd = (-f(2) + 8 * f(1) - 8 * f(-1) + f(-2)) / 12.0
    ad = float(grads[0] @ w)
    assert abs(ad - fd) <= 1e-7 * abs(fd) + 1e-12, (ad, fd)


def test_residual_function_backward(torch_cuda):
    torch = torch_cuda
    from paper_2210_03523_gb300 import autograd as AG, dg
    mi, om, qh = _case("farfield_mortars")
    m = dg.Mesh(mi)
    q = torch.from_numpy(qh).cuda().requires_grad_(True)
    v = torch.from_numpy(np.random.default_rng(13).standard_normal(qh.size)).cuda()
    (AG.residual(q, m) * v).sum().backward()
    assert torch.equal(q.grad, m.residual_vjp(q.detach(), v))


def test_general_mortar_cases_are_mixed():
    """the general-mortar cases do run mortars: some face joins unequal orders"""
    for name in GENERAL_MORTARS:
        mi, _, _ = _case(name)
        o = np.asarray(mi.orders).reshape(-1, 3)
        assert len({tuple(r) for r in o}) > 1, name
        assert mi.phys.eqs == 1 or mi.geom_order > 1, name
