"""Wall force (drag and lift, Sec. 3.3) and gradients of the time-averaged
drag through the discrete adjoint: dg_wall_force against the oracle, its
vector-Jacobian product against central differences of the oracle's force,
and d(averaged drag)/d(initial state) and d/d(far-field state) against
central differences of the GPU forward run, on a small curved O-grid and on
the full cylinder mesh (400 RK3 steps).

Roe's flux has kinks where u.n = 0 (|u.n| in its dissipation).  At a kink
the Dual derivative is one-sided and a central difference averages the two
sides, so the finite-difference directions keep the spanwise momentum zero,
where the two-dimensional flow sits exactly on that kink at the z faces."""
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


def _ogrid(mu=0.05, w0=0.05):
    p0 = 10.0
    ph = I.Physics(1, 1.4, mu, 0.72, p0, (1.0, 0.5, 0.1, w0, p0 / 0.4 + 0.5 * (0.25 + 0.01 + w0 * w0)))
    return I.ogrid_mesh(n_theta=8, n_r=2, ratio=4.0, orders=(2, 2, 1), phys=ph)


def _state(mi, om):
    ph = mi.phys
    qi = np.asarray(ph.qinf)
    u0 = qi[1:4] / qi[0]
    p0 = (ph.gamma - 1) * (qi[4] - 0.5 * qi[0] * u0 @ u0)

    def fn(x, y, z):
        r2 = x * x + y * y
        damp = 1.0 - np.exp(-(r2 - 0.25) * 4.0)
        rho = qi[0] * (1.0 + 0.05 * np.sin(1.3 * x + 0.2) * np.cos(0.9 * y))
        u = [damp * (u0[0] + 0.05 * np.cos(y)), damp * (u0[1] + 0.04 * np.sin(0.7 * x)), damp * u0[2]]
        p = p0 * (1.0 + 0.02 * np.cos(x + 0.5 * y + 0.7))   # the phase: a net pressure force on the body
        return np.stack([rho, rho * u[0], rho * u[1], rho * u[2],
                         p / (ph.gamma - 1) + 0.5 * rho * (u[0] ** 2 + u[1] ** 2 + u[2] ** 2)])
    return I.pointwise_state(om.coords(), mi.orders, fn)


def _fd4(f, h=1.0):
    return (-f(2 * h) + 8 * f(h) - 8 * f(-h) + f(-2 * h)) / (12 * h)


def test_wall_force_matches_oracle(torch_cuda):
    torch = torch_cuda
    import oracle
    from paper_2210_03523_gb300 import dg
    for mi in (_ogrid(), _ogrid(mu=0.0)):
        if mi.phys.mu == 0.0:
            mi.phys.eqs = 0
        om = oracle.Mesh(mi)
        q = _state(mi, om)
        ref = om.wall_force(q)
        got = dg.Mesh(mi).wall_force(torch.from_numpy(q).cuda()).cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max(), (got, ref)


def test_wall_force_vjp_matches_finite_differences(torch_cuda):
    torch = torch_cuda
    import oracle
    from paper_2210_03523_gb300 import dg
    mi = _ogrid()
    om = oracle.Mesh(mi)
    q = _state(mi, om)
    m = dg.Mesh(mi)
    w = np.random.default_rng(21).standard_normal(q.size) * 1e-3
    for lam in ((1.0, 0.0, 0.0), (0.0, 1.0, 0.0), (0.3, -0.7, 0.2)):
        lam = np.asarray(lam)
        gv = m.wall_force_vjp(torch.from_numpy(q).cuda(), torch.from_numpy(lam).cuda()).cpu().numpy()
        fd = _fd4(lambda s: lam @ om.wall_force(q + s * w))
        assert abs(gv @ w - fd) <= 1e-8 * np.abs(gv * w).sum(), (gv @ w, fd)


def _averaged_force(m, q0, dt, n, direction, tag=-2):
    import torch
    q = q0.clone()
    g = torch.zeros_like(q)
    d = torch.tensor(direction, dtype=torch.float64, device=q0.device)
    J = 0.0
    for _ in range(n):
        m.rk_step(q, g, dt)
        J += float(d @ m.wall_force(q, tag))
    return J / n


def _direction(torch, q0, mi, seed, amp):
    """a seeded random perturbation of every variable but the spanwise momentum"""
    w = I.seeded_perturbation(q0.numel(), seed, amp)
    off = I.node_offsets(mi.orders)
    for e in range(mi.n_elem):
        n = off[e + 1] - off[e]
        w[5 * off[e] + 3 * n: 5 * off[e] + 4 * n] = 0.0
    return torch.from_numpy(w).cuda()


def test_averaged_drag_gradient_small(torch_cuda):
    torch = torch_cuda
    import oracle
    from paper_2210_03523_gb300 import autograd as AG, dg
    mi = _ogrid()
    om = oracle.Mesh(mi)
    qh = _state(mi, om)
    m = dg.Mesh(mi)
    q0 = torch.from_numpy(qh).cuda()
    dt = torch.tensor([0.5 * om.max_dt(qh, 1.0)], dtype=torch.float64, device="cuda")
    n = 20
    J, dq, dqinf = AG.time_averaged_force(m, q0, dt, n, snapshots=3)
    assert J == pytest.approx(_averaged_force(m, q0, dt, n, (1.0, 0.0, 0.0)), rel=1e-13)
    w = _direction(torch, q0, mi, 2211, 1e-3)
    fd = _fd4(lambda s: _averaged_force(m, q0 + s * w, dt, n, (1.0, 0.0, 0.0)))
    assert abs(float(dq @ w) - fd) <= 1e-8 * float((dq * w).abs().sum()), (float(dq @ w), fd)
    # the far-field state: meshes rebuilt around a perturbed q_inf
    import dataclasses
    for k in (0, 1, 2, 4):
        def J_at(s):
            qi = list(mi.phys.qinf)
            qi[k] += s * 1e-4
            mk = dg.Mesh(I.MeshInput(mi.n_elem, mi.geom_order, mi.geom, mi.neighbors, mi.orders,
                                     dataclasses.replace(mi.phys, qinf=tuple(qi))))
            return _averaged_force(mk, q0, dt, n, (1.0, 0.0, 0.0))
        fdk = _fd4(J_at) / 1e-4
        assert float(dqinf[k]) == pytest.approx(fdk, rel=1e-6, abs=1e-10), (k, float(dqinf[k]), fdk)


def test_drag_gradient_through_general_mortars(torch_cuda):
    """the curved Navier-Stokes O-grid with mixed orders, so that the force and
    the time integration both cross the general mortar kernels: the force VJP
    against central differences of the oracle's force, d(averaged drag)/dq0
    against central differences of the GPU forward run.  Flow around the body
    puts face nodes near u.n = 0 (Roe's kink), so the averaged drag is only
    piecewise smooth in q0 and the difference step is small: at steps 1, 1/2,
    1/4, 1/8 the oracle's differences approach the adjoint value as about
    h^1.5 (9.5e-10, 3.2e-10, 1.1e-10, 3.9e-11 away)"""
    torch = torch_cuda
    import oracle
    from paper_2210_03523_gb300 import autograd as AG, dg
    mi = _ogrid()
    orders = I.random_orders(mi.n_elem, 1, 3, 2212)
    orders[:, 2] = 1
    mi = mi.with_orders(orders)
    om = oracle.Mesh(mi)
    qh = _state(mi, om)
    m = dg.Mesh(mi)
    q0 = torch.from_numpy(qh).cuda()
    w = np.random.default_rng(22).standard_normal(qh.size) * 1e-3
    lam = np.asarray((0.6, -0.8, 0.1))
    gv = m.wall_force_vjp(q0, torch.from_numpy(lam).cuda()).cpu().numpy()
    fd = _fd4(lambda s: lam @ om.wall_force(qh + s * w))
    assert abs(gv @ w - fd) <= 1e-8 * np.abs(gv * w).sum(), (gv @ w, fd)
    dt = torch.tensor([0.5 * om.max_dt(qh, 1.0)], dtype=torch.float64, device="cuda")
    n = 10
    J, dq, _ = AG.time_averaged_force(m, q0, dt, n, snapshots=2)
    assert J == pytest.approx(_averaged_force(m, q0, dt, n, (1.0, 0.0, 0.0)), rel=1e-13)
    wd = _direction(torch, q0, mi, 2213, 1e-3)
    fd = _fd4(lambda s: _averaged_force(m, q0 + s * wd, dt, n, (1.0, 0.0, 0.0)), h=0.125)
    assert abs(float(dq @ wd) - fd) <= 1e-8 * float((dq * wd).abs().sum()), (float(dq @ wd), fd)
    assert m.get_error() == 0


def test_cylinder_drag_gradient_400_steps(torch_cuda):
    """The cylinder case (40 x 24 curved elements, geometry order 3, P = (6,6,1),
    Re 100, Ma 0.2): the drag averaged over 400 RK3 steps (t ~ 0.015, about
    0.0025 of a shedding period) and its gradient with respect to the initial
    field (a seeded random perturbation, seed 2211, amplitude 1e-3 rho_inf),
    against central differences of the forward run, with 12 snapshots on the
    binomial schedule."""
    torch = torch_cuda
    import bench
    from paper_2210_03523_gb300 import autograd as AG, dg
    mi = I.workload("cylinder")
    m = dg.Mesh(mi)
    qh = bench.initial_state("cylinder", mi, m.coords().cpu().numpy())
    q0 = torch.from_numpy(qh).cuda()
    dtv = m.max_dt(q0, 0.5)
    n = 400
    J, dq, dqinf = AG.time_averaged_force(m, q0, dtv, n, snapshots=12)
    w = _direction(torch, q0, mi, 2211, 1e-3 * mi.phys.qinf[0])
    fd = _fd4(lambda s: _averaged_force(m, q0 + s * w, dtv, n, (1.0, 0.0, 0.0)))
    assert abs(float(dq @ w) - fd) <= 1e-6 * abs(fd) + 1e-9 * float((dq * w).abs().sum()), (float(dq @ w), fd)
    assert m.get_error() == 0


def test_cylinder_drag_gradient_inflow_state(torch_cuda):
    """d(averaged drag)/d(inflow state) on the cylinder case over 400 RK3 steps
    for a flow started impulsively from the inflow state (autograd.
    impulsive_start: the inflow density, energy and momentum, the momentum
    ramped to rest at the wall).  The inflow state enters through the initial
    field and through the far-field ghost states; torch.autograd composes the
    discrete adjoint's dJ/dq0 and dJ/dq_inf (AveragedForce) with the initial
    field's dependence.  Checked against fourth-order central differences of
    the forward run on meshes built with the perturbed inflow state, for the
    density, the two in-plane momenta and the energy (the spanwise momentum
    sits on Roe's kink at the z faces)."""
    torch = torch_cuda
    import dataclasses
    from paper_2210_03523_gb300 import autograd as AG, dg
    mi = I.workload("cylinder")
    m = dg.Mesh(mi)
    xyz = m.coords()
    qinf = torch.tensor(mi.phys.qinf, dtype=torch.float64, device="cuda", requires_grad=True)
    q0 = AG.impulsive_start(m, qinf, xyz)
    dtv = m.max_dt(q0.detach().contiguous(), 0.5)
    n = 400
    J = AG.averaged_force(q0, qinf, m, dtv, n)
    J.backward()
    g = qinf.grad.cpu().numpy()
    assert m.get_error() == 0

    def J_at(k, s):
        qi = list(mi.phys.qinf)
        qi[k] += s
        mk = dg.Mesh(I.MeshInput(mi.n_elem, mi.geom_order, mi.geom, mi.neighbors, mi.orders,
                                 dataclasses.replace(mi.phys, qinf=tuple(qi))))
        qk = AG.impulsive_start(mk, torch.tensor(qi, dtype=torch.float64, device="cuda"), xyz)
        return _averaged_force(mk, qk.contiguous(), dtv, n, (1.0, 0.0, 0.0))
    for k in (0, 1, 2, 4):
        h = 1e-3 * max(abs(mi.phys.qinf[k]), 1.0)
        fd = _fd4(lambda s: J_at(k, s), h=h)
        assert abs(g[k] - fd) <= 1e-6 * abs(fd) + 1e-9 * abs(float(J)), (k, g[k], fd)
    assert abs(g[1]) > 1e-3 * abs(float(J))    # the drag responds to the inflow momentum
