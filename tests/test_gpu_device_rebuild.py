"""dg_set_orders builds the new mesh's order-dependent parts on the device:
node and face-node offsets, the curved elements' metrics at their new
orders, the elements sorted into order buckets, and the faces classified and
sorted by mortar shape (the tau sweep's coarse-order metric bank is built on
the device too).  A mesh created on the host at the same orders is the
reference: the residual, an RK3 step and the FP64 tau maps of the same state
must agree bit for bit, on the curved Navier-Stokes O-grid and on affine Euler
meshes of mixed orders."""
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


def _cylinder_orders(n, seed):
    o = I.random_orders(n, 1, 6, seed)
    o[:, 2] = 1
    return o


def _state(mi, m):
    xyz = m.coords().cpu().numpy()
    if mi.geom_order > 1:   # the cylinder: free stream slowed near the wall, a small swirl
        ph = mi.phys
        p_inf = (ph.gamma - 1) * (ph.qinf[4] - 0.5)

        def fn(x, y, z):
            r2 = x * x + y * y
            damp = 1.0 - np.exp(-(r2 - 0.25) * 8.0)
            u = damp * (1.0 + 0.05 * np.sin(2.0 * y))
            v = 0.05 * damp * np.exp(-((x - 1.5) ** 2 + y * y))
            rho = 1.0 + 0.01 * np.cos(x)
            return np.stack([rho, rho * u, rho * v, 0 * x, p_inf / (ph.gamma - 1) + 0.5 * rho * (u * u + v * v)])
        return I.pointwise_state(xyz, mi.orders, fn)
    return I.pulse_state(xyz, mi.orders, mi.phys, width=0.3, center=(0.1, -0.2, 0.05))


@pytest.mark.parametrize("case", ["cylinder", "box6_mixed", "pulse16mixed"])
def test_set_orders_mesh_equals_a_mesh_built_on_the_host(torch_cuda, case):
    torch = torch_cuda
    from paper_2210_03523_gb300 import dg
    if case == "cylinder":
        mi = I.workload("cylinder")
        new = _cylinder_orders(mi.n_elem, 7)
    elif case == "box6_mixed":
        mi = I.box_mesh(6, orders=I.random_orders(216, 1, 5, 11), phys=I.pulse_physics())
        new = I.random_orders(216, 1, 6, 12)
    else:
        mi = I.workload("pulse16mixed")
        new = I.random_orders(mi.n_elem, 1, 6, 2211)
    m = dg.Mesh(mi)
    q0 = torch.from_numpy(_state(mi, m)).cuda()
    q = m.set_orders(np.asarray(new, dtype=np.int32), q0)        # device-built mesh
    h = dg.Mesh(mi.with_orders(np.asarray(new, dtype=np.int32)))  # host-built mesh
    assert m.n_nodes == h.n_nodes
    assert torch.equal(m.coords(), h.coords())
    # the device offsets (dg_mesh_layout) of both equal the node counts' prefix sums
    off = I.node_offsets(np.asarray(new, dtype=np.int32))
    for mesh in (m, h):
        n, dev_off = mesh.layout()
        assert n == off[-1]
        torch.cuda.synchronize()
        assert np.array_equal(dev_off.cpu().numpy(), np.asarray(off, dtype=np.int64))
    ra, rb = m.residual(q), h.residual(q)
    assert torch.isfinite(ra).all()
    assert torch.equal(ra, rb)
    ia, ib = m.residual(q, isolated=True), h.residual(q, isolated=True)
    assert torch.equal(ia, ib)
    # one CFL step on each
    qa, qb = q.clone(), q.clone()
    ga, gb = torch.zeros_like(q), torch.zeros_like(q)
    dta = torch.empty(1, dtype=torch.float64, device="cuda")
    dtb = torch.empty_like(dta)
    m.max_dt(qa, 0.5, dta)
    h.max_dt(qb, 0.5, dtb)
    assert torch.equal(dta, dtb)
    m.rk_step(qa, ga, dta)
    h.rk_step(qb, gb, dtb)
    assert torch.equal(qa, qb)
    # FP64 isolated tau over every N <= max P (on the cylinder: the coarse-order
    # metric bank of both meshes comes from the device construction)
    sweep = I.full_sweep(np.asarray(new).max(0))
    ta = m.tau_estimate(q, sweep, isolated=True, fp32=False)
    tb = h.tau_estimate(q, sweep, isolated=True, fp32=False)
    for x, y in zip(ta, tb):
        assert torch.equal(x, y)
    assert m.get_error() == 0 and h.get_error() == 0


def test_set_orders_twice_and_back(torch_cuda):
    """Two order changes in a row on the cylinder, then back to the first
    orders: each mesh equals the host-built one (residual bitwise)."""
    torch = torch_cuda
    from paper_2210_03523_gb300 import dg
    mi = I.workload("cylinder")
    m = dg.Mesh(mi)
    q = torch.from_numpy(_state(mi, m)).cuda()
    for seed in (21, 22):
        o = _cylinder_orders(mi.n_elem, seed)
        q = m.set_orders(o, q)
        h = dg.Mesh(mi.with_orders(o))
        assert torch.equal(m.residual(q), h.residual(q))
    o = np.asarray(mi.orders, dtype=np.int32).reshape(-1, 3)
    q = m.set_orders(o, q)
    h = dg.Mesh(mi)
    assert torch.equal(m.residual(q), h.residual(q))
    assert m.get_error() == 0
