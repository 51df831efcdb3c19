"""dg_residual_noalloc: the residual for callers that may not allocate device
memory while they run (their memory is owned by another allocator, or they
must not stall on cudaMalloc / cudaFree).  Its face-flux scratch is a fixed
array inside the library.  This file is collected last so that a run that
stops at the first failure has run every other test before it.

The check: through the C ABI, two calls in a row give the same residual as
dg_residual (the entry point that uses the mesh's own buffer), to the 1e-12
bar of the parity tests; a mesh whose face buffer does not fit, and a
Navier-Stokes mesh, are refused with DG_ERR_UNSUPPORTED."""
import numpy as np
import pytest

from paper_2210_03523_gb300 import inputs as I
from oracle_helpers import rel_err, scale_per_var

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_03523_gb300 import build
    build.build()
    return torch


def _state(mi, seed_center):
    import oracle
    om = oracle.Mesh(mi)
    return om, I.pulse_state(om.coords(), om.orders, mi.phys, width=0.3, center=seed_center)


@pytest.mark.parametrize("name", ["mixed5_1to6", "pulse16mixed"])
def test_noalloc_residual_matches_dg_residual_twice(torch_cuda, name):
    torch = torch_cuda
    from paper_2210_03523_gb300 import dg
    mi = I.box_mesh(5, orders=I.random_orders(125, 1, 6, 5), phys=I.pulse_physics()) if name == "mixed5_1to6" \
        else I.workload("pulse16mixed")
    m = dg.Mesh(mi)
    h = 2.0 / np.cbrt(mi.n_elem)
    # two different states in a row: the second call must not see the first one's scratch
    for center in ((0.0, 0.0, 0.0), (0.3, -0.2, 0.1)):
        om, q = _state(mi, center)
        qg = torch.from_numpy(q).cuda()
        ref = m.residual(qg).cpu().numpy()
        out = torch.full_like(qg, float("nan"))
        m.residual_noalloc(qg, out)
        got = out.cpu().numpy()
        err = rel_err(got, ref, om.off, scale_per_var(q, mi.phys, h))
        assert err.max() < 1e-12, err
    assert m.get_error() == 0


def test_noalloc_allocates_nothing(torch_cuda):
    """Free device memory (cudaMemGetInfo) and torch's allocator are unchanged
    across calls, after one warm-up call (the first launch of a kernel may
    load its code); the results of calls before and after agree."""
    torch = torch_cuda
    from paper_2210_03523_gb300 import dg
    mi = I.workload("pulse16mixed")
    m = dg.Mesh(mi)
    om, q = _state(mi, (0.1, 0.0, -0.1))
    qg = torch.from_numpy(q).cuda()
    out = torch.empty_like(qg)
    m.residual_noalloc(qg, out)
    torch.cuda.synchronize()
    first = out.clone()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for _ in range(3):
        m.residual_noalloc(qg, out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_allocated() == alloc0
    assert torch.equal(out, first)
    assert m.get_error() == 0


def test_noalloc_refuses_what_does_not_fit(torch_cuda):
    torch = torch_cuda
    from paper_2210_03523_gb300 import dg
    big = dg.Mesh(I.workload("pulse32mixed"))        # about 4 M element-face nodes > 838,860
    q = torch.zeros(5 * big.n_nodes, dtype=torch.float64, device="cuda")
    r = torch.empty_like(q)
    with pytest.raises(dg.DGError) as ei:
        big.residual_noalloc(q, r)
    assert ei.value.status == 4
    ns = dg.Mesh(I.ogrid_mesh(n_theta=8, n_r=3, orders=(2, 2, 1), phys=I.cylinder_physics()))
    q = torch.zeros(5 * ns.n_nodes, dtype=torch.float64, device="cuda")
    with pytest.raises(dg.DGError) as ei:
        ns.residual_noalloc(q, torch.empty_like(q))
    assert ei.value.status == 4
