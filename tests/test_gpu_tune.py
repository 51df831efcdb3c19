"""The tile-shape autotuner (dg_autotune) and fixed budgets (dg_set_tiles):
tiling changes no node's arithmetic, so the residual and the RK step must be
bitwise the same for every budget; the tuner keeps, per size class, a budget
no slower than the default."""
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


def _mesh(torch, nx=5, lo=1, hi=8, seed=17):
    import oracle
    from paper_2210_03523_gb300 import dg
    ph = I.pulse_physics(mach=0.3)
    mi = I.box_mesh(nx, orders=I.random_orders(nx ** 3, lo, hi, seed), phys=ph)
    q = I.pulse_state(oracle.Mesh(mi).coords(), mi.orders, ph, width=0.3)
    return dg.Mesh(mi), torch.from_numpy(q).cuda()


def test_budgets_change_no_result(torch_cuda):
    torch = torch_cuda
    m, q = _mesh(torch)
    r0 = m.residual(q)
    q1, g1 = q.clone(), torch.zeros_like(q)
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    m.advance(q1, g1, t, math.inf, 0.5, max_steps=3, eager=True)
    for vb, mb in (([64, 1, 512, 1024], [1, 64, 384, 100]), ([1000, 96, 32, 7], [512, 512, 8, 300])):
        m.set_tiles(vb, mb)
        assert m.tiles()["vol_budget"] == vb and m.tiles()["mortar_budget"] == mb
        assert torch.equal(m.residual(q), r0)
        q2, g2 = q.clone(), torch.zeros_like(q)
        t.zero_()
        m.advance(q2, g2, t, math.inf, 0.5, max_steps=3)
        assert torch.equal(q2, q1)
    assert m.get_error() == 0
    from paper_2210_03523_gb300 import dg
    for vb, mb in (([1025, 1, 1, 1], [1, 1, 1, 1]), ([1, 1, 1, 1], [1, 513, 1, 1]), ([0, 1, 1, 1], [1, 1, 1, 1])):
        with pytest.raises(dg.DGError):
            m.set_tiles(vb, mb)


def test_autotune_keeps_the_fastest(torch_cuda):
    torch = torch_cuda
    m, q = _mesh(torch, nx=8)
    r0 = m.residual(q)
    rep = m.autotune(q, reps=3)
    for k in range(4):
        for a, d in (("vol_ms", "vol_ms_default"), ("mortar_ms", "mortar_ms_default")):
            if rep[d][k] >= 0:
                assert rep[a][k] <= rep[d][k]
    assert m.tiles()["vol_budget"] == rep["vol_budget"]
    assert torch.equal(m.residual(q), r0)
    # graphs are rebuilt for the new work lists
    g = torch.zeros_like(q)
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    qa = q.clone()
    m.advance(qa, g, t, math.inf, 0.5, max_steps=40)
    qb = q.clone()
    g.zero_()
    t.zero_()
    m.advance(qb, g, t, math.inf, 0.5, max_steps=40, eager=True)
    assert torch.equal(qa, qb) and m.get_error() == 0
