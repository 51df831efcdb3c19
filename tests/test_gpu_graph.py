"""The CFL-adaptive RK3 loop (dg_max_dt + dg_rk_step, device-scalar dt)
captured in a CUDA graph replays exactly the eager launches."""
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


@pytest.mark.parametrize("name", ["pulse4", "pulse16mixed"])
def test_rk_loop_graph_replay_matches_eager(torch_cuda, name):
    torch = torch_cuda
    from paper_2210_03523_gb300 import dg
    mi = I.workload(name)
    m = dg.Mesh(mi)
    q0 = torch.from_numpy(I.pulse_state_fast(m.coords().cpu().numpy(), mi.orders, mi.phys)).cuda()
    steps = 10

    def run(q, g, dt):
        for _ in range(steps):
            m.max_dt(q, 0.5, dt)
            m.rk_step(q, g, dt)

    q, g, dt = q0.clone(), torch.zeros_like(q0), torch.zeros(1, dtype=torch.float64, device="cuda")
    run(q, g, dt)                          # eager (also warms the kernels' attributes up)
    torch.cuda.synchronize()
    q_eager, dt_eager = q.clone(), dt.clone()

    qg, gg, dtg = q0.clone(), torch.zeros_like(q0), torch.zeros(1, dtype=torch.float64, device="cuda")
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        with torch.cuda.graph(graph):
            m.set_stream(torch.cuda.current_stream())
            run(qg, gg, dtg)
    m.set_stream(torch.cuda.current_stream())
    torch.cuda.synchronize()
    qg.copy_(q0)
    gg.zero_()
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(qg, q_eager) and torch.equal(dtg, dt_eager)
    assert m.get_error() == 0
    # replay is repeatable
    qg.copy_(q0)
    gg.zero_()
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(qg, q_eager)
