"""dg_step_host: one pass of the hot path (RK3 steps, then the tau sweep) on
host buffers through the C ABI, the copies inside the call.  Its state, time
and maps must equal, bit for bit, the same calls made on device buffers
(dg_advance, dg_tau_estimate), for a CFL step count and for a given end
time, and its maps must F_max-accumulate across calls."""
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


def _case(torch):
    from paper_2210_03523_gb300 import dg
    mi = I.box_mesh(5, orders=I.random_orders(125, 1, 6, 31), phys=I.pulse_physics())
    m = dg.Mesh(mi)
    q0 = I.pulse_state(m.coords().cpu().numpy(), mi.orders, mi.phys, width=0.3, center=(0.1, 0.2, -0.1))
    sweep = I.full_sweep(np.asarray(mi.orders).max(0))
    return mi, m, q0, sweep


def _device_pass(torch, m, q0, sweep, t_end, steps, fp32, maps=None):
    q = torch.from_numpy(q0).cuda()
    g = torch.zeros_like(q)
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    m.advance(q, g, t, t_end, 0.5, max_steps=steps)
    kw = {} if maps is None else {"map_new": maps[0], "map_trad": maps[1]}
    mn, mt = m.tau_estimate(q, sweep, isolated=True, fp32=fp32, accumulate=maps is not None, **kw)
    return q.cpu(), float(t.item()), mn.cpu(), mt.cpu()


@pytest.mark.parametrize("fp32", [True, False])
@pytest.mark.parametrize("t_end,steps", [(math.inf, 7), (0.05, 1000)])
def test_step_host_equals_the_device_calls(torch_cuda, fp32, t_end, steps):
    torch = torch_cuda
    mi, m, q0, sweep = _case(torch)
    dt = torch.float32 if fp32 else torch.float64
    q_in = torch.from_numpy(q0).pin_memory()
    q_out = torch.empty_like(q_in).pin_memory()
    mn = torch.empty((mi.n_elem, len(sweep)), dtype=dt).pin_memory()
    mt = torch.empty_like(mn).pin_memory()
    t = m.step_host(q_in, q_out, 0.0, t_end, 0.5, steps, sweep, fp32=fp32, map_new=mn, map_trad=mt)
    qd, td, mnd, mtd = _device_pass(torch, m, q0, sweep, t_end, steps, fp32)
    assert torch.equal(q_out, qd)
    assert t == td
    if math.isfinite(t_end):
        assert t == t_end
    assert torch.equal(mn, mnd) and torch.equal(mt, mtd)
    assert torch.equal(q_in, torch.from_numpy(q0))   # the input is not written
    assert m.get_error() == 0


def test_step_host_accumulates_and_takes_pageable_buffers(torch_cuda):
    """Two calls with F_max accumulation (the second from the first's end
    state) equal two accumulating device passes; plain (pageable) host
    tensors work as well, with synchronous copies."""
    torch = torch_cuda
    mi, m, q0, sweep = _case(torch)
    q_a = torch.from_numpy(q0.copy())
    q_b = torch.empty_like(q_a)
    mn = torch.empty((mi.n_elem, len(sweep)), dtype=torch.float32)
    mt = torch.empty_like(mn)
    m.step_host(q_a, q_b, 0.0, math.inf, 0.5, 4, sweep, accumulate=True, map_new=mn, map_trad=mt)
    m.step_host(q_b, q_b, 0.0, math.inf, 0.5, 4, sweep, accumulate=True, map_new=mn, map_trad=mt)
    maps = (torch.zeros((mi.n_elem, len(sweep)), dtype=torch.float32, device="cuda"),
            torch.zeros((mi.n_elem, len(sweep)), dtype=torch.float32, device="cuda"))
    q1, _, _, _ = _device_pass(torch, m, q0, sweep, math.inf, 4, True, maps)
    q2, _, mnd, mtd = _device_pass(torch, m, q1.numpy(), sweep, math.inf, 4, True, maps)
    assert torch.equal(q_b, q2)
    assert torch.equal(mn, mnd) and torch.equal(mt, mtd)
    assert m.get_error() == 0


def test_step_host_rejects_bad_arguments(torch_cuda):
    torch = torch_cuda
    from paper_2210_03523_gb300 import dg
    mi, m, q0, sweep = _case(torch)
    q = torch.from_numpy(q0)
    lib = dg._lib()
    sw = np.ascontiguousarray(np.asarray(sweep, dtype=np.int32))
    import ctypes as C
    p = sw.ctypes.data_as(C.POINTER(C.c_int32))
    t = C.c_double(0)
    qp = C.c_void_p(q.data_ptr())
    assert lib.dg_step_host(m.h, qp, qp, 0.0, 1.0, 0.5, 1, p, len(sweep), 0x3, None, None, C.byref(t)) == 1
    assert lib.dg_step_host(m.h, None, qp, 0.0, 1.0, 0.5, 1, p, len(sweep), 0x3, qp, None, C.byref(t)) == 1
    assert lib.dg_step_host(m.h, qp, qp, 0.0, 1.0, 0.5, 1, p, 0, 0x3, qp, None, C.byref(t)) == 1
