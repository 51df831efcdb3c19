"""Physics check of the Navier-Stokes path: vortex shedding behind the
cylinder at Re = 100 (Sec. 3.2 expects a shedding period of about 6 time
units, D = U_inf = 1).  A long run (about 10^5 RK3 steps), opt-in with
DG_LONG=1: the CFL-adaptive RK loop runs as CUDA-graph chunks, the
cross-stream velocity v is sampled at a wake probe, and the period is the
mean spacing of its upward zero crossings over the last oscillations."""
import math
import os

import numpy as np
import pytest

from paper_2210_03523_gb300 import inputs as I

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.mark.skipif(os.environ.get("DG_LONG") != "1", reason="long run; set DG_LONG=1")
def test_cylinder_shedding_period():
    import torch
    from paper_2210_03523_gb300 import build, dg
    build.build()
    ph = I.cylinder_physics()
    mi = I.ogrid_mesh(orders=(4, 4, 1), phys=ph)
    m = dg.Mesh(mi)
    xyz = m.coords().cpu().numpy()
    p_inf = (ph.gamma - 1) * (ph.qinf[4] - 0.5)

    def fn(x, y, z):
        # free stream slowed near the wall, plus an off-axis vortex behind the
        # cylinder that breaks the symmetry
        r2 = x * x + y * y
        damp = 1.0 - np.exp(-(r2 - 0.25) * 8.0)
        g = 0.5 * np.exp(-((x - 1.5) ** 2 + (y - 0.4) ** 2) / 0.25)
        u = damp * (1.0 - g * (y - 0.4) / 0.5)
        v = damp * g * (x - 1.5) / 0.5
        rho = np.ones_like(x)
        return np.stack([rho, rho * u, rho * v, 0 * x, p_inf / (ph.gamma - 1) + 0.5 * rho * (u * u + v * v)])
    q = torch.from_numpy(I.pointwise_state(xyz, mi.orders, fn)).cuda()
    g = torch.zeros_like(q)
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    # probe: the node closest to (3, 0)
    off = I.node_offsets(mi.orders)
    best = None
    for e in range(mi.n_elem):
        n = off[e + 1] - off[e]
        c = xyz[3 * off[e]:3 * off[e + 1]].reshape(3, n)
        d = (c[0] - 3.0) ** 2 + c[1] ** 2
        k = int(np.argmin(d))
        if best is None or d[k] < best[0]:
            best = (d[k], 5 * off[e] + 2 * n + k)     # rho v at that node
    iv, ir = best[1], best[1] - 2 * (off[1] - off[0])  # rho at the same node (uniform orders)
    chunk = 200
    graph = torch.cuda.CUDAGraph()
    for _ in range(3):                                 # eager warm-up
        m.max_dt(q, 0.5, dt)
        m.rk_step(q, g, dt)
        t += dt
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        with torch.cuda.graph(graph):
            m.set_stream(torch.cuda.current_stream())
            for _ in range(chunk):
                m.max_dt(q, 0.5, dt)
                m.rk_step(q, g, dt)
                t += dt
    m.set_stream(torch.cuda.current_stream())
    times, vs = [], []
    t_end = float(os.environ.get("DG_SHEDDING_T", "90"))
    while t.item() < t_end:
        graph.replay()
        torch.cuda.synchronize()
        times.append(t.item())
        vs.append(q[iv].item() / q[ir].item())
    assert m.get_error() == 0
    times, vs = np.array(times), np.array(vs)
    late = times > 0.5 * t_end
    tl, vl = times[late], vs[late] - vs[late].mean()
    up = [tl[i] + (tl[i + 1] - tl[i]) * (-vl[i]) / (vl[i + 1] - vl[i])
          for i in range(len(vl) - 1) if vl[i] < 0 <= vl[i + 1]]
    assert len(up) >= 3, "no sustained shedding"
    period = float(np.mean(np.diff(up)))
    amp = float(np.abs(vl).max())
    print(f"shedding period {period:.3f} (Strouhal {1.0 / period:.4f}), probe v amplitude {amp:.3f}, "
          f"{len(up)} crossings, t_end {t_end}")
    assert abs(period - 6.0) / 6.0 < 0.10
