"""autograd.impulsive_start (the initial state of a flow started impulsively
from the inflow state, differentiable in that state) on the CPU: the state
layout and values against the same recipe evaluated pointwise with numpy, and
its vector-Jacobian product (torch.autograd) against central differences."""
import numpy as np
import torch

from paper_2210_03523_gb300 import autograd as AG, dg, inputs as I


class _LayoutOnly:
    """what impulsive_start reads from a mesh: its orders (the state layout)"""

    def __init__(self, mi):
        self._ord = np.asarray(mi.orders, dtype=np.int32).reshape(-1, 3)

    offsets = dg.Mesh.offsets


def _coords(mi):
    """node coordinates in the dg_node_coords layout from the oracle mesh"""
    import oracle
    return oracle.Mesh(mi).coords()


def test_values_and_layout():
    mi = I.ogrid_mesh(n_theta=8, n_r=2, orders=(2, 3, 1), phys=I.cylinder_physics())
    xyz = _coords(mi)
    qi = np.asarray(mi.phys.qinf)
    q = AG.impulsive_start(_LayoutOnly(mi), torch.tensor(qi), torch.from_numpy(xyz)).numpy()

    def fn(x, y, z):
        d = 1.0 - np.exp(-(x * x + y * y - 0.25) * 8.0)
        ke = 0.5 * (qi[1:4] @ qi[1:4]) / qi[0]
        return np.stack([qi[0] + 0 * x, qi[1] * d, qi[2] * d, qi[3] * d, qi[4] - ke * (1 - d * d)])
    ref = I.pointwise_state(xyz, mi.orders, fn)
    assert np.abs(q - ref).max() <= 1e-14 * np.abs(ref).max()
    # the pressure is the inflow pressure at every node; the wall nodes are at rest
    off = I.node_offsets(mi.orders)
    for e in range(mi.n_elem):
        Q = q[5 * off[e]: 5 * off[e + 1]].reshape(5, -1)
        p = 0.4 * (Q[4] - 0.5 * (Q[1] ** 2 + Q[2] ** 2 + Q[3] ** 2) / Q[0])
        p_inf = 0.4 * (qi[4] - 0.5 * (qi[1:4] @ qi[1:4]) / qi[0])
        assert np.abs(p - p_inf).max() <= 1e-12 * p_inf


def test_vjp_matches_central_differences():
    mi = I.ogrid_mesh(n_theta=8, n_r=2, orders=(2, 2, 1), phys=I.cylinder_physics())
    xyz = torch.from_numpy(_coords(mi))
    lay = _LayoutOnly(mi)
    qi = torch.tensor(mi.phys.qinf, dtype=torch.float64) + torch.tensor([0.0, 0.0, 0.1, 0.05, 0.0])
    w = torch.from_numpy(np.random.default_rng(4).standard_normal(5 * int(lay.offsets()[-1])))
    x = qi.clone().requires_grad_(True)
    (AG.impulsive_start(lay, x, xyz) @ w).backward()
    for k in range(5):
        h = 1e-4 * max(abs(float(qi[k])), 1.0)
        e = torch.zeros(5, dtype=torch.float64)
        e[k] = h
        fd = float((AG.impulsive_start(lay, qi + e, xyz) - AG.impulsive_start(lay, qi - e, xyz)) @ w) / (2 * h)
        assert abs(float(x.grad[k]) - fd) <= 1e-7 * max(abs(fd), 1.0), (k, float(x.grad[k]), fd)
