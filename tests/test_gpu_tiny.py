"""Exhaustive tiny cases against the oracle, element by element: every order
triple with N_i in {1,2,3} as a single periodic element (its faces are its own
neighbours), and the 27 triples together in one 3x3x3 periodic mesh (a seeded
permutation, so every pair of neighbouring orders meets at a mortar), plus
small far-field, wall and Navier-Stokes meshes.  Residual (face-coupled and
isolated), CFL step, RK3 steps and the FP64 tau sweep, each output scanned
for NaN and infinity, with the sticky error word clear at the end."""
import itertools

import numpy as np
import pytest

from paper_2210_03523_gb300 import inputs as I
from oracle_helpers import rel_err, scale_per_var, state_scale

pytestmark = pytest.mark.gpu

RTOL = 1e-12
TRIPLES = [t for t in itertools.product((1, 2, 3), repeat=3)]


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_03523_gb300 import build
    build.build()
    return torch


def _finite(*arrs):
    for a in arrs:
        assert np.isfinite(a).all()


def _check_case(torch, mi, width=0.6, rk_steps=3, tau=True):
    import oracle
    from paper_2210_03523_gb300 import dg
    om = oracle.Mesh(mi)
    q = I.pulse_state(om.coords(), mi.orders, mi.phys, width=width, center=(0.1, -0.2, 0.05))
    m = dg.Mesh(mi)
    h = 2.0 / max(np.cbrt(mi.n_elem), 1.0)
    qg = torch.from_numpy(q).cuda()
    for isolated in (False, True):
        r = m.residual(qg, isolated=isolated).cpu().numpy()
        ro = om.residual(q, isolated=isolated)
        _finite(r)
        err = rel_err(r, ro, om.off, scale_per_var(q, mi.phys, h))
        assert err.max() < RTOL, (isolated, err)
    dt = om.max_dt(q, 0.5)
    dtg = m.max_dt(qg, 0.5).item()
    assert abs(dtg - dt) <= RTOL * dt
    gg = torch.zeros_like(qg)
    dtd = torch.tensor([dt], dtype=torch.float64, device="cuda")
    qo, go = q.copy(), np.zeros_like(q)
    for _ in range(rk_steps):
        m.rk_step(qg, gg, dtd)
        om.rk_step(qo, go, dt)
    qs = qg.cpu().numpy()
    _finite(qs)
    assert rel_err(qs, qo, om.off, state_scale(qo, om.off)).max() < RTOL
    if tau:
        sweep = I.full_sweep(np.asarray(mi.orders).reshape(-1, 3).max(0))
        tn, tt = m.tau_estimate(qg, sweep)
        on, ot = om.tau(qs, sweep)
        tn, tt = tn.cpu().numpy(), tt.cpu().numpy()
        _finite(tn, tt)
        assert np.array_equal(tn < 0, on < 0)
        s = scale_per_var(qs, mi.phys, h).max()
        Jmax = max(om.metrics(e)[2].max() for e in range(om.n_elem))
        assert np.abs(tn - on).max() <= RTOL * max(np.abs(on).max(), s)
        assert np.abs(tt - ot).max() <= RTOL * max(np.abs(ot).max(), s * Jmax)
    assert m.get_error() == 0


@pytest.mark.parametrize("orders", TRIPLES, ids=lambda t: "%d%d%d" % t)
def test_single_periodic_element(torch_cuda, orders):
    _check_case(torch_cuda, I.box_mesh(1, orders=orders, phys=I.pulse_physics(mach=0.3)))


def test_all_27_triples_in_one_mesh(torch_cuda):
    perm = np.random.default_rng(27).permutation(len(TRIPLES))
    orders = np.array([TRIPLES[i] for i in perm], dtype=np.int32)
    _check_case(torch_cuda, I.box_mesh(3, orders=orders, phys=I.pulse_physics(mach=0.3)), width=0.4)


@pytest.mark.parametrize("shape", [(2, 2, 2), (2, 1, 1), (1, 2, 3)])
def test_far_field_boxes(torch_cuda, shape):
    n = int(np.prod(shape))
    orders = I.random_orders(n, 1, 3, 100 + n)
    mi = I.box_mesh(*shape, orders=orders, phys=I.pulse_physics(mach=0.3), periodic=(False, False, False))
    _check_case(torch_cuda, mi, width=0.4)


def test_walls_two_elements(torch_cuda):
    mi = I.box_mesh(1, 2, 1, orders=I.random_orders(2, 1, 3, 7), phys=I.pulse_physics(mach=0.3),
                    periodic=(True, False, True),
                    tags=(I.FAR_FIELD, I.FAR_FIELD, I.WALL, I.WALL, I.FAR_FIELD, I.FAR_FIELD))
    _check_case(torch_cuda, mi, width=0.4)


@pytest.mark.parametrize("orders", [(1, 1, 1), (1, 2, 3), (3, 2, 1), (3, 3, 3)], ids=lambda t: "%d%d%d" % t)
def test_navier_stokes_tiny(torch_cuda, orders):
    """conforming Navier-Stokes meshes (one order triple per mesh): a single
    periodic element and a 2x2x1 block with far-field sides"""
    ph = I.Physics(1, 1.4, 0.05, 0.72, 2.0, (1.0, 0.4, -0.3, 0.2, 8.0))
    _check_case(torch_cuda, I.box_mesh(1, orders=orders, phys=ph), width=0.8)
    _check_case(torch_cuda, I.box_mesh(2, 2, 1, orders=orders, phys=ph, periodic=(False, False, True)), width=0.8)
