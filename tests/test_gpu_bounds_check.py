"""The bounds-checking build (libdg compiled with -DDG_BOUNDS_CHECK).

A child process loads it (DG_LIBRARY=checked).  On clean meshes its
residuals, RK steps, CFL steps, tau maps (isolated FP64 and FP32,
non-isolated) and adjoint products equal the release build's bit for bit and
the error word stays clear.  Then, one at a time, a bad index is planted in
each work list the kernels read (the volume tiles' element list: an element
out of range and an element of other orders; the tau tiles' element list;
a face record's element; a mortar face's element and direction); every
operation that reads the list returns normally with DG_ERR_INDEX in the
sticky error word, and once the entry is restored the results equal the
clean ones again.  The release build refuses to plant (DG_ERR_UNSUPPORTED),
so a bad index never reaches kernels that do not check."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_03523_gb300 import build
    build.build()
    build.build(checked=True)
    return torch


def _meshes():
    from paper_2210_03523_gb300 import inputs as I
    euler = I.box_mesh(3, orders=I.random_orders(27, 1, 5, 8), phys=I.pulse_physics(mach=0.3),
                       periodic=(False, False, False))
    ph = I.Physics(1, 1.4, 0.05, 0.72, 2.0, (1.0, 0.4, -0.3, 0.2, 8.0))
    ns = I.box_mesh(2, geom_order=2, mapping=I.wavy_map(0.05), orders=(2, 3, 2), phys=ph,
                    periodic=(True, False, True),
                    tags=(I.FAR_FIELD, I.FAR_FIELD, I.WALL, I.WALL, I.FAR_FIELD, I.FAR_FIELD))
    return {"euler_mortars": euler, "ns_curved_walls": ns}


def _state(mi):
    import oracle
    from paper_2210_03523_gb300 import inputs as I
    return I.pulse_state(oracle.Mesh(mi).coords(), mi.orders, mi.phys, width=0.5, center=(0.1, -0.2, 0.05))


def _compute(dg, torch, name, mi, m=None):
    """every operation on one mesh; numpy outputs by name"""
    from paper_2210_03523_gb300 import inputs as I
    m = m or dg.Mesh(mi)
    q = torch.from_numpy(_state(mi)).cuda()
    out = {"residual": m.residual(q).cpu().numpy(), "residual_iso": m.residual(q, isolated=True).cpu().numpy()}
    dt = m.max_dt(q, 0.5)
    out["dt"] = dt.cpu().numpy()
    qs, g = q.clone(), torch.zeros_like(q)
    for _ in range(3):
        m.rk_step(qs, g, dt)
    out["rk"] = qs.cpu().numpy()
    sweep = I.full_sweep(np.asarray(mi.orders).reshape(-1, 3).max(0))
    for fp32 in (False, True):
        tn, tt = m.tau_estimate(q, sweep, fp32=fp32)
        out[f"tau_new_{int(fp32)}"], out[f"tau_trad_{int(fp32)}"] = tn.cpu().numpy(), tt.cpu().numpy()
    if name == "euler_mortars":
        tn, tt = m.tau_estimate(q, sweep, isolated=False)
        out["tau_noniso"] = tn.cpu().numpy()
    v = torch.from_numpy(np.random.default_rng(4).standard_normal(q.numel())).cuda()
    out["vjp"] = m.residual_vjp(q, v).cpu().numpy()
    if name == "ns_curved_walls":
        out["force"] = m.wall_force(q).cpu().numpy()
    out["error"] = m.get_error()
    return out


def child_main(path):
    """run in a process with DG_LIBRARY=checked"""
    import torch
    from paper_2210_03523_gb300 import dg
    assert os.path.dirname(dg.LIB_PATH).endswith("_build_checked")
    res = {"clean": {}, "planted": []}
    for name, mi in _meshes().items():
        clean = _compute(dg, torch, name, mi)
        np.savez(path + f".{name}.npz", **{k: np.asarray(v) for k, v in clean.items()})
        res["clean"][name] = int(clean["error"])
    # plant one bad index at a time; every reader reports DG_ERR_INDEX
    mi = _meshes()["euler_mortars"]
    q = torch.from_numpy(_state(mi)).cuda()
    v = torch.ones_like(q)
    sweep = np.array([[1, 1, 1], [2, 1, 1]], dtype=np.int32)
    orders = np.asarray(mi.orders).reshape(-1, 3)
    m = dg.Mesh(mi)
    ref = m.residual(q).cpu().numpy()
    assert m.get_error() == 0
    other = int(np.flatnonzero((orders != orders[5]).any(1))[0])

    def ops_volume():
        return [("residual", lambda: m.residual(q)), ("max_dt", lambda: m.max_dt(q, 0.5)),
                ("rk_step", lambda: m.rk_step(q.clone(), torch.zeros_like(q), m.max_dt(q, 0.5))),
                ("residual_vjp", lambda: m.residual_vjp(q, v))]

    plants = [
        (dg.DG_LIST_VOLUME_ELEMENTS, 5, mi.n_elem + 100, ops_volume()),
        (dg.DG_LIST_VOLUME_ELEMENTS, 5, -2, ops_volume()),
        (dg.DG_LIST_TAU_ELEMENTS, 3, -3, [("tau", lambda: m.tau_estimate(q, sweep))]),
        (dg.DG_LIST_FACE_LEFT, 0, mi.n_elem + 7, [("residual", lambda: m.residual(q)),
                                                  ("residual_vjp", lambda: m.residual_vjp(q, v))]),
        (dg.DG_LIST_MORTAR_FACES, 2, 7, [("residual", lambda: m.residual(q)),
                                         ("residual_vjp", lambda: m.residual_vjp(q, v))]),
        (dg.DG_LIST_MORTAR_FACES, 1, -1, [("residual", lambda: m.residual(q))]),
    ]
    # an element of other orders in a tile: its node block would not match the tile's
    vol_list_other = (dg.DG_LIST_VOLUME_ELEMENTS, None, other, [("residual", lambda: m.residual(q))])
    for lst, i, val, ops in plants + [vol_list_other]:
        if i is None:   # the slot of element 5 in the volume list holds 5's id: find it by planting and reading back
            i = 0
            while True:
                old = m.debug_set_index(lst, i, -5)
                m.debug_set_index(lst, i, old)
                if old == 5:
                    break
                i += 1
        old = m.debug_set_index(lst, i, val)
        for what, fn in ops:
            fn()
            status = m.get_error()
            res["planted"].append([int(lst), int(i), int(val), what, int(status)])
        m.debug_set_index(lst, i, old)
        again = m.residual(q).cpu().numpy()
        res["planted"].append([int(lst), int(i), int(val), "restored_equal", int(np.array_equal(again, ref))])
        res["planted"].append([int(lst), int(i), int(val), "restored_error", int(m.get_error())])
    json.dump(res, open(path, "w"))


def test_checked_build_matches_release_and_flags_planted_indices(torch_cuda, tmp_path):
    torch = torch_cuda
    from paper_2210_03523_gb300 import dg
    # the release build refuses to plant
    mi = _meshes()["euler_mortars"]
    m = dg.Mesh(mi)
    with pytest.raises(dg.DGError) as ei:
        m.debug_set_index(dg.DG_LIST_VOLUME_ELEMENTS, 0, 0)
    assert ei.value.status == 4
    path = str(tmp_path / "checked.json")
    env = dict(os.environ, DG_LIBRARY="checked")
    code = (f"import sys; sys.path.insert(0, {ROOT!r}); sys.path.insert(0, {os.path.join(ROOT, 'tests')!r}); "
            f"import test_gpu_bounds_check as t; t.child_main({path!r})")
    r = subprocess.run([sys.executable, "-c", code], env=env, cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    res = json.load(open(path))
    # clean runs: error word clear, every output bitwise the release build's,
    # except FP32 tau on Navier-Stokes meshes: the checking build's kernels
    # differ, and the compiler may contract the FP32 viscous terms into
    # multiply-adds differently; those maps agree to FP32 rounding
    for name, mi in _meshes().items():
        assert res["clean"][name] == 0, name
        rel = _compute(dg, torch, name, mi)
        chk = np.load(path + f".{name}.npz")
        for k, a in rel.items():
            a = np.asarray(a)
            if k.endswith("_1") and name.startswith("ns"):
                assert np.abs(a - chk[k]).max() <= 64 * np.finfo(np.float32).eps * np.abs(a).max(), (name, k)
            else:
                assert np.array_equal(a, chk[k]), (name, k)
    # planted indices: DG_ERR_INDEX from every reader, clean again once restored
    for lst, i, val, what, status in res["planted"]:
        if what == "restored_equal":
            assert status == 1, (lst, i, val)
        elif what == "restored_error":
            assert status == 0, (lst, i, val)
        else:
            assert status == 7, (lst, i, val, what, status)
