"""The C-ABI library builds, loads and exports every function that
include/dg.h declares; host-side argument checks reject bad input without
touching a GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "dg.h")).read()
    return sorted(set(re.findall(r"^(?:dg_status|const char\*)\s+(dg_\w+)\s*\(", src, re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2210_03523_gb300 import build
    build.build()
    from paper_2210_03523_gb300 import dg
    return dg._lib()


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    from paper_2210_03523_gb300 import dg
    assert sorted(dg.exported_symbols()) == names


def test_status_strings(lib):
    for s in range(8):
        assert lib.dg_status_str(s)
        assert b"unknown" not in lib.dg_status_str(s)


def test_count_nodes(lib):
    from paper_2210_03523_gb300 import dg
    o = np.array([[1, 2, 3], [4, 4, 4]], dtype=np.int32)
    assert dg.dg_count_nodes(o) == 2 * 3 * 4 + 125
    with pytest.raises(dg.DGError):
        dg.dg_count_nodes(np.array([[0, 2, 3]], dtype=np.int32))
    with pytest.raises(dg.DGError):
        dg.dg_count_nodes(np.array([[9, 2, 3]], dtype=np.int32))


def _desc(dg, mi):
    d = dg.dg_mesh_desc()
    d.n_elem = mi.n_elem
    d.geom_order = mi.geom_order
    g = np.ascontiguousarray(mi.geom)
    nb = np.ascontiguousarray(mi.neighbors, dtype=np.int32)
    o = np.ascontiguousarray(mi.orders, dtype=np.int32)
    d.geom = g.ctypes.data_as(C.POINTER(C.c_double))
    d.neighbors = nb.ctypes.data_as(C.POINTER(C.c_int32))
    d.orders = o.ctypes.data_as(C.POINTER(C.c_int32))
    ph = mi.phys
    d.phys = dg.dg_physics(ph.eqs, ph.gamma, ph.mu, ph.Pr, ph.Rgas, (C.c_double * 5)(*ph.qinf))
    return d, (g, nb, o)


def test_mesh_create_rejects_bad_input_on_the_host(lib):
    """These inputs fail validation before any CUDA call."""
    from paper_2210_03523_gb300 import dg, inputs as I
    h = C.c_void_p()
    assert lib.dg_mesh_create(None, None, C.byref(h)) == 1
    mi = I.box_mesh(2, orders=(3, 3, 3), phys=I.pulse_physics())
    bad = mi.with_orders(np.full((8, 3), 9))
    d, keep = _desc(dg, bad)
    assert lib.dg_mesh_create(C.byref(d), None, C.byref(h)) == 1
    bad = mi.with_orders(np.zeros((8, 3)))
    d, keep = _desc(dg, bad)
    assert lib.dg_mesh_create(C.byref(d), None, C.byref(h)) == 1
    nb = mi.neighbors.copy()
    nb[0, 1] = 3                  # element 3 does not point back through its -xi1 face
    bad = I.MeshInput(mi.n_elem, mi.geom_order, mi.geom, nb, mi.orders, mi.phys)
    d, keep = _desc(dg, bad)
    assert lib.dg_mesh_create(C.byref(d), None, C.byref(h)) == 1
    nb = mi.neighbors.copy()
    nb[0, 1] = -7                 # unknown boundary tag
    bad = I.MeshInput(mi.n_elem, mi.geom_order, mi.geom, nb, mi.orders, mi.phys)
    d, keep = _desc(dg, bad)
    assert lib.dg_mesh_create(C.byref(d), None, C.byref(h)) == 1
    geom = mi.geom.copy()
    geom[:, :, 0] *= -1.0         # mirrored elements: J < 0
    bad = I.MeshInput(mi.n_elem, mi.geom_order, geom, mi.neighbors, mi.orders, mi.phys)
    d, keep = _desc(dg, bad)
    assert lib.dg_mesh_create(C.byref(d), None, C.byref(h)) == 1
    for fn in ("dg_residual", "dg_rk_step", "dg_max_dt", "dg_set_orders", "dg_get_error", "dg_mesh_destroy",
               "dg_tau_estimate", "dg_node_coords", "dg_advance", "dg_tau_extrapolate", "dg_select_orders",
               "dg_autotune", "dg_get_tiles", "dg_set_tiles", "dg_residual_vjp", "dg_rk_step_vjp",
               "dg_wall_force", "dg_wall_force_vjp", "dg_debug_set_index"):
        f = getattr(lib, fn)
        args = [0 if t in (C.c_uint32, C.c_int32, C.c_int64) else (1.0 if t is C.c_double else None)
                for t in f.argtypes]
        assert f(*args) == 1, fn


def test_bounds_checking_build_builds_and_exports():
    """The -DDG_BOUNDS_CHECK variant compiles and exports the same symbols;
    its debug hook validates arguments on the host."""
    import ctypes as C
    from paper_2210_03523_gb300 import build, dg
    path = build.build(checked=True)
    lib = C.CDLL(path)
    for n in dg.exported_symbols():
        assert hasattr(lib, n), n
    lib.dg_debug_set_index.argtypes = [C.c_void_p, C.c_int32, C.c_int64, C.c_int32, C.POINTER(C.c_int32)]
    assert lib.dg_debug_set_index(None, 0, 0, 0, None) == 1
