"""Thin ctypes binding of libdg (include/dg.h).

It does argument marshalling only: every step of the hot path runs in the
CUDA library. Device buffers are torch tensors, used for memory and streams
and nothing else. The binding fails loudly when libdg.so has not been built;
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# DG_LIBRARY=checked loads the bounds-checking build (build.build(checked=True))
LIB_PATH = os.path.join(_HERE, "_build_checked" if os.environ.get("DG_LIBRARY") == "checked" else "_build",
                        "libdg.so")

DG_EULER, DG_NAVIER_STOKES = 0, 1
DG_ISOLATED = 0x1
DG_TAU_ISOLATED = 0x1
DG_TAU_FP32 = 0x2
DG_TAU_ACCUM_MAX = 0x4
DG_MAX_ORDER = 8
DG_EXTRAP_DECOUPLED = 0x1
DG_EXTRAP_ACCUM_MAX = 0x2
DG_ADVANCE_EAGER = 0x1
DG_TAU_UNITS_AUTO, DG_TAU_UNITS_GROUPED, DG_TAU_UNITS_SPLIT = 0, 1, 2
KERNELS = {"face_flux": 0, "face_qhat": 1, "gradient": 2, "volume": 3, "max_dt": 4, "tau": 5, "tau_combine": 6,
           "project": 7, "select": 8, "extrap": 9, "mortar": 10, "adjoint": 11}
STATUS = {0: "DG_OK", 1: "DG_ERR_ARG", 2: "DG_ERR_NOMEM", 3: "DG_ERR_CUDA", 4: "DG_ERR_UNSUPPORTED",
          5: "DG_ERR_NONPHYSICAL", 6: "DG_ERR_TIMEOUT", 7: "DG_ERR_INDEX"}
DG_LIST_VOLUME_ELEMENTS, DG_LIST_TAU_ELEMENTS, DG_LIST_FACE_LEFT, DG_LIST_MORTAR_FACES = 0, 1, 2, 3


class DGError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)} ({_lib().dg_status_str(status).decode()})")


class dg_physics(C.Structure):
    _fields_ = [("eqs", C.c_int32), ("gamma", C.c_double), ("mu", C.c_double), ("Pr", C.c_double),
                ("Rgas", C.c_double), ("q_inf", C.c_double * 5)]


class dg_mesh_desc(C.Structure):
    _fields_ = [("n_elem", C.c_int32), ("geom_order", C.c_int32), ("geom", C.POINTER(C.c_double)),
                ("neighbors", C.POINTER(C.c_int32)), ("orders", C.POINTER(C.c_int32)), ("phys", dg_physics)]


class dg_tiles(C.Structure):
    _fields_ = [("vol_budget", C.c_int32 * 4), ("mortar_budget", C.c_int32 * 4), ("vol_ms", C.c_double * 4),
                ("vol_ms_default", C.c_double * 4), ("mortar_ms", C.c_double * 4),
                ("mortar_ms_default", C.c_double * 4)]


def _tiles_dict(t):
    return {k: list(getattr(t, k)) for k, _ in dg_tiles._fields_}


_L = None


def _lib():
    global _L
    if _L is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libdg.so is not built ({LIB_PATH}); run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        vp, i64p, i32p = C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int32)
        L.dg_status_str.restype = C.c_char_p
        L.dg_status_str.argtypes = [C.c_int]
        sig = {
            "dg_mesh_create": [C.POINTER(dg_mesh_desc), vp, C.POINTER(vp)],
            "dg_mesh_destroy": [vp],
            "dg_mesh_info": [vp, i64p, i32p],
            "dg_mesh_layout": [vp, i64p, C.POINTER(vp)],
            "dg_count_nodes": [C.c_int32, i32p, i64p],
            "dg_set_stream": [vp, vp],
            "dg_node_coords": [vp, vp],
            "dg_residual": [vp, vp, vp, C.c_uint32],
            "dg_residual_noalloc": [vp, vp, vp],
            "dg_select_orders": [vp, vp, C.c_int32, i32p, C.c_int32, C.c_double, C.c_int32, C.c_int32, C.c_int32,
                                 C.c_int32, i32p],
            "dg_tau_extrapolate": [vp, vp, C.c_int32, i32p, C.c_int32, i32p, C.c_int32, C.c_int32, C.c_double,
                                   C.c_uint32, vp],
            "dg_advance": [vp, vp, vp, vp, C.c_double, C.c_double, C.c_int64, C.c_uint32, i64p],
            "dg_step_host": [vp, vp, vp, C.c_double, C.c_double, C.c_double, C.c_int64, i32p, C.c_int32, C.c_uint32,
                             vp, vp, C.POINTER(C.c_double)],
            "dg_autotune": [vp, vp, C.c_int32, C.POINTER(dg_tiles)],
            "dg_residual_vjp": [vp, vp, vp, vp, vp],
            "dg_rk_step_vjp": [vp, vp, vp, vp, vp],
            "dg_wall_force": [vp, vp, C.c_int32, vp],
            "dg_debug_set_index": [vp, C.c_int32, C.c_int64, C.c_int32, i32p],
            "dg_state_write": [C.c_char_p, C.c_int32, i32p, C.POINTER(C.c_double), C.c_double],
            "dg_state_info": [C.c_char_p, i32p, i64p, C.POINTER(C.c_double)],
            "dg_state_read": [C.c_char_p, C.c_int32, i32p, C.POINTER(C.c_double), C.POINTER(C.c_double)],
            "dg_wall_force_vjp": [vp, vp, C.c_int32, vp, vp, vp],
            "dg_get_tiles": [vp, C.POINTER(dg_tiles)],
            "dg_set_tiles": [vp, C.POINTER(dg_tiles)],
            "dg_max_dt": [vp, vp, C.c_double, vp],
            "dg_rk_step": [vp, vp, vp, vp],
            "dg_tau_estimate": [vp, vp, vp, i32p, C.c_int32, C.c_uint32, vp, vp],
            "dg_set_orders": [vp, i32p, vp, vp],
            "dg_get_error": [vp],
            "dg_profile_enable": [vp, C.c_int],
            "dg_profile_read": [vp, C.c_int, C.POINTER(C.c_double), i64p],
            "dg_launch_count": [vp, i64p],
            "dg_set_tau_units": [vp, C.c_int32],
            "dg_tau_units_info": [vp, C.c_int32, i32p, i32p, i32p],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_int
        _L = L
    return _L


def exported_symbols():
    return ["dg_mesh_create", "dg_mesh_destroy", "dg_mesh_info", "dg_count_nodes", "dg_set_stream", "dg_node_coords",
            "dg_residual", "dg_max_dt", "dg_rk_step", "dg_tau_estimate", "dg_set_orders", "dg_get_error",
            "dg_status_str", "dg_profile_enable", "dg_profile_read", "dg_launch_count", "dg_residual_noalloc",
            "dg_select_orders", "dg_tau_extrapolate", "dg_advance", "dg_autotune", "dg_get_tiles", "dg_set_tiles",
            "dg_residual_vjp", "dg_rk_step_vjp", "dg_wall_force", "dg_wall_force_vjp", "dg_state_write",
            "dg_state_info", "dg_state_read", "dg_debug_set_index", "dg_set_tau_units", "dg_tau_units_info",
            "dg_step_host", "dg_mesh_layout"]


def _check(st, where):
    if st != 0:
        raise DGError(st, where)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _i32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32).reshape(-1, 3))


def _p32(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def _check_map(t, n_elem, n_cols, device, dtype=None):
    """A device map must be a contiguous [n_elem, n_cols] float32/float64 tensor."""
    import torch
    ok = (isinstance(t, torch.Tensor) and t.device == device and t.is_contiguous() and
          tuple(t.shape) == (n_elem, n_cols) and t.dtype in (torch.float32, torch.float64) and
          (dtype is None or t.dtype == dtype))
    if not ok:
        raise ValueError(f"map: expected a contiguous float32/float64 [{n_elem}, {n_cols}] tensor on {device}")


def _stream_handle(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def dg_count_nodes(orders) -> int:
    o = np.ascontiguousarray(np.asarray(orders, dtype=np.int32).reshape(-1, 3))
    n = C.c_int64()
    _check(_lib().dg_count_nodes(o.shape[0], o.ctypes.data_as(C.POINTER(C.c_int32)), C.byref(n)), "dg_count_nodes")
    return n.value


def save_state(path, orders, q, t=0.0):
    """dg_state_write: orders [n_elem, 3] and the state (a host array or a device
    tensor, copied to the host) at time t."""
    o = np.ascontiguousarray(np.asarray(orders, dtype=np.int32).reshape(-1, 3))
    qh = q.detach().cpu().numpy() if hasattr(q, "detach") else q
    qh = np.ascontiguousarray(qh, dtype=np.float64)
    _check(_lib().dg_state_write(str(path).encode(), o.shape[0], o.ctypes.data_as(C.POINTER(C.c_int32)),
                                 qh.ctypes.data_as(C.POINTER(C.c_double)), float(t)), "dg_state_write")


def load_state(path):
    """dg_state_read: returns (orders [n_elem, 3], host state, t)."""
    ne, nn, t = C.c_int32(), C.c_int64(), C.c_double()
    _check(_lib().dg_state_info(str(path).encode(), C.byref(ne), C.byref(nn), C.byref(t)), "dg_state_info")
    o = np.empty((ne.value, 3), dtype=np.int32)
    q = np.empty(5 * nn.value)
    _check(_lib().dg_state_read(str(path).encode(), ne.value, o.ctypes.data_as(C.POINTER(C.c_int32)),
                                q.ctypes.data_as(C.POINTER(C.c_double)), C.byref(t)), "dg_state_read")
    return o, q, t.value


class Mesh:
    """A libdg mesh built from a ``paper_2210_03523_gb300.inputs.MeshInput``."""

    def __init__(self, mi, stream=None):
        import torch
        self.mi = mi
        self._geom = np.ascontiguousarray(mi.geom, dtype=np.float64)
        self._nbr = np.ascontiguousarray(mi.neighbors, dtype=np.int32)
        self._ord = np.ascontiguousarray(mi.orders, dtype=np.int32)
        ph = mi.phys
        d = dg_mesh_desc()
        d.n_elem = mi.n_elem
        d.geom_order = mi.geom_order
        d.geom = self._geom.ctypes.data_as(C.POINTER(C.c_double))
        d.neighbors = self._nbr.ctypes.data_as(C.POINTER(C.c_int32))
        d.orders = self._ord.ctypes.data_as(C.POINTER(C.c_int32))
        d.phys = dg_physics(ph.eqs, ph.gamma, ph.mu, ph.Pr, ph.Rgas, (C.c_double * 5)(*ph.qinf))
        self.device = torch.device("cuda", torch.cuda.current_device())
        self._stream = stream
        h = C.c_void_p()
        _check(_lib().dg_mesh_create(C.byref(d), _stream_handle(stream), C.byref(h)), "dg_mesh_create")
        self.h = h
        self._refresh()

    def _refresh(self):
        n, e = C.c_int64(), C.c_int32()
        _check(_lib().dg_mesh_info(self.h, C.byref(n), C.byref(e)), "dg_mesh_info")
        self.n_nodes, self.n_elem = n.value, e.value

    def close(self):
        if getattr(self, "h", None):
            _lib().dg_mesh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------
    def new_state(self):
        import torch
        return torch.zeros(5 * self.n_nodes, dtype=torch.float64, device=self.device)

    def set_stream(self, stream):
        self._stream = stream
        _check(_lib().dg_set_stream(self.h, _stream_handle(stream)), "dg_set_stream")

    def layout(self):
        """dg_mesh_layout: (node count, the element node offsets as a torch
        int64 tensor of n_elem + 1 values viewing the mesh's device array: valid
        until set_orders or the mesh's end, not to be written)."""
        import torch
        n = C.c_int64(0)
        ptr = C.c_void_p(0)
        _check(_lib().dg_mesh_layout(self.h, C.byref(n), C.byref(ptr)), "dg_mesh_layout")

        class _View:
            __cuda_array_interface__ = {"shape": (self.n_elem + 1,), "typestr": "<i8",
                                        "data": (ptr.value, False), "version": 2}
        with torch.cuda.device(self.device):
            return n.value, torch.as_tensor(_View(), device=self.device)

    def coords(self):
        import torch
        x = torch.empty(3 * self.n_nodes, dtype=torch.float64, device=self.device)
        _check(_lib().dg_node_coords(self.h, _ptr(x)), "dg_node_coords")
        return x

    def residual(self, q, r=None, isolated=False):
        r = self.new_state() if r is None else r
        self._check_state(q, r)
        _check(_lib().dg_residual(self.h, _ptr(q), _ptr(r), DG_ISOLATED if isolated else 0), "dg_residual")
        return r

    def residual_noalloc(self, q, r):
        """dg_residual_noalloc: same residual, face scratch in the library's fixed
        device array; r must be a caller-allocated state-layout tensor.  The
        C function needs the mesh's device current; this call makes it so."""
        import torch
        self._check_state(q, r)
        with torch.cuda.device(self.device):
            _check(_lib().dg_residual_noalloc(self.h, _ptr(q), _ptr(r)), "dg_residual_noalloc")
        return r

    def max_dt(self, q, cfl, dt=None):
        import torch
        self._check_state(q)
        dt = torch.empty(1, dtype=torch.float64, device=self.device) if dt is None else dt
        _check(_lib().dg_max_dt(self.h, _ptr(q), float(cfl), _ptr(dt)), "dg_max_dt")
        return dt

    def rk_step(self, q, g, dt):
        self._check_state(q, g)
        _check(_lib().dg_rk_step(self.h, _ptr(q), _ptr(g), _ptr(dt)), "dg_rk_step")

    def tau_estimate(self, q, sweep, isolated=True, fp32=False, accumulate=False, r_p=None, map_new=None,
                     map_trad=None, want=(True, True)):
        import torch
        sw = np.ascontiguousarray(np.asarray(sweep, dtype=np.int32).reshape(-1, 3))
        ns = sw.shape[0]
        dt = torch.float32 if fp32 else torch.float64
        if map_new is None and want[0]:
            map_new = torch.empty((self.n_elem, ns), dtype=dt, device=self.device)
        if map_trad is None and want[1]:
            map_trad = torch.empty((self.n_elem, ns), dtype=dt, device=self.device)
        self._check_state(q, r_p)
        for mp in (map_new, map_trad):
            if mp is not None:
                _check_map(mp, self.n_elem, ns, self.device, dt)
        flags = (DG_TAU_ISOLATED if isolated else 0) | (DG_TAU_FP32 if fp32 else 0) | \
                (DG_TAU_ACCUM_MAX if accumulate else 0)
        self._sweep_keep = sw
        _check(_lib().dg_tau_estimate(self.h, _ptr(q), _ptr(r_p), sw.ctypes.data_as(C.POINTER(C.c_int32)), ns, flags,
                                      _ptr(map_new), _ptr(map_trad)), "dg_tau_estimate")
        return map_new, map_trad

    def set_tau_units(self, mode):
        """dg_set_tau_units: DG_TAU_UNITS_AUTO, _GROUPED or _SPLIT (how the
        isolated sweep's entries are split into units of work)."""
        _check(_lib().dg_set_tau_units(self.h, int(mode)), "dg_set_tau_units")

    def tau_units_info(self):
        """dg_tau_units_info: per shared-memory size class of the last isolated
        sweep, (units, units holding two or more groups)."""
        nu, ns_ = (C.c_int32 * 8)(), (C.c_int32 * 8)()
        nc = C.c_int32()
        _check(_lib().dg_tau_units_info(self.h, 8, C.byref(nc), nu, ns_), "dg_tau_units_info")
        return [(nu[k], ns_[k]) for k in range(min(nc.value, 8))]

    def step_host(self, q_in, q_out, t0, t_end, cfl, max_steps, sweep, isolated=True, fp32=True, accumulate=False,
                  map_new=None, map_trad=None):
        """dg_step_host: one pass of time stepping and the tau sweep on host
        buffers (torch CPU tensors, page-locked for asynchronous copies):
        q_in / q_out the state (float64), map_new / map_trad [n_elem][n_sweep]
        (float32 if fp32 else float64, either may be None).  Returns the time
        reached.  The call makes the mesh's device current."""
        sw = np.ascontiguousarray(np.asarray(sweep, dtype=np.int32).reshape(-1, 3))
        n = 5 * self.n_nodes
        mt = "float32" if fp32 else "float64"
        for x, name in ((q_in, "q_in"), (q_out, "q_out")):
            if x.device.type != "cpu" or str(x.dtype) != "torch.float64" or x.numel() != n or not x.is_contiguous():
                raise ValueError(f"{name}: a contiguous CPU float64 tensor of {n} values")
        for x, name in ((map_new, "map_new"), (map_trad, "map_trad")):
            if x is not None and (x.device.type != "cpu" or str(x.dtype) != f"torch.{mt}" or
                                  x.numel() != self.n_elem * sw.shape[0] or not x.is_contiguous()):
                raise ValueError(f"{name}: a contiguous CPU {mt} tensor of n_elem x n_sweep values")
        flags = (DG_TAU_ISOLATED if isolated else 0) | (DG_TAU_FP32 if fp32 else 0) | \
                (DG_TAU_ACCUM_MAX if accumulate else 0)
        import torch
        t = C.c_double(0.0)
        with torch.cuda.device(self.device):
            _check(_lib().dg_step_host(self.h, _ptr(q_in), _ptr(q_out), float(t0), float(t_end), float(cfl),
                                       int(max_steps), sw.ctypes.data_as(C.POINTER(C.c_int32)), sw.shape[0], flags,
                                       _ptr(map_new) if map_new is not None else None,
                                       _ptr(map_trad) if map_trad is not None else None, C.byref(t)),
                   "dg_step_host")
        return t.value

    def set_orders(self, new_orders, q_old):
        import torch
        o = np.ascontiguousarray(np.asarray(new_orders, dtype=np.int32).reshape(-1, 3))
        if o.shape[0] != self.n_elem:
            raise ValueError(f"new_orders: expected [{self.n_elem}, 3]")
        self._check_state(q_old)
        q_new = torch.empty(5 * dg_count_nodes(o), dtype=torch.float64, device=self.device)
        _check(_lib().dg_set_orders(self.h, o.ctypes.data_as(C.POINTER(C.c_int32)), _ptr(q_old), _ptr(q_new)),
               "dg_set_orders")
        self._ord = o
        self._refresh()
        return q_new

    def debug_set_index(self, lst, i, value):
        """dg_debug_set_index (bounds-checking build only): overwrite entry i of
        a work list on the device; returns the previous value."""
        old = C.c_int32()
        _check(_lib().dg_debug_set_index(self.h, int(lst), int(i), int(value), C.byref(old)), "dg_debug_set_index")
        return old.value

    def orders(self):
        """the current element orders, host [n_elem, 3] (a copy)"""
        return self._ord.copy()

    def offsets(self):
        """node offsets of the state layout, host [n_elem + 1] (off_e: element e
        starts at 5 off_e)"""
        n = np.prod(self._ord.astype(np.int64) + 1, axis=1)
        return np.concatenate([[0], np.cumsum(n)]).astype(np.int64)

    def save_state(self, path, q, t=0.0):
        """Checkpoint: this mesh's orders, the device state q and the time t
        (a float or a device scalar) to a dg_state_write file."""
        self._check_state(q)
        save_state(path, self._ord, q, float(t))

    def load_state(self, path):
        """Resume from a dg_state_write file of this mesh's elements: adopts the
        file's orders (dg_set_orders when they differ) and returns the state on
        the device and the time as a 1-element float64 device tensor."""
        import torch
        o, qh, t = load_state(path)
        if o.shape[0] != self.n_elem:
            raise ValueError(f"{path}: {o.shape[0]} elements, the mesh has {self.n_elem}")
        if not np.array_equal(o, self._ord):
            self.set_orders(o, self.new_state())
        q = torch.from_numpy(qh).to(self.device)
        return q, torch.tensor([t], dtype=torch.float64, device=self.device)

    def select_orders(self, map_, sweep, tau_max, n_min=1, n_max=DG_MAX_ORDER, jump_rule=0, max_decrease=-1):
        """p-adaptation order selection (approach 2) from a device tau map over
        sweep; max_decrease >= 0 bounds the fall below the current orders.
        Returns host orders [n_elem, 3] for set_orders."""
        import torch
        sw = _i32(sweep)
        _check_map(map_, self.n_elem, sw.shape[0], self.device)
        out = np.empty((self.n_elem, 3), dtype=np.int32)
        _check(_lib().dg_select_orders(self.h, _ptr(map_), int(map_.dtype == torch.float32), _p32(sw), sw.shape[0],
                                       float(tau_max), int(n_min), int(n_max), int(jump_rule), int(max_decrease),
                                       _p32(out)), "dg_select_orders")
        return out

    def tau_extrapolate(self, map_, sweep, targets, n_fit=0, tau_floor=0.0, decoupled=False, out=None,
                        accumulate=False):
        """dg_tau_extrapolate: the map over sweep extended to the target list
        (device [n_elem, n_targets], the map's dtype)."""
        import torch
        sw, tg = _i32(sweep), _i32(targets)
        _check_map(map_, self.n_elem, sw.shape[0], self.device)
        if out is None:
            out = torch.empty((self.n_elem, tg.shape[0]), dtype=map_.dtype, device=self.device)
        _check_map(out, self.n_elem, tg.shape[0], self.device, map_.dtype)
        flags = (DG_EXTRAP_DECOUPLED if decoupled else 0) | (DG_EXTRAP_ACCUM_MAX if accumulate else 0)
        _check(_lib().dg_tau_extrapolate(self.h, _ptr(map_), int(map_.dtype == torch.float32), _p32(sw), sw.shape[0],
                                         _p32(tg), tg.shape[0], int(n_fit), float(tau_floor), flags, _ptr(out)),
               "dg_tau_extrapolate")
        return out

    def advance(self, q, g, t, t_end, cfl, max_steps=1 << 40, eager=False, count=False):
        """dg_advance: CFL-adaptive RK3 steps from the device time t (a 1-element
        float64 tensor, updated) to t_end; t_end = inf runs exactly max_steps
        steps asynchronously.  Returns the number of steps when count."""
        import torch
        self._check_state(q, g)
        if not (isinstance(t, torch.Tensor) and t.dtype == torch.float64 and t.numel() >= 1 and t.device == self.device):
            raise ValueError("t: a float64 device tensor")
        n = C.c_int64()
        _check(_lib().dg_advance(self.h, _ptr(q), _ptr(g), _ptr(t), float(t_end), float(cfl), int(max_steps),
                                 DG_ADVANCE_EAGER if eager else 0, C.byref(n) if count else None), "dg_advance")
        return n.value if count else None

    def residual_vjp(self, q, v, out=None, qinf_adj=None):
        """dg_residual_vjp: (dR/dq)^T v at q; qinf_adj (5 doubles, device) accumulates
        the far-field state's cotangent."""
        out = self.new_state() if out is None else out
        self._check_state(q, v, out)
        _check(_lib().dg_residual_vjp(self.h, _ptr(q), _ptr(v), _ptr(out), _ptr(qinf_adj)), "dg_residual_vjp")
        return out

    def rk_step_vjp(self, q0, dt, lam, qinf_adj=None):
        """dg_rk_step_vjp: lam <- (d step(q0) / d q0)^T lam in place, dt a device scalar."""
        self._check_state(q0, lam)
        _check(_lib().dg_rk_step_vjp(self.h, _ptr(q0), _ptr(dt), _ptr(lam), _ptr(qinf_adj)), "dg_rk_step_vjp")
        return lam

    def wall_force(self, q, tag=-2, out=None):
        """dg_wall_force: the force of the fluid on the boundary faces of this tag (3, device)."""
        import torch
        self._check_state(q)
        out = torch.empty(3, dtype=torch.float64, device=self.device) if out is None else out
        _check(_lib().dg_wall_force(self.h, _ptr(q), int(tag), _ptr(out)), "dg_wall_force")
        return out

    def wall_force_vjp(self, q, lam, tag=-2, out=None, scale=None):
        """dg_wall_force_vjp: (dF/dq)^T lam (lam: 3 doubles on the device); with
        scale (device scalar) out += scale * ... instead."""
        out = self.new_state() if out is None else out
        self._check_state(q, out)
        _check(_lib().dg_wall_force_vjp(self.h, _ptr(q), int(tag), _ptr(lam), _ptr(out), _ptr(scale)),
               "dg_wall_force_vjp")
        return out

    def autotune(self, q, reps=5):
        """dg_autotune: time each tile budget per size class on this mesh and
        state, keep the fastest; returns the report as a dict."""
        self._check_state(q)
        t = dg_tiles()
        _check(_lib().dg_autotune(self.h, _ptr(q), int(reps), C.byref(t)), "dg_autotune")
        return _tiles_dict(t)

    def tiles(self):
        t = dg_tiles()
        _check(_lib().dg_get_tiles(self.h, C.byref(t)), "dg_get_tiles")
        return _tiles_dict(t)

    def set_tiles(self, vol_budget, mortar_budget):
        t = dg_tiles()
        t.vol_budget[:] = [int(x) for x in vol_budget]
        t.mortar_budget[:] = [int(x) for x in mortar_budget]
        _check(_lib().dg_set_tiles(self.h, C.byref(t)), "dg_set_tiles")

    def _check_state(self, *states):
        """State-layout device tensors: float64, contiguous, 5 * n_nodes values."""
        import torch
        for x in states:
            if x is None:
                continue
            if not (isinstance(x, torch.Tensor) and x.dtype == torch.float64 and x.is_contiguous() and
                    x.device == self.device and x.numel() == 5 * self.n_nodes):
                raise ValueError(f"state: expected a contiguous float64 tensor of {5 * self.n_nodes} values on "
                                 f"{self.device}")

    def get_error(self):
        return _lib().dg_get_error(self.h)

    def profile_enable(self, on=True):
        _check(_lib().dg_profile_enable(self.h, int(on)), "dg_profile_enable")

    def profile_read(self, kernel):
        ms, n = C.c_double(), C.c_int64()
        _check(_lib().dg_profile_read(self.h, int(kernel), C.byref(ms), C.byref(n)), "dg_profile_read")
        return ms.value, n.value

    def launch_count(self):
        n = C.c_int64()
        _check(_lib().dg_launch_count(self.h, C.byref(n)), "dg_launch_count")
        return n.value
