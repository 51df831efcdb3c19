"""CPU oracle for the DGSEM hot path: a ctypes wrapper around dg_oracle.c.

TEST INFRASTRUCTURE ONLY. Only the tests, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package. The CUDA
product path never does.

The C code (dg_oracle.c) is plain FP64 loops written from the paper's
definitions. Every function there cites the section or equation it follows.
It shares no code with the CUDA library. ``build()`` compiles it with gcc
(OpenMP, no FMA contraction) into ``oracle/_build/liboracle.so``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dg_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

dp = C.POINTER(C.c_double)
ip = C.POINTER(C.c_int)


def build(force: bool = False) -> str:
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-std=c99", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        L.orc_mesh_new.restype = C.c_void_p
        L.orc_mesh_new.argtypes = [C.c_int, C.c_int, dp, ip, ip, C.c_int, C.c_double, C.c_double, C.c_double,
                                   C.c_double, dp]
        L.orc_mesh_free.argtypes = [C.c_void_p]
        L.orc_n_nodes.restype = C.c_long
        L.orc_n_nodes.argtypes = [C.c_void_p]
        L.orc_node_coords.argtypes = [C.c_void_p, dp]
        L.orc_elem_metrics.argtypes = [C.c_void_p, C.c_int, ip, dp, dp, dp]
        L.orc_residual.argtypes = [C.c_void_p, dp, dp, C.c_int]
        L.orc_gradient.argtypes = [C.c_void_p, dp, dp, C.c_int]
        L.orc_rk_step.argtypes = [C.c_void_p, dp, dp, C.c_double]
        L.orc_max_dt.restype = C.c_double
        L.orc_max_dt.argtypes = [C.c_void_p, dp, C.c_double]
        L.orc_tau.argtypes = [C.c_void_p, dp, dp, ip, C.c_int, C.c_int, C.c_int, dp, dp]
        L.orc_isolated_residual_at.argtypes = [C.c_void_p, C.c_int, ip, dp, dp]
        L.orc_set_orders.argtypes = [C.c_void_p, ip, dp, dp]
        L.orc_gl.argtypes = [C.c_int, dp, dp]
        L.orc_dmat.argtypes = [C.c_int, dp]
        L.orc_interp_mat.argtypes = [C.c_int, C.c_int, dp]
        L.orc_proj_mat.argtypes = [C.c_int, C.c_int, dp]
        L.orc_roe.argtypes = [C.c_double, dp, dp, dp, dp]
        L.orc_euler_flux.argtypes = [C.c_double, dp, C.c_int, dp]
        L.orc_visc_flux.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, C.c_double, dp, dp, C.c_int, dp]
        L.orc_rk_coeffs.argtypes = [dp, dp]
        L.orc_select_orders.argtypes = [C.c_int, C.c_int, ip, dp, C.c_double, C.c_int, C.c_int, C.c_int, ip, ip,
                                        C.c_int, ip]
        L.orc_tau_extrapolate.argtypes = [C.c_int, ip, C.c_int, ip, dp, C.c_int, ip, C.c_int, C.c_double, C.c_int,
                                          C.c_int, dp]
        L.orc_residual_vjp_fd.argtypes = [C.c_void_p, dp, dp, C.c_double, C.c_int, dp]
        L.orc_rk_step_vjp_fd.argtypes = [C.c_void_p, dp, C.c_double, dp, C.c_double, dp]
        L.orc_wall_force.argtypes = [C.c_void_p, dp, C.c_int, dp]
        L.orc_advance.restype = C.c_int
        L.orc_advance.argtypes = [C.c_void_p, dp, dp, C.c_double, dp, C.c_double, C.c_int]
        _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(dp)


def _i(a):
    return a.ctypes.data_as(ip)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


# ---------------------------------------------------------------- 1D basis
def gl(N):
    x, w = np.empty(N + 1), np.empty(N + 1)
    lib().orc_gl(N, _d(x), _d(w))
    return x, w


def dmat(N):
    D = np.empty((N + 1, N + 1))
    lib().orc_dmat(N, _d(D))
    return D


def interp_mat(Nf, Nt):
    I = np.empty((Nt + 1, Nf + 1))
    lib().orc_interp_mat(Nf, Nt, _d(I))
    return I


def proj_mat(Nf, Nt):
    P = np.empty((Nt + 1, Nf + 1))
    lib().orc_proj_mat(Nf, Nt, _d(P))
    return P


def rk_coeffs():
    A, B = np.empty(3), np.empty(3)
    lib().orc_rk_coeffs(_d(A), _d(B))
    return A, B


# ----------------------------------------------------------------- fluxes
def roe(gamma, qL, qR, n):
    f = np.empty(5)
    lib().orc_roe(gamma, _d(_f64(qL)), _d(_f64(qR)), _d(_f64(n)), _d(f))
    return f


def euler_flux(gamma, q, d):
    f = np.empty(5)
    lib().orc_euler_flux(gamma, _d(_f64(q)), d, _d(f))
    return f


def visc_flux(phys, q, gq, d):
    """gq[v, c] = d q_v / d x_c"""
    f = np.empty(5)
    lib().orc_visc_flux(phys.eqs, phys.gamma, phys.mu, phys.Pr, phys.Rgas, _d(_f64(q)), _d(_f64(gq).ravel()), d,
                        _d(f))
    return f


# ------------------------------------------------------------------- mesh
class Mesh:
    """Oracle mesh built from a ``MeshInput`` (paper_2210_03523_gb300.inputs)."""

    def __init__(self, mi):
        self.mi = mi
        self.n_elem = mi.n_elem
        self.orders = _i32(mi.orders).reshape(-1, 3)
        ph = mi.phys
        self._geom = _f64(mi.geom)
        self._nbr = _i32(mi.neighbors)
        qinf = _f64(ph.qinf)
        self.h = lib().orc_mesh_new(mi.n_elem, mi.geom_order, _d(self._geom), _i(self._nbr), _i(self.orders),
                                    ph.eqs, ph.gamma, ph.mu, ph.Pr, ph.Rgas, _d(qinf))
        self.n_nodes = lib().orc_n_nodes(self.h)
        n = (self.orders[:, 0] + 1) * (self.orders[:, 1] + 1) * (self.orders[:, 2] + 1)
        self.off = np.concatenate([[0], np.cumsum(n)]).astype(np.int64)

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_mesh_free(self.h)
            self.h = None

    @property
    def n_state(self):
        return 5 * self.n_nodes

    def coords(self):
        x = np.empty(3 * self.n_nodes)
        lib().orc_node_coords(self.h, _d(x))
        return x

    def metrics(self, e, N=None):
        N = _i32(self.orders[e] if N is None else N)
        n = int((N[0] + 1) * (N[1] + 1) * (N[2] + 1))
        X, Ja, J = np.empty(3 * n), np.empty(9 * n), np.empty(n)
        lib().orc_elem_metrics(self.h, e, _i(N), _d(X), _d(Ja), _d(J))
        return X.reshape(3, n), Ja.reshape(3, 3, n), J

    def residual(self, q, isolated=False):
        q = _f64(q)
        r = np.empty_like(q)
        lib().orc_residual(self.h, _d(q), _d(r), int(isolated))
        return r

    def gradient(self, q, isolated=False):
        q = _f64(q)
        g = np.empty(3 * q.size)
        lib().orc_gradient(self.h, _d(q), _d(g), int(isolated))
        return g

    def rk_step(self, q, G, dt):
        """Advances q and the RK register G in place by one RK3 step."""
        assert q.dtype == np.float64 and G.dtype == np.float64 and q.flags.c_contiguous and G.flags.c_contiguous
        lib().orc_rk_step(self.h, _d(q), _d(G), float(dt))

    def max_dt(self, q, cfl):
        return lib().orc_max_dt(self.h, _d(_f64(q)), float(cfl))

    def advance(self, q, G, cfl, t, t_end, max_steps=1 << 30):
        """CFL-adaptive RK3 steps from t to t_end (the last one shortened to
        land on t_end); q and G advance in place.  Returns (t, steps)."""
        assert q.dtype == np.float64 and G.dtype == np.float64 and q.flags.c_contiguous and G.flags.c_contiguous
        tt = C.c_double(t)
        n = lib().orc_advance(self.h, _d(q), _d(G), float(cfl), C.byref(tt), float(t_end), int(max_steps))
        return tt.value, n

    def tau(self, q, sweep, isolated=True, rP=None, accumulate=None):
        """Returns (tau_new, tau_trad) maps [n_elem, n_sweep]; accumulate=(new, trad)
        maps to max-accumulate into (modified in place and returned)."""
        q = _f64(q)
        sweep = _i32(sweep).reshape(-1, 3)
        ns = sweep.shape[0]
        if accumulate is not None:
            tn, tt = accumulate
        else:
            tn, tt = np.empty((self.n_elem, ns)), np.empty((self.n_elem, ns))
        rp = _d(_f64(rP)) if rP is not None else None
        lib().orc_tau(self.h, _d(q), rp, _i(sweep), ns, int(isolated), int(accumulate is not None), _d(tn), _d(tt))
        return tn, tt

    def residual_vjp_fd(self, q, v, eps=1e-3, isolated=False):
        """(dR/dq)^T v by fourth-order central differences of every Jacobian column."""
        q, v = _f64(q), _f64(v)
        out = np.empty_like(q)
        lib().orc_residual_vjp_fd(self.h, _d(q), _d(v), float(eps), int(isolated), _d(out))
        return out

    def rk_step_vjp_fd(self, q, dt, lam, eps=1e-3):
        """(d step(q)/dq)^T lam for one RK3 step of size dt, the same way."""
        q, lam = _f64(q), _f64(lam)
        out = np.empty_like(q)
        lib().orc_rk_step_vjp_fd(self.h, _d(q), float(dt), _d(lam), float(eps), _d(out))
        return out

    def wall_force(self, q, tag=-2):
        """Force of the fluid on the boundary faces with this tag (3 values)."""
        F = np.empty(3)
        lib().orc_wall_force(self.h, _d(_f64(q)), int(tag), _d(F))
        return F

    def isolated_residual_at(self, e, N, qN):
        N = _i32(N)
        qN = _f64(qN)
        R = np.empty_like(qN)
        lib().orc_isolated_residual_at(self.h, e, _i(N), _d(qN), _d(R))
        return R

    def set_orders(self, new_orders, q_old):
        new_orders = _i32(new_orders).reshape(-1, 3)
        n = (new_orders[:, 0] + 1) * (new_orders[:, 1] + 1) * (new_orders[:, 2] + 1)
        q_new = np.empty(5 * int(n.sum()))
        lib().orc_set_orders(self.h, _i(new_orders), _d(_f64(q_old)), _d(q_new))
        return q_new

    # helpers ------------------------------------------------------------
    def elem(self, a, e, nvar=5):
        """view of element e in a state-layout array: [nvar, n_e]"""
        n = self.off[e + 1] - self.off[e]
        return a[nvar * self.off[e]: nvar * self.off[e + 1]].reshape(nvar, n)


def select_orders(map_, sweep, tau_max, n_min, n_max, jump_rule, neighbors, prev=None, max_decrease=-1):
    """Static p-adaptation selection (approach 2) and jump rule: 0 none,
    1 floor(2N/3) (Eq. N23), 2 N-1 (Eq. N_1).  map_: [n_elem, n_sweep].
    prev / max_decrease: an order falls by at most max_decrease below prev
    (dynamic adaptation, Sec. 3.2); max_decrease < 0: no limit."""
    m = _f64(map_)
    n_elem, ns = m.shape
    sw = _i32(sweep).reshape(-1, 3)
    nb = _i32(neighbors).reshape(-1, 6)
    out = np.empty((n_elem, 3), dtype=np.int32)
    pv = _i32(prev).reshape(-1, 3) if prev is not None else None
    lib().orc_select_orders(n_elem, ns, _i(sw), _d(m), float(tau_max), int(n_min), int(n_max), int(jump_rule),
                            _i(nb), _i(pv) if pv is not None else None, int(max_decrease), _i(out))
    return out


def tau_extrapolate(map_, orders, sweep, targets, n_fit=0, decoupled=False, accumulate=None, tau_floor=0.0):
    """Truncation-error extrapolation to N_i >= P_i (reading stated in
    dg_oracle.c).  map_: [n_elem, n_sweep] over sweep; orders: [n_elem, 3]
    (P); targets: [n_target, 3].  Returns [n_elem, n_target]; accumulate: an
    array of that shape to max-accumulate into (modified and returned);
    tau_floor: a direction whose value just below P is at or under it counts
    as resolved."""
    m = _f64(map_)
    n_elem, ns = m.shape
    sw = _i32(sweep).reshape(-1, 3)
    assert sw.shape[0] == ns
    P = _i32(orders).reshape(-1, 3)
    tg = _i32(targets).reshape(-1, 3)
    if accumulate is not None:
        out = accumulate
        assert out.dtype == np.float64 and out.flags.c_contiguous and out.shape == (n_elem, tg.shape[0])
    else:
        out = np.empty((n_elem, tg.shape[0]))
    lib().orc_tau_extrapolate(n_elem, _i(P), ns, _i(sw), _d(m), tg.shape[0], _i(tg), int(n_fit), float(tau_floor),
                              int(decoupled), int(accumulate is not None), _d(out))
    return out
