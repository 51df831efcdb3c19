"""Seeded synthetic inputs: meshes, polynomial orders and initial states.

This module feeds both the CUDA library and the CPU oracle, so it holds none
of the method's arithmetic. It builds:

* geometry as node coordinates on an equispaced (G+1)^3 reference lattice per
  element, sampled from an analytic map;
* face connectivity by index arithmetic on structured grids;
* polynomial orders drawn by ``numpy.random.default_rng(seed)``;
* pointwise initial conditions, as functions of node coordinates that the
  caller supplies.

The workloads stand in for the paper's two test cases. Neither the paper's
841-quad pulse mesh nor its 1282-quad cylinder mesh is available, so:

* Euler density pulse (Sec. 3.1): a periodic cube [-1,1]^3 of straight hexes
  carrying rho = 1 + 0.5 exp(-ln2 |x|^2 / 0.1^2), velocity (1,1,0) and a
  constant pressure set by the Mach number.
* Cylinder at Re=100 (Sec. 3.2): a log-polar O-grid of curved hexes of
  geometry order 3, one element thick and periodic in z, with a no-slip
  adiabatic wall at r=0.5 and a far field at r=40.

Layout shared by both implementations: element e owns
n_e = (N1+1)(N2+1)(N3+1) nodes. Its state starts at 5*sum_{e'<e} n_e' and is
ordered [var][k][j][i].
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

FAR_FIELD = -1
WALL = -2


@dataclass
class Physics:
    """Gas constants and free-stream state (conservative variables)."""
    eqs: int = 0            # 0 Euler, 1 Navier-Stokes
    gamma: float = 1.4
    mu: float = 0.0
    Pr: float = 0.72
    Rgas: float = 1.0
    qinf: tuple = (1.0, 0.0, 0.0, 0.0, 2.5)


@dataclass
class MeshInput:
    n_elem: int
    geom_order: int
    geom: np.ndarray        # float64 [n_elem, (G+1)^3, 3], equispaced lattice, a fastest
    neighbors: np.ndarray   # int32 [n_elem, 6]: faces (-xi1,+xi1,-xi2,+xi2,-xi3,+xi3)
    orders: np.ndarray      # int32 [n_elem, 3]
    phys: Physics = field(default_factory=Physics)

    def with_orders(self, orders) -> "MeshInput":
        o = np.ascontiguousarray(np.asarray(orders, dtype=np.int32).reshape(self.n_elem, 3))
        return MeshInput(self.n_elem, self.geom_order, self.geom, self.neighbors, o, self.phys)


def node_counts(orders) -> np.ndarray:
    o = np.asarray(orders).reshape(-1, 3).astype(np.int64)
    return (o[:, 0] + 1) * (o[:, 1] + 1) * (o[:, 2] + 1)


def node_offsets(orders) -> np.ndarray:
    n = node_counts(orders)
    off = np.zeros(len(n) + 1, dtype=np.int64)
    np.cumsum(n, out=off[1:])
    return off


def _lattice(G):
    t = np.linspace(0.0, 1.0, G + 1)
    c, b, a = np.meshgrid(t, t, t, indexing="ij")
    return a.ravel(), b.ravel(), c.ravel()          # a fastest


def _structured_neighbors(nx, ny, nz, periodic, tags):
    """Face neighbours of an nx*ny*nz block, element e = ix + nx*(iy + ny*iz).
    periodic: 3 bools; tags: boundary tag per face (6 ints) where not periodic."""
    n = nx * ny * nz
    nb = np.empty((n, 6), dtype=np.int32)
    ix, iy, iz = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    ix, iy, iz = ix.ravel(), iy.ravel(), iz.ravel()
    e = ix + nx * (iy + ny * iz)
    dims = (nx, ny, nz)
    idx = [ix, iy, iz]
    for d in range(3):
        for side, step in ((0, -1), (1, 1)):
            j = [a.copy() for a in idx]
            j[d] = j[d] + step
            out = (j[d] < 0) | (j[d] >= dims[d])
            j[d] = j[d] % dims[d]
            other = j[0] + nx * (j[1] + ny * j[2])
            val = np.where(out & (not periodic[d]), tags[2 * d + side], other)
            nb[e, 2 * d + side] = val
    return nb


def box_mesh(nx, ny=None, nz=None, lo=-1.0, hi=1.0, periodic=(True, True, True), tags=(FAR_FIELD,) * 6,
             geom_order=1, mapping=None, orders=(4, 4, 4), phys=None) -> MeshInput:
    """Structured hex block on [lo,hi]^3 with an optional analytic node map.

    ``mapping(x, y, z) -> (x', y', z')`` is applied to every geometry lattice
    node; a smooth map with a period-2 structure keeps periodic meshes watertight."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    G = geom_order
    a, b, c = _lattice(G)
    h = [(hi - lo) / nx, (hi - lo) / ny, (hi - lo) / nz]
    n = nx * ny * nz
    ix, iy, iz = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    e = (ix + nx * (iy + ny * iz)).ravel()
    geom = np.empty((n, (G + 1) ** 3, 3))
    X = lo + (ix.ravel()[:, None] + a[None, :]) * h[0]
    Y = lo + (iy.ravel()[:, None] + b[None, :]) * h[1]
    Z = lo + (iz.ravel()[:, None] + c[None, :]) * h[2]
    if mapping is not None:
        X, Y, Z = mapping(X, Y, Z)
    geom[e, :, 0], geom[e, :, 1], geom[e, :, 2] = X, Y, Z
    nb = _structured_neighbors(nx, ny, nz, periodic, tags)
    o = np.broadcast_to(np.asarray(orders, dtype=np.int32), (n, 3)) if np.ndim(orders) == 1 else orders
    return MeshInput(n, G, np.ascontiguousarray(geom), nb, np.ascontiguousarray(np.asarray(o, dtype=np.int32)),
                     phys or Physics())


def affine_map(A, shift=(0.0, 0.0, 0.0)):
    A = np.asarray(A, dtype=np.float64)

    def f(x, y, z):
        return (A[0, 0] * x + A[0, 1] * y + A[0, 2] * z + shift[0],
                A[1, 0] * x + A[1, 1] * y + A[1, 2] * z + shift[1],
                A[2, 0] * x + A[2, 1] * y + A[2, 2] * z + shift[2])
    return f


def wavy_map(amp=0.05):
    """Smooth period-2 deformation of [-1,1]^3 (keeps periodic faces matched)."""
    s = math.pi

    def f(x, y, z):
        return (x + amp * np.sin(s * x) * np.sin(s * y) * np.sin(s * z),
                y + amp * np.sin(s * (x + 0.5)) * np.sin(s * y) * np.sin(s * (z + 0.25)),
                z + amp * np.sin(s * (x + 0.25)) * np.sin(s * (y + 0.5)) * np.sin(s * z))
    return f


def random_orders(n_elem, lo, hi, seed) -> np.ndarray:
    """Per-element, per-direction orders drawn i.i.d. uniformly from {lo..hi}."""
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(rng.integers(lo, hi + 1, size=(n_elem, 3)).astype(np.int32))


def ogrid_mesh(n_theta=40, n_r=24, r_in=0.5, ratio=80.0, geom_order=3, lz=1.0, orders=(6, 6, 1),
               phys=None) -> MeshInput:
    """Log-polar O-grid around a cylinder of diameter 2*r_in: radii
    r_k = r_in * ratio^(k/n_r), uniform angle, one element of length lz in z.
    Reference directions: xi1 = r, xi2 = theta, xi3 = z (right-handed).
    Element e = ir + n_r*it.  Wall at r_in, far field at the outer radius,
    periodic in theta and in z (a single element is its own z neighbour)."""
    G = geom_order
    a, b, c = _lattice(G)
    n = n_theta * n_r
    geom = np.empty((n, (G + 1) ** 3, 3))
    nb = np.empty((n, 6), dtype=np.int32)
    for it in range(n_theta):
        for ir in range(n_r):
            e = ir + n_r * it
            r = r_in * ratio ** ((ir + a) / n_r)
            th = 2.0 * math.pi * (it + b) / n_theta
            geom[e, :, 0] = r * np.cos(th)
            geom[e, :, 1] = r * np.sin(th)
            geom[e, :, 2] = lz * c
            nb[e, 0] = WALL if ir == 0 else e - 1
            nb[e, 1] = FAR_FIELD if ir == n_r - 1 else e + 1
            nb[e, 2] = ir + n_r * ((it - 1) % n_theta)
            nb[e, 3] = ir + n_r * ((it + 1) % n_theta)
            nb[e, 4] = e
            nb[e, 5] = e
    o = np.broadcast_to(np.asarray(orders, dtype=np.int32), (n, 3))
    return MeshInput(n, G, np.ascontiguousarray(geom), nb, np.ascontiguousarray(o), phys or Physics())


# --------------------------------------------------------------------------
# physical parameters of the workloads
# --------------------------------------------------------------------------

def pulse_physics(mach=0.1, gamma=1.4, velocity=(1.0, 1.0, 0.0)) -> Physics:
    """Euler pulse: rho_inf = 1, |v| = |velocity|, p0 = rho_inf |v|^2 / (gamma Ma^2)."""
    v2 = float(np.dot(velocity, velocity))
    p0 = v2 / (gamma * mach ** 2)
    E = p0 / (gamma - 1.0) + 0.5 * v2
    return Physics(0, gamma, 0.0, 0.72, 1.0, (1.0, velocity[0], velocity[1], velocity[2], E))


def cylinder_physics(Re=100.0, mach=0.2, Pr=0.72, gamma=1.4) -> Physics:
    """rho_inf = U_inf = D = T_inf = 1, p_inf = 1/(gamma Ma^2), R = p_inf, mu = 1/Re."""
    p = 1.0 / (gamma * mach ** 2)
    E = p / (gamma - 1.0) + 0.5
    return Physics(1, gamma, 1.0 / Re, Pr, p, (1.0, 1.0, 0.0, 0.0, E))


def pulse_primitive(x, y, z, amp=0.5, width=0.1, center=(0.0, 0.0, 0.0), period=2.0, images=1):
    """rho = 1 + amp exp(-ln2 |x - c|^2 / width^2), summed over periodic images
    within +-images periods in every direction."""
    rho = np.ones_like(x)
    rng = range(-images, images + 1) if images else [0]
    for i in rng:
        for j in rng:
            for k in rng:
                d2 = (x - center[0] - i * period) ** 2 + (y - center[1] - j * period) ** 2 + \
                     (z - center[2] - k * period) ** 2
                rho = rho + amp * np.exp(-math.log(2.0) * d2 / width ** 2)
    return rho


def pulse_state(coords, orders, phys: Physics, amp=0.5, width=0.1, center=(0.0, 0.0, 0.0), images=1):
    """Conservative state of the advected density pulse at the nodes.
    coords: float64 [3*n_nodes] in the per-element [d][node] layout."""
    off = node_offsets(orders)
    q = np.empty(5 * off[-1])
    u = np.array(phys.qinf[1:4]) / phys.qinf[0]
    p0 = (phys.gamma - 1.0) * (phys.qinf[4] - 0.5 * phys.qinf[0] * float(u @ u))
    for e in range(len(off) - 1):
        n = off[e + 1] - off[e]
        c = coords[3 * off[e]: 3 * off[e + 1]].reshape(3, n)
        rho = pulse_primitive(c[0], c[1], c[2], amp, width, center, images=images)
        blk = q[5 * off[e]: 5 * off[e + 1]].reshape(5, n)
        blk[0] = rho
        blk[1:4] = rho[None, :] * u[:, None]
        blk[4] = p0 / (phys.gamma - 1.0) + 0.5 * rho * float(u @ u)
    return q


def pulse_state_fast(coords, orders, phys: Physics, amp=0.5, width=0.1, center=(0.0, 0.0, 0.0)):
    """Vectorised pulse_state without periodic images (width 0.1 on a period-2
    box: the nearest image contributes below 1e-30)."""
    off = node_offsets(orders)
    n_e = np.diff(off)
    e_of = np.repeat(np.arange(len(n_e)), n_e)
    loc = np.arange(off[-1]) - off[e_of]
    base = 3 * off[e_of] + loc
    x, y, z = coords[base], coords[base + n_e[e_of]], coords[base + 2 * n_e[e_of]]
    rho = 1.0 + amp * np.exp(-math.log(2.0) * ((x - center[0]) ** 2 + (y - center[1]) ** 2 +
                                                (z - center[2]) ** 2) / width ** 2)
    u = np.array(phys.qinf[1:4]) / phys.qinf[0]
    p0 = (phys.gamma - 1.0) * (phys.qinf[4] - 0.5 * phys.qinf[0] * float(u @ u))
    q = np.empty(5 * off[-1])
    qb = 5 * off[e_of] + loc
    q[qb] = rho
    for c in range(3):
        q[qb + (1 + c) * n_e[e_of]] = rho * u[c]
    q[qb + 4 * n_e[e_of]] = p0 / (phys.gamma - 1.0) + 0.5 * rho * float(u @ u)
    return q


def uniform_state(orders, qc) -> np.ndarray:
    off = node_offsets(orders)
    q = np.empty(5 * off[-1])
    for e in range(len(off) - 1):
        n = off[e + 1] - off[e]
        q[5 * off[e]: 5 * off[e + 1]].reshape(5, n)[:] = np.asarray(qc)[:, None]
    return q


def pointwise_state(coords, orders, fn) -> np.ndarray:
    """State from a pointwise function fn(x, y, z) -> (5, n) conservative values."""
    off = node_offsets(orders)
    q = np.empty(5 * off[-1])
    for e in range(len(off) - 1):
        n = off[e + 1] - off[e]
        c = coords[3 * off[e]: 3 * off[e + 1]].reshape(3, n)
        q[5 * off[e]: 5 * off[e + 1]].reshape(5, n)[:] = fn(c[0], c[1], c[2])
    return q


def smooth_state(coords, orders, phys: Physics, amp=0.05, width=0.3) -> np.ndarray:
    """A smooth state in which every conservative variable varies: the
    density pulse of the given width on top of velocity and pressure
    variations of relative size amp (periods 2 and 1 across [-1, 1]^3)."""
    u0 = np.array(phys.qinf[1:4]) / phys.qinf[0]
    p0 = (phys.gamma - 1.0) * (phys.qinf[4] - 0.5 * phys.qinf[0] * float(u0 @ u0))
    s = max(float(np.linalg.norm(u0)), 1.0)

    def fn(x, y, z):
        rho = pulse_primitive(x, y, z, 0.5, width)
        u = u0[0] + amp * s * np.sin(np.pi * x) * np.cos(np.pi * z)
        v = u0[1] + amp * s * np.cos(np.pi * y + 0.3) * np.sin(2 * np.pi * x)
        w = u0[2] + amp * s * np.sin(np.pi * (z - y))
        p = p0 * (1.0 + amp * np.cos(np.pi * x + 0.7) * np.cos(np.pi * y) * np.sin(np.pi * z + 0.2))
        return np.stack([rho, rho * u, rho * v, rho * w, p / (phys.gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w)])
    return pointwise_state(coords, orders, fn)


def seeded_perturbation(n_scalars, seed, amplitude) -> np.ndarray:
    return amplitude * np.random.default_rng(seed).standard_normal(n_scalars)


# --------------------------------------------------------------------------
# the named workloads
# --------------------------------------------------------------------------

def workload(name: str) -> MeshInput:
    """pulse4: 4^3 periodic straight hexes, P=(4,4,4);
    pulse16mixed: 16^3, orders iid U{1..6} (seed 2210);
    pulse32mixed: 32^3, orders iid U{1..6} (seed 2210), a working set above L2;
    cylinder: 40x24x1 curved O-grid, geometry order 3, P=(6,6,1);
    pulse48mixed: 48^3, orders iid U{2..8} (seed 2210);
    pulse48uniform: 48^3, P=(5,5,5);
    pulse24mixed: 24^3, orders iid U{2..8} (seed 2210): the 48^3 mesh's order
    distribution at an eighth of its size (a working set above L2, small
    enough for multi-pass profiler captures)."""
    if name == "pulse4":
        return box_mesh(4, orders=(4, 4, 4), phys=pulse_physics())
    if name == "pulse16mixed":
        return box_mesh(16, orders=random_orders(16 ** 3, 1, 6, 2210), phys=pulse_physics())
    if name == "cylinder":
        return ogrid_mesh(phys=cylinder_physics())
    if name == "pulse32mixed":
        return box_mesh(32, orders=random_orders(32 ** 3, 1, 6, 2210), phys=pulse_physics())
    if name == "pulse48mixed":
        return box_mesh(48, orders=random_orders(48 ** 3, 2, 8, 2210), phys=pulse_physics())
    if name == "pulse24mixed":
        return box_mesh(24, orders=random_orders(24 ** 3, 2, 8, 2210), phys=pulse_physics())
    if name == "pulse48uniform":
        return box_mesh(48, orders=(5, 5, 5), phys=pulse_physics())
    raise KeyError(name)


def full_sweep(P) -> np.ndarray:
    """All anisotropic orders N with 1 <= N_i <= P_i, including P itself
    (whose tau is zero by construction), N3 slowest."""
    P = [int(p) for p in P]
    s = [(a, b, c) for c in range(1, P[2] + 1) for b in range(1, P[1] + 1) for a in range(1, P[0] + 1)]
    return np.ascontiguousarray(np.array(s, dtype=np.int32))
