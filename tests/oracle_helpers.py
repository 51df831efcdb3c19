"""Shared helpers of the oracle pin tests (no method arithmetic beyond what
each test states)."""
import numpy as np
from numpy.polynomial import legendre as npleg


def np_gl(N):
    """Gauss-Lobatto nodes/weights from numpy's Legendre routines."""
    c = np.zeros(N + 1)
    c[N] = 1.0
    inner = np.sort(np.real(npleg.legroots(npleg.legder(c)))) if N > 1 else np.array([])
    x = np.concatenate([[-1.0], inner, [1.0]])
    LN = npleg.legval(x, c)
    w = 2.0 / (N * (N + 1) * LN ** 2)
    return x, w


def np_lagrange_deriv_matrix(x):
    """D_ij = ell_j'(x_i) from numpy polynomial objects."""
    from numpy.polynomial import Polynomial
    n = len(x)
    D = np.empty((n, n))
    for j in range(n):
        others = np.delete(x, j)
        p = Polynomial.fromroots(others)
        p = p / p(x[j])
        D[:, j] = p.deriv()(x)
    return D


def tensor_weights(orders):
    w = [np_gl(int(N))[1] for N in orders]
    return np.einsum("k,j,i->kji", w[2], w[1], w[0]).ravel()


def scale_per_var(q, phys, h):
    """flux scale per variable divided by the element size: the normaliser
    of residual errors (near-zero residuals are compared against it)"""
    qi = np.asarray(phys.qinf)
    u = qi[1:4] / qi[0]
    p = (phys.gamma - 1) * (qi[4] - 0.5 * qi[0] * u @ u)
    c = np.sqrt(phys.gamma * p / qi[0])
    s = np.array([qi[0], qi[0] + p, qi[0] + p, qi[0] + p, qi[4] + p]) * (np.linalg.norm(u) + c) / h
    return s


def rel_err(a, b, nvar_off, s=None):
    """per-variable ||a-b||_inf / max(||b||_inf, s) over a state-layout array"""
    off = nvar_off
    n_el = len(off) - 1
    A = [np.concatenate([a[5 * off[e]:5 * off[e + 1]].reshape(5, -1)[v] for e in range(n_el)]) for v in range(5)]
    B = [np.concatenate([b[5 * off[e]:5 * off[e + 1]].reshape(5, -1)[v] for e in range(n_el)]) for v in range(5)]
    out = []
    for v in range(5):
        den = np.abs(B[v]).max()
        if s is not None:
            den = max(den, s[v])
        out.append(np.abs(A[v] - B[v]).max() / den)
    return np.array(out)


def state_scale(q, off):
    """per-variable state scale: |rho|, the largest momentum component (for all
    three momenta, so an identically-zero component is measured against the
    others), |rho E|"""
    n_el = len(off) - 1
    blk = [q[5 * off[e]:5 * off[e + 1]].reshape(5, -1) for e in range(n_el)]
    mx = np.array([max(np.abs(b[v]).max() for b in blk) for v in range(5)])
    m = mx[1:4].max()
    return np.array([mx[0], m, m, m, mx[4]])
