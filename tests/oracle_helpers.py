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


def fp32_tau_scale(om, q, mi, dn, grad=None):
    """Per element, the size of the terms whose FP32 rounding enters the FP32
    tau sweep, which works on deviations from the element's first-node state
    (q_r): S_e = (sum_i ||D^(P_i)||_inf) F_e max|J a| / min J, with F_e the
    largest term of the flux deviations f(q) - f(q_r) at the element's nodes
    at the size of the operands the sweep forms them from: u' = (m' - u_r
    rho') / rho has the operand scale U = (|m'| + |u_r||rho'|) / rho, p' the
    scale P = (gamma-1) (|E'| + |rho'||u_r|^2/2 + rho (|u_r| U + U^2/2)); mass
    |m'|; momentum |m_r| U + |m'||u| + P; energy |h| U + (|E'| + P)|u|,
    h = E_r + p_r), plus eps32 times the reference flux (the FP32 rounding of
    the reference constants), plus, for Navier-Stokes (grad: the oracle's
    isolated gradient [c][v][node] per element), a bound of the viscous flux.
    dn[N] = ||D^(N)||_inf.  Returns (S_dev, S_full): S_full has the largest
    term of the flux f(q) itself in place of F_e, the size of the FP64
    reference's own rounding (it forms the full fluxes, which cancel in the
    derivative)."""
    gam = mi.phys.gamma
    gm1 = gam - 1.0
    eps = float(np.finfo(np.float32).eps)
    out, full = np.empty(om.n_elem), np.empty(om.n_elem)
    for e in range(om.n_elem):
        Q = om.elem(q, e)
        rho, m, E = Q[0], Q[1:4], Q[4]
        u = m / rho
        p = gm1 * (E - 0.5 * (m * u).sum(0))
        Ff = max(np.abs(m).max(), (np.abs(m[:, None, :] * u[None, :, :]) + np.abs(p)[None, None, :]).max(),
                 np.abs((E + p)[None, :] * u).max())
        ur, pr, mr, Er = u[:, 0], p[0], m[:, 0], E[0]
        h = Er + pr
        dm, dr, dE = m - mr[:, None], rho - rho[0], E - Er
        U = (np.abs(dm) + np.abs(ur)[:, None] * np.abs(dr)[None, :]) / rho                  # [c][node]
        Pd = gm1 * (np.abs(dE) + 0.5 * np.abs(dr) * (ur @ ur) + rho * ((np.abs(ur)[:, None] * U).sum(0)
                                                                        + 0.5 * (U * U).sum(0)))
        mom = np.abs(mr)[:, None, None] * U[None, :, :] + np.abs(dm)[:, None, :] * np.abs(u)[None, :, :]
        F = max(np.abs(dm).max(), (mom + Pd[None, None, :]).max(),
                (abs(h) * U + (np.abs(dE) + Pd)[None, :] * np.abs(u)).max())
        F += eps * max(np.abs(mr).max(), np.abs(np.outer(mr, ur)).max() + abs(pr), abs(h) * np.abs(ur).max())
        if grad is not None:
            n = Q.shape[1]
            g = grad[15 * om.off[e]: 15 * om.off[e + 1]].reshape(3, 5, n)      # [c][v][node]
            gu = (g[:, 1:4, :] - u[None, :, :] * g[:, 0:1, :]) / rho            # d u_i / d x_c
            gE = g[:, 4, :] - (u[None, :, :] * g[:, 1:4, :]).sum(1) + 0.5 * (u * u).sum(0) * g[:, 0, :]
            dT = (gm1 * gE - (p / rho) * g[:, 0, :]) / rho
            kR = mi.phys.mu * gam / (gm1 * mi.phys.Pr)
            tau = 4.0 * mi.phys.mu * np.abs(gu).max()
            F += max(tau, 3.0 * np.abs(u).max() * tau + kR * np.abs(dT).max())
        _, Ja, J = om.metrics(e)
        geo = sum(dn[int(N)] for N in om.orders[e]) * np.abs(Ja).max() / J.min()
        out[e], full[e] = geo * F, geo * Ff
    return out, full


def fp32_tau_ratio(tau32, tau64, S):
    """max over the valid entries (tau64 >= 0) of |tau32 - tau64| in units of
    eps32 S_dev + eps64 S_full (S = fp32_tau_scale's pair, per element)."""
    unit = np.finfo(np.float32).eps * S[0] + np.finfo(np.float64).eps * S[1]
    ok = tau64 >= 0
    return float((np.abs(tau32 - tau64) / unit[:, None])[ok].max())


def plain_rel_err(a, b, nvar_off):
    """per-variable ||a-b||_inf / ||b||_inf over a state-layout array, with no
    floor: next to rel_err it shows how much of the error budget the floor
    (the flux scale of terms that cancel) grants a small residual"""
    return rel_err(a, b, nvar_off, None)
