"""Pins of the oracle's fluxes (Sec. 3: Roe advective flux, BR1 viscous
flux; Sec. 2.1 first-order form) against properties the mathematics fixes."""
import numpy as np
import pytest

G = 1.4


def cons(rho, u, p, gamma=G):
    u = np.asarray(u, dtype=float)
    return np.array([rho, *(rho * u), p / (gamma - 1) + 0.5 * rho * u @ u])


def nflux(orc, q, n):
    return sum(orc.euler_flux(G, q, d) * n[d] for d in range(3))


def rand_states(rng, k):
    for _ in range(k):
        n = rng.standard_normal(3)
        n /= np.linalg.norm(n)
        qL = cons(rng.uniform(0.5, 2), rng.uniform(-1, 1, 3), rng.uniform(0.5, 2))
        qR = cons(rng.uniform(0.5, 2), rng.uniform(-1, 1, 3), rng.uniform(0.5, 2))
        yield qL, qR, n


def test_euler_flux_jacobian_eigenvalues(orc):
    """Eigenvalues of d(f.n)/dq (central differences) are u.n - c, u.n (x3),
    u.n + c with c^2 = gamma p / rho: fixes pressure law and flux layout."""
    rng = np.random.default_rng(1)
    for _ in range(5):
        rho, u, p = rng.uniform(0.5, 2), rng.uniform(-1, 1, 3), rng.uniform(0.5, 2)
        n = rng.standard_normal(3)
        n /= np.linalg.norm(n)
        q = cons(rho, u, p)
        A = np.empty((5, 5))
        for j in range(5):
            h = 1e-6 * max(1.0, abs(q[j]))
            dq = np.zeros(5)
            dq[j] = h
            A[:, j] = (nflux(orc, q + dq, n) - nflux(orc, q - dq, n)) / (2 * h)
        ev = np.sort(np.real(np.linalg.eigvals(A)))
        un, c = u @ n, np.sqrt(G * p / rho)
        np.testing.assert_allclose(ev, np.sort([un - c, un, un, un, un + c]), atol=1e-6)
        # Euler flux is homogeneous of degree one: f(q) = A(q) q
        np.testing.assert_allclose(A @ q, nflux(orc, q, n), rtol=1e-6, atol=1e-7)


def test_roe_consistency(orc):
    rng = np.random.default_rng(2)
    for qL, qR, n in rand_states(rng, 20):
        np.testing.assert_allclose(orc.roe(G, qL, qL, n), nflux(orc, qL, n), rtol=1e-14, atol=1e-14)


def test_roe_conservation_symmetry(orc):
    rng = np.random.default_rng(3)
    for qL, qR, n in rand_states(rng, 20):
        np.testing.assert_allclose(orc.roe(G, qL, qR, n), -orc.roe(G, qR, qL, -n), rtol=1e-13, atol=1e-14)


def test_roe_supersonic_upwinding(orc):
    """All wave speeds positive: Roe reduces to f(qL).n exactly (its linearisation
    satisfies f(qR) - f(qL) = A~ (qR - qL)); all negative: f(qR).n."""
    rng = np.random.default_rng(4)
    for s in (+1, -1):
        for _ in range(10):
            n = rng.standard_normal(3)
            n /= np.linalg.norm(n)
            uL = s * 3.0 * n + 0.3 * rng.standard_normal(3)
            uR = s * 3.2 * n + 0.3 * rng.standard_normal(3)
            qL = cons(rng.uniform(0.8, 1.2), uL, rng.uniform(0.3, 0.5))
            qR = cons(rng.uniform(0.8, 1.2), uR, rng.uniform(0.3, 0.5))
            ref = nflux(orc, qL if s > 0 else qR, n)
            np.testing.assert_allclose(orc.roe(G, qL, qR, n), ref, rtol=1e-12, atol=1e-12)


def test_roe_rotation_invariance(orc):
    rng = np.random.default_rng(5)
    for qL, qR, n in rand_states(rng, 10):
        Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
        rot = lambda q: np.array([q[0], *(Q @ q[1:4]), q[4]])
        f = orc.roe(G, qL, qR, n)
        np.testing.assert_allclose(orc.roe(G, rot(qL), rot(qR), Q @ n), rot(f), rtol=1e-12, atol=1e-13)


def test_roe_contact_wave_reduction(orc):
    """Equal velocity and pressure on both sides: only the entropy wave
    carries a jump, and Roe is the upwind flux of the advected density
    (the density-pulse family of Sec. 3.1)."""
    rng = np.random.default_rng(6)
    for _ in range(10):
        u = rng.uniform(-1, 1, 3)
        p = rng.uniform(0.5, 2)
        n = rng.standard_normal(3)
        n /= np.linalg.norm(n)
        rL, rR = rng.uniform(0.5, 2, 2)
        qL, qR = cons(rL, u, p), cons(rR, u, p)
        un = u @ n
        rho_up = rL if un > 0 else rR
        f = orc.roe(G, qL, qR, n)
        expect = nflux(orc, cons(rho_up, u, p), n)
        np.testing.assert_allclose(f, expect, rtol=1e-13, atol=1e-13)


def _visc_fd(orc, phys, prim, x0, d):
    """viscous flux at x0 for primitive fields prim(x) -> (rho, u[3], p),
    conservative gradient by central differences"""
    def q_at(x):
        rho, u, p = prim(x)
        return cons(rho, u, p, phys.gamma)
    gq = np.empty((5, 3))
    for c in range(3):
        dx = np.zeros(3)
        dx[c] = 1e-5
        gq[:, c] = (q_at(x0 + dx) - q_at(x0 - dx)) / 2e-5
    return orc.visc_flux(phys, q_at(x0), gq, d)


def test_viscous_flux_invariants(orc):
    from paper_2210_03523_gb300.inputs import Physics
    ph = Physics(1, 1.4, 0.3, 0.72, 2.0)
    x0 = np.array([0.3, -0.2, 0.5])
    w = np.array([0.4, -1.1, 0.7])
    # rigid rotation, uniform temperature: no stress, no heat flux
    rot = lambda x: (1.3, np.cross(w, x), 1.3 * 2.0 * 1.7)
    for d in range(3):
        np.testing.assert_allclose(_visc_fd(orc, ph, rot, x0, d), 0.0, atol=1e-8)
    # uniform dilatation u = a x: the deviatoric stress vanishes
    dil = lambda x: (1.1, 0.8 * x, 1.1 * 2.0 * 1.3)
    for d in range(3):
        np.testing.assert_allclose(_visc_fd(orc, ph, dil, x0, d)[:4], 0.0, atol=1e-8)
    # simple shear u = (a y, 0, 0) at constant T: tau_xy = mu a, energy flux u tau
    a = 0.9
    shear = lambda x: (1.2, np.array([a * x[1], 0.0, 0.0]), 1.2 * 2.0 * 1.5)
    f = _visc_fd(orc, ph, shear, x0, 1)
    np.testing.assert_allclose(f, [0, ph.mu * a, 0, 0, a * x0[1] * ph.mu * a], atol=1e-8)
    # pure conduction: T = T0 + b.x at rest with constant pressure
    b = np.array([0.2, -0.3, 0.1])
    p0 = 3.0
    cond = lambda x: (p0 / (ph.Rgas * (1.5 + b @ x)), np.zeros(3), p0)
    kappa = ph.mu * ph.gamma * ph.Rgas / ((ph.gamma - 1) * ph.Pr)
    for d in range(3):
        np.testing.assert_allclose(_visc_fd(orc, ph, cond, x0, d), [0, 0, 0, 0, kappa * b[d]], atol=1e-8)
