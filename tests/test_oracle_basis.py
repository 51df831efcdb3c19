"""Pins of the oracle's 1D basis (Sec. 2.1: tensor Lagrange basis on the
N+1 Gauss-Lobatto nodes) against closed forms, numpy's Legendre routines and
exactness properties."""
import math
import os

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

GOLD = os.path.join(os.path.dirname(__file__), "golden", "gl_closed_forms.txt")


def _golden():
    rows = []
    env = {"sqrt": math.sqrt}
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        n, xs, ws = line.split("|")
        rows.append((int(n), [eval(t, env) for t in xs.split(",")], [eval(t, env) for t in ws.split(",")]))
    return rows


@pytest.mark.parametrize("row", _golden(), ids=lambda r: f"N{r[0]}")
def test_gl_closed_forms(orc, row):
    N, xs, ws = row
    x, w = orc.gl(N)
    np.testing.assert_allclose(x, xs, rtol=0, atol=2e-16)
    np.testing.assert_allclose(w, ws, rtol=4e-16)


@pytest.mark.parametrize("N", range(1, 13))
def test_gl_nodes_are_lobatto_points(orc, N):
    x, w = orc.gl(N)
    # interior nodes = roots of L_N' (numpy's Legendre series)
    c = np.zeros(N + 1)
    c[N] = 1.0
    ref = np.sort(np.real(npleg.legroots(npleg.legder(c)))) if N > 1 else np.array([])
    np.testing.assert_allclose(x[1:-1], ref, atol=1e-14)
    assert x[0] == -1.0 and x[-1] == 1.0
    # quadrature exact for degree <= 2N-1
    for k in range(2 * N):
        exact = 2.0 / (k + 1) if k % 2 == 0 else 0.0
        assert abs(np.dot(w, x ** k) - exact) < 2e-15
    # and not for degree 2N (GL is exact only up to 2N-1)
    assert abs(np.dot(w, x ** (2 * N)) - 2.0 / (2 * N + 1)) > 1e-9


@pytest.mark.parametrize("N", range(1, 11))
def test_derivative_matrix(orc, N):
    x, w = orc.gl(N)
    D = orc.dmat(N)
    for k in range(N + 1):
        d = k * x ** (k - 1) if k > 0 else np.zeros_like(x)
        np.testing.assert_allclose(D @ x ** k, d, atol=5e-13 * max(1, N * N))
    np.testing.assert_allclose(D.sum(axis=1), 0.0, atol=1e-13 * N * N)
    # summation-by-parts: W D + D^T W = diag(-1, 0, ..., 0, 1)
    B = np.diag(w) @ D + D.T @ np.diag(w)
    E = np.zeros_like(B)
    E[0, 0], E[-1, -1] = -1.0, 1.0
    np.testing.assert_allclose(B, E, atol=1e-13)


@pytest.mark.parametrize("Nf,Nt", [(4, 2), (6, 1), (8, 5), (3, 3), (2, 7)])
def test_interpolation(orc, Nf, Nt):
    xf, _ = orc.gl(Nf)
    xt, _ = orc.gl(Nt)
    I = orc.interp_mat(Nf, Nt)
    for k in range(min(Nf, Nt) + 1):
        np.testing.assert_allclose(I @ xf ** k, xt ** k, atol=1e-14)
    if Nt < Nf:
        np.testing.assert_allclose(I @ orc.interp_mat(Nt, Nf), np.eye(Nt + 1), atol=1e-14)
    if Nt == Nf:
        assert np.array_equal(I, np.eye(Nt + 1))      # exact identity: tau^P is exactly zero


@pytest.mark.parametrize("Nf,Nt", [(5, 2), (6, 1), (8, 7), (3, 3)])
def test_projection(orc, Nf, Nt):
    xf, wf = orc.gl(Nf)
    xt, wt = orc.gl(Nt)
    Pm = orc.proj_mat(Nf, Nt)
    for k in range(Nt + 1):
        np.testing.assert_allclose(Pm @ xf ** k, xt ** k, atol=1e-13)
    rng = np.random.default_rng(0)
    f = rng.standard_normal(Nf + 1)
    assert abs(wt @ (Pm @ f) - wf @ f) < 1e-14          # discrete conservation
    if Nf == Nt:
        assert np.array_equal(Pm, np.eye(Nt + 1))
        return
    # Galerkin orthogonality of the residual f - Pi f against every degree-Nt
    # Lagrange polynomial, integrated with numpy's 30-point Gauss-Legendre rule
    xq, wq = npleg.leggauss(30)

    def lag(nodes, vals, t):
        out = np.zeros_like(t)
        for j in range(len(nodes)):
            lj = np.ones_like(t)
            for m in range(len(nodes)):
                if m != j:
                    lj *= (t - nodes[m]) / (nodes[j] - nodes[m])
            out += vals[j] * lj
        return out
    err = lag(xf, f, xq) - lag(xt, Pm @ f, xq)
    for j in range(Nt + 1):
        e = np.zeros(Nt + 1)
        e[j] = 1.0
        assert abs(np.dot(wq, err * lag(xt, e, xq))) < 1e-14
