"""Pins of the oracle's truncation-error extrapolation to N_i >= P_i
(Sec. 2.3 and Sec. 2.4: approach 2 needs the extrapolated map; a direction
that cannot be extrapolated gets a high value).  Exponential decay must be
recovered exactly, the fit must be the least-squares line of ln tau, and
the special cases (no decay, too few points, exact zero) must give the
stated values."""
import numpy as np
import pytest

from paper_2210_03523_gb300 import inputs as I


def _grid(nmax):
    return np.array([(a, b, c) for c in range(1, nmax + 1) for b in range(1, nmax + 1) for a in range(1, nmax + 1)],
                    dtype=np.int32)


def _element_map(P, sweep, inner, directional):
    """One element's map over sweep: directional(i, n) on entries that differ
    from P in direction i only, inner(N) on the other entries N <= P, -1 above
    P and 0 at P (tau^P = 0)."""
    row = np.empty(len(sweep))
    for s, N in enumerate(sweep):
        diff = [i for i in range(3) if N[i] != P[i]]
        if any(N[i] > P[i] for i in range(3)):
            row[s] = -1.0
        elif not diff:
            row[s] = 0.0
        elif len(diff) == 1:
            row[s] = directional(diff[0], N[diff[0]])
        else:
            row[s] = inner(tuple(N))
    return row[None, :]


C = np.array([3.0, 0.7, 11.0])
R = np.array([0.3, 0.55, 0.12])


def _exp(i, n):
    return C[i] * R[i] ** n


@pytest.mark.parametrize("P", [(4, 5, 3), (3, 3, 3), (6, 4, 5)])
def test_exponential_decay_is_extrapolated_exactly(orc, P):
    sweep = I.full_sweep(P)
    inner = lambda N: 1e3 + N[0] + 10 * N[1] + 100 * N[2]       # arbitrary, only copied through
    mp = _element_map(P, sweep, inner, _exp)
    tg = _grid(8)
    out = orc.tau_extrapolate(mp, [P], sweep, tg)[0]
    for t, N in enumerate(tg):
        Nc = tuple(min(N[i], P[i]) for i in range(3))
        diff = [i for i in range(3) if Nc[i] != P[i]]
        base = 0.0 if not diff else (_exp(diff[0], Nc[diff[0]]) if len(diff) == 1 else inner(Nc))
        want = base + sum(_exp(i, N[i]) for i in range(3) if N[i] >= P[i])
        assert out[t] == pytest.approx(want, rel=1e-13), (N, out[t], want)


def test_decoupled_map_is_the_sum_of_directional_parts(orc):
    P = (5, 4, 3)
    sweep = np.array([(n if i == 0 else P[0], n if i == 1 else P[1], n if i == 2 else P[2])
                      for i in range(3) for n in range(1, P[i])], dtype=np.int32)   # sum_i (P_i - 1) entries
    mp = np.array([[_exp(int(np.argmax(np.array(N) != np.array(P))), N[np.argmax(np.array(N) != np.array(P))])
                    for N in sweep]])
    tg = _grid(7)
    out = orc.tau_extrapolate(mp, [P], sweep, tg, decoupled=True)[0]
    for t, N in enumerate(tg):
        assert out[t] == pytest.approx(sum(_exp(i, N[i]) for i in range(3)), rel=1e-13)
    # the coupled reading cannot use the directional sweep for inner entries
    out_c = orc.tau_extrapolate(mp, [P], sweep, np.array([[1, 1, 3]], np.int32))[0]
    assert out_c[0] == -1.0


def test_fit_is_least_squares_of_log_tau(orc):
    rng = np.random.default_rng(4)
    P = (7, 7, 7)
    sweep = I.full_sweep(P)
    noise = {(i, n): np.exp(0.2 * rng.standard_normal()) for i in range(3) for n in range(1, 7)}
    d = lambda i, n: _exp(i, n) * noise[(i, n)]
    mp = _element_map(P, sweep, lambda N: 1.0, d)
    tg = np.array([[8, 7, 7], [7, 8, 7], [7, 7, 8]], np.int32)
    for n_fit in (0, 3, 2):
        ns = np.arange(1 if n_fit == 0 else 7 - n_fit, 7)
        fit = [np.polyfit(ns, np.log([d(i, n) for n in ns]), 1) for i in range(3)]    # (slope, intercept)
        e = lambda i, n: np.exp(fit[i][1] + fit[i][0] * n)
        out = orc.tau_extrapolate(mp, [P], sweep, tg, n_fit=n_fit)[0]
        for i in range(3):
            # target i: direction i at 8, the others at P = 7 (their e_j(7) adds in)
            want = e(i, 8) + sum(e(j, 7) for j in range(3) if j != i)
            assert out[i] == pytest.approx(want, rel=1e-12)


def test_special_cases(orc):
    P = (4, 2, 3)
    sweep = I.full_sweep(P)
    # xi1 grows with n: not in the asymptotic range -> infinity; xi2 has a
    # single point -> infinity; xi3 decays
    mp = _element_map(P, sweep, lambda N: 0.5, lambda i, n: 0.1 * 2.0 ** n if i == 0 else _exp(i, n))
    tg = np.array([[4, 1, 1], [3, 2, 1], [3, 1, 1], [3, 1, 4], [5, 2, 1]], np.int32)
    out = orc.tau_extrapolate(mp, [P], sweep, tg)[0]
    assert np.isinf(out[0]) and np.isinf(out[1]) and np.isinf(out[4])
    assert out[2] == 0.5                      # inner entry, copied through
    assert out[3] == pytest.approx(0.5 + _exp(2, 4), rel=1e-13)
    # P_i = 1: no point below P, every N_i >= 1 gets the high value
    P = (3, 3, 1)
    sweep = I.full_sweep(P)
    mp = _element_map(P, sweep, lambda N: 0.5, _exp)
    assert np.all(np.isinf(orc.tau_extrapolate(mp, [P], sweep, _grid(4))))
    # an exact zero just below P: the direction is resolved, e = 0
    P = (3, 3, 3)
    sweep = I.full_sweep(P)
    mp = _element_map(P, sweep, lambda N: 0.25, lambda i, n: 0.0 if i == 0 else _exp(i, n))
    out = orc.tau_extrapolate(mp, [P], sweep, np.array([[6, 2, 2], [3, 3, 3]], np.int32))[0]
    assert out[0] == 0.25
    assert out[1] == pytest.approx(_exp(1, 3) + _exp(2, 3), rel=1e-13)
    # a floor: values at or below it count as resolved, the others still decay
    mp = _element_map(P, sweep, lambda N: 0.25, lambda i, n: 1e-13 * (n + 1) if i == 0 else _exp(i, n))
    out = orc.tau_extrapolate(mp, [P], sweep, np.array([[4, 3, 3]], np.int32), tau_floor=1e-12)[0]
    assert out[0] == pytest.approx(_exp(1, 3) + _exp(2, 3), rel=1e-13)
    assert np.isinf(orc.tau_extrapolate(mp, [P], sweep, np.array([[4, 3, 3]], np.int32))[0, 0])
    # entries missing from the sweep give -1
    keep = sweep[:, 0] != 1
    out = orc.tau_extrapolate(mp[:, keep], [P], sweep[keep], np.array([[1, 2, 2]], np.int32))[0]
    assert out[0] == -1.0


def test_accumulate_is_fmax(orc):
    P = (4, 4, 4)
    sweep = I.full_sweep(P)
    tg = _grid(6)
    m1 = _element_map(P, sweep, lambda N: 0.2, _exp)
    m2 = _element_map(P, sweep, lambda N: 0.3, lambda i, n: 0.5 * _exp(i, n) if i else 2 * _exp(i, n))
    acc = orc.tau_extrapolate(m1, [P], sweep, tg)
    orc.tau_extrapolate(m2, [P], sweep, tg, accumulate=acc)
    np.testing.assert_array_equal(acc, np.maximum(orc.tau_extrapolate(m1, [P], sweep, tg),
                                                  orc.tau_extrapolate(m2, [P], sweep, tg)))


@pytest.mark.slow
def test_extrapolation_tracks_a_finer_reference(orc):
    """On a smooth state, the map extrapolated from P = 4 must agree in order
    of magnitude with the map estimated directly from the finer reference
    P = 6 (directional entries N_i = 5 in the two directions the flow
    crosses; the velocity has no xi3 part): the method's premise that tau decays
    exponentially (Sec. 1, Sec. 2.3)."""
    ph = I.pulse_physics(mach=0.5)
    mi4 = I.box_mesh(2, orders=(4, 4, 4), phys=ph)
    mi6 = mi4.with_orders(np.full((mi4.n_elem, 3), 6, np.int32))
    maps = []
    for mi in (mi4, mi6):
        m = orc.Mesh(mi)
        q = I.pulse_state(m.coords(), mi.orders, ph, width=0.6)
        P = tuple(int(v) for v in mi.orders[0])
        maps.append((m.tau(q, I.full_sweep(P))[0], I.full_sweep(P)))
    (t4, s4), (t6, s6) = maps
    tg = np.array([[5, 6, 6], [6, 5, 6]], np.int32)
    # xi3 carries no flux (w = 0): its estimates sit at roundoff, below the floor
    ext = orc.tau_extrapolate(t4, mi4.orders, s4, tg, tau_floor=1e-10)
    direct = t6[:, [int(np.flatnonzero((s6 == N).all(1))[0]) for N in tg]]
    ratio = ext / direct
    assert np.all(np.isfinite(ratio)) and np.all((ratio > 0.1) & (ratio < 10.0)), ratio
