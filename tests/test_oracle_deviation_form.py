"""The FP32 tau sweep forms R^N(I q) from deviations q - q_r of the state from
the element's first-node state q_r, with the constant flux f(q_r) taken out
of every flux.  That changes nothing in exact arithmetic because (a) a flux
field constant over the element has zero divergence under the GL derivative
and the curl-form metrics, and (b) the interpolation reproduces constants.
These CPU tests pin (a) on the oracle at every coarse order of the isolated
sweep, on curved elements, and check the deviation-flux algebra the kernels
use against f(q) - f(q_r) computed plainly, in FP64 (equal to roundoff) and
in FP32 (rounding relative to the deviations, not to the state)."""
import numpy as np
import pytest

from paper_2210_03523_gb300 import inputs as I

GAMMA = 1.4


def _flux(q, gam=GAMMA):
    """Euler fluxes f[d][v] of conservative states q[5, n] (plain form)."""
    rho, m, E = q[0], q[1:4], q[4]
    u = m / rho
    p = (gam - 1.0) * (E - 0.5 * (m * u).sum(0))
    f = np.empty((3, 5) + rho.shape, dtype=q.dtype)
    for d in range(3):
        f[d, 0] = m[d]
        for c in range(3):
            f[d, 1 + c] = m[c] * u[d] + (p if c == d else 0.0)
        f[d, 4] = (E + p) * u[d]
    return f


def _reference(qr, gam=GAMMA):
    """The reference record of the deviation form from the first-node state
    (FP64 arithmetic, FP32 values): rho_r, u_f, m_r, c0 = m_r - u_f rho_r,
    c1 = (g-1) E_r - (g-1)/2 rho_r |u_f|^2 - p_f, h = E_r + p_f, |u_f|^2, p_f."""
    r, m, E = qr[0], qr[1:4], qr[4]
    uf = (m / r).astype(np.float32).astype(np.float64)
    u2 = float(uf @ uf)
    pf = float(np.float32((gam - 1.0) * (E - 0.5 * float(m @ m) / r)))
    return {"rho": r, "u": uf, "m": m, "c0": m - uf * r, "c1": (gam - 1.0) * E - 0.5 * (gam - 1.0) * r * u2 - pf,
            "h": E + pf, "u2": u2, "p": pf}


def _dev_flux(d, ref, dtype, gam=GAMMA):
    """Flux deviations from the deviations d = q - q_r, in the given float type."""
    t = lambda x: np.asarray(x, dtype=dtype)
    R = {k: t(v) for k, v in ref.items()}
    gm1 = t(gam - 1.0)
    d = t(d)
    rho = R["rho"] + d[0]
    ir = t(1.0) / rho
    ud = np.stack([(R["c0"][c] + d[1 + c] - R["u"][c] * d[0]) * ir for c in range(3)])
    u = np.stack([R["u"][c] + ud[c] for c in range(3)])
    pd = R["c1"] + gm1 * (d[4] - t(0.5) * d[0] * R["u2"] - rho * ((R["u"][:, None] * ud).sum(0) + t(0.5) * (ud * ud).sum(0)))
    f = np.empty((3, 5) + d.shape[1:], dtype=dtype)
    for k in range(3):
        f[k, 0] = d[1 + k]
        for c in range(3):
            f[k, 1 + c] = R["m"][c] * ud[k] + d[1 + c] * u[k] + (pd if c == k else t(0.0))
        f[k, 4] = R["h"] * ud[k] + (d[4] + pd) * u[k]
    return f


def _states(rng, n, amp):
    """n states near a Mach-0.1 free stream (p0 = 142.9), relative variations amp."""
    rho = 1.0 + amp * rng.standard_normal(n)
    u = np.array([1.0, 1.0, 0.0])[:, None] + amp * rng.standard_normal((3, n))
    p = 142.857 * (1.0 + amp * rng.standard_normal(n))
    return np.concatenate([[rho], rho * u, [p / (GAMMA - 1.0) + 0.5 * rho * (u * u).sum(0)]])


@pytest.mark.parametrize("amp", [1e-1, 1e-3, 1e-6])
def test_deviation_flux_equals_plain_difference_fp64(amp):
    q = _states(np.random.default_rng(7), 64, amp)
    ref = _reference(q[:, 0])
    fd = _dev_flux(q - q[:, :1], ref, np.float64)
    # f(q) - [the constants the deviation form drops]: m_r,d; m_r,c u_f,d + p_f; h u_f,d
    f = _flux(q)
    const = np.zeros((3, 5))
    for d in range(3):
        const[d, 0] = ref["m"][d]
        for c in range(3):
            const[d, 1 + c] = ref["m"][c] * ref["u"][d] + (ref["p"] if c == d else 0.0)
        const[d, 4] = ref["h"] * ref["u"][d]
    plain = f - const[:, :, None]
    scale = np.abs(f).max()
    assert np.abs(fd - plain).max() <= 1e-13 * scale
    # the dropped constants are f(q_r) up to the FP32 rounding of u_f and p_f:
    # at the reference node the deviation fluxes are that rounding alone
    assert np.abs(fd[:, :, 0]).max() <= 2 * np.finfo(np.float32).eps * scale


@pytest.mark.parametrize("amp", [1e-2, 1e-4])
def test_deviation_flux_fp32_rounds_relative_to_deviations(amp):
    """In FP32 the deviation form errs by a few eps32 of the flux deviations
    plus eps32 of the reference flux's rounding, while the plain FP32 flux
    errs by eps32 of the full flux (about 500 for the energy at Mach 0.1)."""
    q = _states(np.random.default_rng(8), 256, amp)
    ref = _reference(q[:, 0])
    d64 = q - q[:, :1]
    exact = _dev_flux(d64, ref, np.float64)
    got = _dev_flux(d64.astype(np.float32), ref, np.float32).astype(np.float64)
    eps = float(np.finfo(np.float32).eps)
    dev_scale = np.abs(exact).max() + np.abs(_flux(q[:, :1])).max() * eps
    assert np.abs(got - exact).max() <= 16 * eps * dev_scale
    plain32 = _flux(q.astype(np.float32)).astype(np.float64) - _flux(q[:, :1].astype(np.float32)).astype(np.float64)
    plain_err = np.abs(plain32 - (_flux(q) - _flux(q[:, :1]))).max()
    assert np.abs(got - exact).max() < plain_err / 10


def test_constant_flux_has_zero_isolated_residual_at_every_coarse_order(orc):
    """(a) on the oracle: a uniform state's isolated residual vanishes at
    every order N <= P of the sweep, on curved elements (coarse geometry
    interpolated to N) and on sheared straight ones."""
    cases = [I.box_mesh(2, geom_order=3, mapping=I.wavy_map(0.08), orders=(4, 3, 5), phys=I.pulse_physics(mach=0.3)),
             I.box_mesh(2, mapping=I.affine_map([[1.0, 0.3, 0.1], [0.0, 0.9, -0.2], [0.1, 0.0, 1.2]]),
                        orders=(3, 4, 2), phys=I.pulse_physics())]
    qc = np.array([1.1, 0.9, -0.4, 0.3, 150.0])
    for mi in cases:
        om = orc.Mesh(mi)
        flux = np.abs(_flux(qc[:, None])).max()
        for e in range(om.n_elem):
            P = om.orders[e]
            for N in I.full_sweep(P):
                n = int(np.prod(N + 1))
                R = om.isolated_residual_at(e, N, np.repeat(qc, n))
                _, Ja, J = om.metrics(e, N)
                assert np.abs(R).max() <= 1e-13 * flux * np.abs(Ja).max() / J.min(), (e, N)
