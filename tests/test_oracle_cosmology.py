"""Pins of the oracle's LambdaCDM background (Sec. IV-A.2): the
Einstein-de Sitter limit in closed form, the growing mode against a direct
integration of the linear growth equation and against published fits, and a
Zel'dovich plane wave that grows as D(a) under the oracle's integrator."""

import math

import numpy as np
from scipy import integrate

from oracle import cosmology, dynamics

# the paper's run: Omega_c = 0.214, Omega_b = 0.044, flat
OM, OL = 0.258, 0.742


def test_einstein_de_sitter_limit_is_closed_form():
    eds = cosmology.Cosmology(1.0, 0.0)
    for a_lo, a_hi in ((0.02, 0.03), (0.1, 0.5), (0.5, 1.0)):
        np.testing.assert_allclose(eds.kick_integral(a_lo, a_hi),
                                   2 * (math.sqrt(a_hi) - math.sqrt(a_lo)), rtol=1e-12)
        np.testing.assert_allclose(eds.drift_integral(a_lo, a_hi),
                                   2 * (a_lo ** -0.5 - a_hi ** -0.5), rtol=1e-12)
    for a in (0.01, 0.3, 1.0):
        np.testing.assert_allclose(eds.growth(a), a, rtol=1e-10)
        np.testing.assert_allclose(eds.growth_rate(a), 1.0, rtol=1e-10)
        np.testing.assert_allclose(eds.ic_momentum_factor(a), math.sqrt(a), rtol=1e-10)
    for n in range(10):
        a = dynamics.step_factors(0.02, 1.0, 10, n, 4096, 32)
        b = dynamics.step_factors(0.02, 1.0, 10, n, 4096, 32, eds)
        np.testing.assert_allclose(b, a, rtol=1e-12)


def _growth_ode(om, ol, a_eval):
    """D and f from the linear growth equation in ln a,
    D'' + (2 + dlnE/dlna) D' - (3/2) Omega_m / (a^3 E^2) D = 0,
    started on the growing mode D = a deep in matter domination."""
    ok = 1.0 - om - ol

    def rhs(x, y):
        a = math.exp(x)
        e2 = om / a ** 3 + ok / a ** 2 + ol
        dlne = (-3 * om / a ** 3 - 2 * ok / a ** 2) / (2 * e2)
        return [y[1], -(2 + dlne) * y[1] + 1.5 * om / (a ** 3 * e2) * y[0]]

    a0 = 1e-10     # curvature shifts D from a by O(a Omega_k / Omega_m) at the start
    sol = integrate.solve_ivp(rhs, (math.log(a0), math.log(max(a_eval))), [a0, a0],
                              t_eval=np.log(a_eval), rtol=1e-12, atol=1e-20, method="DOP853")
    return sol.y[0], sol.y[1] / sol.y[0]


def test_growth_matches_the_linear_growth_equation():
    a_eval = np.array([0.01, 0.1, 0.5, 1.0])
    for om, ol in ((OM, OL), (0.3, 0.7), (0.3, 0.0)):
        c = cosmology.Cosmology(om, ol)
        D, f = _growth_ode(om, ol, a_eval)
        np.testing.assert_allclose([c.growth(a) for a in a_eval], D, rtol=1e-7)
        np.testing.assert_allclose([c.growth_rate(a) for a in a_eval], f, rtol=1e-7)


def test_growth_against_published_fits():
    c = cosmology.Cosmology(OM, OL)
    # Carroll, Press & Turner (1992): g = D(1) / a within about 1%
    g = 2.5 * OM / (OM ** (4 / 7) - OL + (1 + OM / 2) * (1 + OL / 70))
    assert abs(c.growth(1.0) / g - 1) < 0.01
    # Linder (2005): f = Omega_m(a)^0.55 within about 1% for flat LambdaCDM
    for a in (0.2, 0.5, 1.0):
        om_a = OM / a ** 3 / c.E(a) ** 2
        assert abs(c.growth_rate(a) / om_a ** 0.55 - 1) < 0.01
    # matter domination at z = 99: D = a and f = 1 to 1e-5
    assert abs(c.growth(0.01) / 0.01 - 1) < 1e-5 and abs(c.growth_rate(0.01) - 1) < 1e-5


def test_lcdm_factors_are_the_integrals():
    # kick and drift factors of a step against a plain midpoint sum of the
    # integrands (an independent quadrature), and the Omega_m in the kick
    c = cosmology.Cosmology(OM, OL)
    ai, af, S, N, nf = 0.01, 1.0, 12, 4096, 32
    a = dynamics.schedule(ai, af, S)
    rho = N / nf ** 3
    for n in (0, 5, 11):
        k, d = dynamics.step_factors(ai, af, S, n, N, nf, c)
        a_lo = a[0] if n == 0 else math.sqrt(a[n - 1] * a[n])
        a_hi = math.sqrt(a[n] * a[n + 1])
        m = 200000
        x = a_lo + (np.arange(m) + 0.5) * (a_hi - a_lo) / m
        e = np.sqrt(OM / x ** 3 + OL)
        kref = 3 * OM / (8 * math.pi * rho) * ((a_hi - a_lo) / m) * (1 / (x * x * e)).sum()
        x = a[n] + (np.arange(m) + 0.5) * (a[n + 1] - a[n]) / m
        e = np.sqrt(OM / x ** 3 + OL)
        dref = ((a[n + 1] - a[n]) / m) * (1 / (x ** 3 * e)).sum()
        np.testing.assert_allclose(k, kref, rtol=1e-8)
        np.testing.assert_allclose(d, dref, rtol=1e-8)


def _lattice(n_p, spacing):
    i = np.arange(n_p)
    qz, qy, qx = np.meshgrid(i, i, i, indexing="ij")
    return (np.stack([qx.ravel(), qy.ravel(), qz.ravel()], axis=1) + 0.5) * spacing


def test_lcdm_plane_wave_grows_as_the_growth_factor():
    # a planar Zel'dovich wave is exact in any Friedmann background until
    # shell crossing: x = q + D(a) Psi.  From a = 0.05 to 0.8 in LambdaCDM the
    # amplitude must grow by D(0.8) / D(0.05) (about 0.78 of the EdS factor);
    # a missing Omega_m in the kick or an EdS time factor misses by >10%.
    n_p, nc, nf = 32, 16, 64
    ai, af, S = 0.05, 0.8, 24
    c = cosmology.Cosmology(OM, OL)
    Df = c.growth(af)
    A = 0.5 * nf / (2 * np.pi * Df)                    # D A 2 pi / L = 0.5 at the end
    q = _lattice(n_p, 2.0)
    disp = np.zeros_like(q)
    disp[:, 0] = c.growth(ai) * A * np.sin(2 * np.pi * q[:, 0] / nf)
    Q = np.mod(np.floor((q + disp) * 64).astype(np.int64), nc * 256)
    p = (c.ic_momentum_factor(ai) * disp).astype(np.float32)
    st = dynamics.encode(Q, p, nc, ai)
    st = dynamics.Simulation(nc, ai, af, S, cosmo=c).run(st, S)
    xf = st.positions()
    qs = np.sort(q[:, 0])
    d = np.sort(xf[:, 0]) - qs
    d -= nf * np.round(d / nf)
    planes = d.reshape(n_p, -1)
    assert np.all(planes.max(axis=1) == planes.min(axis=1))
    qp = qs.reshape(n_p, -1)[:, 0]
    shape = np.sin(2 * np.pi * qp / nf)
    amp = planes[:, 0] @ shape / (shape @ shape)
    assert 0.98 < amp / (Df * A) < 1.01, amp / (Df * A)
    # per plane: mesh smoothing and the 1-byte velocity codec, re-quantised
    # over 24 steps
    assert np.abs(planes[:, 0] - Df * A * shape).max() < 0.04 * Df * A
