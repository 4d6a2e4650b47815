"""Pins of the oracle's Zel'dovich initial conditions and power spectrum."""

import os

import numpy as np

from oracle import cic, codec, ic, power


def _splitmix64_bigint(seed, j):
    # the published SplitMix64 output function, in Python integers mod 2^64
    M = (1 << 64) - 1
    z = (seed + (j + 1) * 0x9E3779B97F4A7C15) & M
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
    return z ^ (z >> 31)


def test_splitmix64_vectorised_matches_integer_arithmetic():
    for seed in (0, 1, 12345, (1 << 64) - 1):
        j = np.array([0, 1, 2, 3, 1000, 123456789, (1 << 40) + 7], dtype=np.uint64)
        got = ic.splitmix64(seed, j)
        for a, b in zip(got, j):
            assert int(a) == _splitmix64_bigint(seed, int(b))


def test_splitmix64_published_outputs():
    """The generator's own published outputs from state 0 pin its increment
    and mixing constants (a mistyped constant in both the vectorised and the
    integer form would pass the test above)."""
    path = os.path.join(os.path.dirname(__file__), "golden", "splitmix64_vectors.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 3
    for seed, j, out in rows:
        got = ic.splitmix64(int(seed), np.array([int(j)], dtype=np.uint64))[0]
        assert int(got) == int(out, 16)


def test_white_noise_is_unit_gaussian():
    w = ic.white_noise(7, 32).ravel()
    n = w.size
    assert abs(w.mean()) < 5 / np.sqrt(n)
    assert abs(w.var() - 1) < 5 * np.sqrt(2.0 / n)
    # fourth moment of a Gaussian is 3
    assert abs((w ** 4).mean() - 3) < 0.15


def test_displacement_is_potential_flow_of_the_field():
    # delta = -div Psi must reproduce the filtered input field: compare
    # spectrally on modes off the Nyquist planes
    n_p, nf, slope, kc = 16, 32, -1.5, np.pi / 2
    psi = ic.displacement(3, n_p, nf, slope, kc)
    n = ic.lattice_frequencies(n_p)
    nz_, ny_, nx_ = np.meshgrid(n, n, n, indexing="ij")
    k = [2 * np.pi * m / nf for m in (nx_, ny_, nz_)]
    div_hat = sum(1j * k[d] * np.fft.fftn(psi[d]) for d in range(3))
    w_hat = np.fft.fftn(ic.white_noise(3, n_p))
    kk = np.sqrt(k[0] ** 2 + k[1] ** 2 + k[2] ** 2)
    delta_hat = w_hat * np.sqrt(ic.power_law(kk, slope, kc))
    nyq = -(n_p // 2)
    ok = (kk > 0) & (nx_ != nyq) & (ny_ != nyq) & (nz_ != nyq)
    np.testing.assert_allclose(-div_hat[ok], delta_hat[ok], rtol=1e-10,
                               atol=1e-12 * np.abs(delta_hat).max())
    # the displacement is curl-free: k x Psi~ = 0
    ph = [np.fft.fftn(psi[d]) for d in range(3)]
    curl = k[1] * ph[2] - k[2] * ph[1]
    assert np.abs(curl).max() < 1e-10 * np.abs(ph[0]).max()


def test_zeldovich_normalisation_and_growing_mode():
    n_p, nc, ai = 16, 8, 0.02
    st, x, p = ic.zeldovich(11, n_p, nc, ai, rms_disp=0.3)
    i = np.arange(n_p)
    qz, qy, qx = np.meshgrid(i, i, i, indexing="ij")
    q = (np.stack([qx.ravel(), qy.ravel(), qz.ravel()], 1) + 0.5) * (4 * nc / n_p)
    disp = x - q
    rms = np.sqrt((disp ** 2).sum(1).mean())
    assert abs(rms - 0.3) < 1e-12
    np.testing.assert_allclose(p, disp * np.sqrt(ai), rtol=0, atol=1e-14)  # p = a^(3/2) Psi
    # the stored state decodes to the ICs within half a quantum
    Qx = np.mod(np.floor(x * 64).astype(np.int64), nc * 256)
    key = lambda a: np.lexsort(a.T[::-1])
    Qd = st.codes()
    np.testing.assert_array_equal(Qd[key(Qd)], Qx[key(Qx)])


def test_shell_binning_brute_force():
    rng = np.random.default_rng(0)
    n = 8
    L = 20.0
    delta = rng.normal(size=(n, n, n))
    k, P, cnt = power.spectrum_from_delta(delta, L, n // 2)
    dk = np.fft.fftn(delta)
    sums = np.zeros(n // 2 + 1)
    ks = np.zeros(n // 2 + 1)
    cs = np.zeros(n // 2 + 1, dtype=int)
    for a in range(n):
        for b in range(n):
            for c in range(n):
                f = [m if m < n // 2 else m - n for m in (a, b, c)]
                r = np.sqrt(f[0] ** 2 + f[1] ** 2 + f[2] ** 2)
                j = int(np.floor(r + 0.5))
                if 1 <= j <= n // 2:
                    sums[j] += abs(dk[a, b, c]) ** 2 * L ** 3 / n ** 6
                    ks[j] += 2 * np.pi * r / L
                    cs[j] += 1
    np.testing.assert_array_equal(cnt, cs[1:])
    np.testing.assert_allclose(P, sums[1:] / cs[1:], rtol=1e-12)
    np.testing.assert_allclose(k, ks[1:] / cs[1:], rtol=1e-12)


def test_parseval_normalisation():
    rng = np.random.default_rng(1)
    n, L = 16, 50.0
    delta = rng.normal(size=(n, n, n))
    dk = np.fft.fftn(delta)
    P = (L ** 3 / n ** 6) * np.abs(dk) ** 2
    # sum over modes of P / L^3 is the variance of delta (Parseval)
    np.testing.assert_allclose(P.sum() / L ** 3, (delta ** 2).mean(), rtol=1e-12)


def test_poisson_particles_give_shot_noise():
    # uniform random particles: CIC shot noise (Jing 2005, ApJ 620, 559)
    # P(k) = (L^3 / N) prod_d [1 - (2/3) sin^2(pi n_d / nmesh)], shell-averaged
    rng = np.random.default_rng(2)
    nc, N = 16, 400000
    nf = 4 * nc
    nmesh = nf // 2
    Q = rng.integers(0, nc * 256, size=(N, 3))
    nb = 8
    k, P, cnt = power.power_spectrum(Q, nmesh, nb, nf)
    n = np.rint(np.fft.fftfreq(nmesh) * nmesh)
    nz_, ny_, nx_ = np.meshgrid(n, n, n, indexing="ij")
    win = np.ones_like(nx_)
    for m in (nx_, ny_, nz_):
        win = win * (1 - 2.0 / 3.0 * np.sin(np.pi * m / nmesh) ** 2)
    j = np.rint(np.sqrt(nx_ ** 2 + ny_ ** 2 + nz_ ** 2)).astype(int)
    expect = np.array([win[j == s].mean() for s in range(1, nb + 1)]) * nf ** 3 / N
    ratio = P / expect
    assert np.all(np.abs(ratio - 1) < 4 * np.sqrt(1.0 / cnt) + 0.02)
    assert abs(np.average(ratio, weights=cnt) - 1) < 0.03


def test_initial_spectrum_follows_the_input_shape():
    # the ZA density of the ICs follows the input P(k) at low k up to a
    # common factor (scatter ~ sqrt(2 / N_modes) per shell)
    n_p, nc, ai = 64, 32, 0.02
    nf = 4 * nc
    st, x, p = ic.zeldovich(5, n_p, nc, ai, slope=-1.5, rms_disp=0.3)
    Q = st.codes()
    k, P, cnt = power.power_spectrum(Q, nf // 2, 8, nf)
    Pin = ic.power_law(k, -1.5, np.pi / 2)
    r = (P / Pin)[:6]
    c = cnt[:6]
    ref = np.average(r, weights=c)
    assert np.all(np.abs(r / ref - 1) < 4 * np.sqrt(2.0 / c) + 0.05)
