"""Pins of the oracle's integrator and cell-ordered re-encode."""

import math

import numpy as np

from oracle import codec, dynamics


def test_step_factors_telescope():
    # Sum of drift factors is 2 (a_0^-1/2 - a_S^-1/2); sum of kick factors
    # is the kick from a_0 to a_{S-1/2}: (3/(8 pi rho)) 2 (sqrt(a_{S-1/2}) - sqrt(a_0)).
    ai, af, S, N, nf = 0.02, 1.0, 20, 8 ** 3, 16
    a = dynamics.schedule(ai, af, S)
    np.testing.assert_allclose(np.log(a[1:] / a[:-1]), np.log(af / ai) / S, rtol=1e-12)
    kick = drift = 0.0
    for n in range(S):
        k, d = dynamics.step_factors(ai, af, S, n, N, nf)
        kick += k
        drift += d
    rho = N / nf ** 3
    np.testing.assert_allclose(drift, 2 * (ai ** -0.5 - af ** -0.5), rtol=1e-12)
    a_last_half = math.sqrt(a[S - 1] * a[S])
    np.testing.assert_allclose(kick, 3 / (8 * math.pi * rho) * 2 * (math.sqrt(a_last_half)
                                                                   - math.sqrt(ai)), rtol=1e-12)


def _lattice(n_p):
    i = np.arange(n_p)
    qz, qy, qx = np.meshgrid(i, i, i, indexing="ij")
    return (np.stack([qx.ravel(), qy.ravel(), qz.ravel()], axis=1) + 0.5) * 2.0


def test_uniform_lattice_streams_freely():
    # A uniform lattice feels no force (every particle is a centre of point
    # symmetry); with one common momentum it streams freely, and every
    # particle's integer displacement is the sum of the rounded per-step drifts.
    n_p, nc = 8, 4
    ai, af, S = 0.1, 0.6, 6
    q = _lattice(n_p)
    p0 = np.float32(0.75)
    p = np.zeros_like(q, dtype=np.float32)
    p[:, 0] = p0
    p[:, 1] = -p0 / 2
    Q0 = np.mod(np.floor(q * 64).astype(np.int64), nc * 256)
    st = dynamics.encode(Q0, p, nc, ai)
    sim = dynamics.Simulation(nc, ai, af, S)
    expect = np.zeros(3, dtype=np.int64)
    total = 0.0
    for n in range(S):
        _, d = dynamics.step_factors(ai, af, S, n, q.shape[0], 4 * nc)
        cd = np.float32(d * 64)
        for c, pc in ((0, p0), (1, np.float32(-p0 / 2))):
            expect[c] += int(np.floor(np.float32(pc * cd) + np.float32(0.5)))
        total += d
    st = sim.run(st, S)
    Q1 = st.codes()
    got = np.sort(np.mod(Q1 - expect[None, :], nc * 256), axis=0)
    np.testing.assert_array_equal(got, np.sort(Q0, axis=0))
    # and the decoded momenta are unchanged
    np.testing.assert_array_equal(st.momenta()[:, 0], np.full(q.shape[0], p0, np.float32))
    # the integer path stays within half a quantum per step of the exact drift
    assert abs(expect[0] / 64.0 - float(p0) * total) <= S / 128.0


def test_zeldovich_plane_wave_grows_linearly():
    # Einstein-de Sitter: the Zel'dovich solution x = q + a Psi(q) is exact
    # until shell crossing.  Evolve a box-scale plane wave from a = 0.05 to
    # a = 0.4 (a A 2 pi / L = 0.5 at the end).  Expected deviations: the
    # coarse-mesh CIC window at the fundamental mode (~1% of the amplitude at
    # 16 coarse cells) and the 1-byte velocity codec, which re-quantises the
    # same coherent flow each step.  A wrong force constant or time factor
    # gives >10%.
    n_p, nc, nf = 32, 16, 64
    ai, af, S = 0.05, 0.4, 16
    A = 0.5 * nf / (2 * np.pi * af)
    q = _lattice(n_p)
    psi = np.zeros_like(q)
    psi[:, 0] = A * np.sin(2 * np.pi * q[:, 0] / nf)
    Q = np.mod(np.floor((q + ai * psi) * 64).astype(np.int64), nc * 256)
    st = dynamics.encode(Q, (ai ** 1.5 * psi).astype(np.float32), nc, ai)
    st = dynamics.Simulation(nc, ai, af, S).run(st, S)
    xf = st.positions()
    qs = np.sort(q[:, 0])
    disp = np.sort(xf[:, 0]) - qs
    disp -= nf * np.round(disp / nf)
    planes = disp.reshape(n_p, -1)
    # every particle of a lattice plane moves identically (no transverse force)
    assert np.all(planes.max(axis=1) == planes.min(axis=1))
    np.testing.assert_array_equal(np.sort(st.codes()[:, 1]), np.sort(Q[:, 1]))
    qp = qs.reshape(n_p, -1)[:, 0]
    shape = np.sin(2 * np.pi * qp / nf)
    amp = planes[:, 0] @ shape / (shape @ shape)
    assert 0.98 < amp / (af * A) < 1.005
    assert np.abs(planes[:, 0] - af * A * shape).max() < 0.03 * af * A


def test_encode_invariants_and_exact_sums():
    rng = np.random.default_rng(4)
    nc = 6
    N = 3000
    Q = rng.integers(0, nc * 256, size=(N, 3))
    Q[:400] = Q[0]                         # a crowded cell
    p = (rng.normal(size=(N, 3)) * 3 + 1.0).astype(np.float32)
    st = dynamics.encode(Q, p, nc, 0.5)
    assert st.counts.sum() == N
    # decoded positions lie in their cells and equal the input multiset
    Qd = st.codes()
    cell = codec.cell_index_of_particles(st.counts)
    np.testing.assert_array_equal(codec.flatten_cell(Qd // 256, nc), cell)
    key = lambda a: np.lexsort(a.T[::-1])
    np.testing.assert_array_equal(Qd[key(Qd)], Q[key(Q)])
    # v_c against exact rational means (Python integers / fractions)
    cell_in = codec.flatten_cell(Q // 256, nc)
    P = [[int(round(float(v) * 2 ** 24)) for v in row] for row in p]
    for c in np.unique(cell_in)[:50]:
        members = np.nonzero(cell_in == c)[0]
        for d in range(3):
            S = sum(P[i][d] for i in members)
            # float32 division of the rounded sum, and within one float32
            # rounding of the exact rational mean
            ref = np.float32(np.float32(np.float32(S) * np.float32(2.0 ** -24))
                             / np.float32(len(members)))
            assert st.vc[c, d] == ref
            exact = S / len(members) * 2.0 ** -24
            assert abs(float(st.vc[c, d]) - exact) <= 2.5e-7 * abs(exact) + 1e-12
    # sigma: the variance of the fixed-point momenta about the exact cell
    # means, against exact rationals (Python Fractions), per cell and axis
    from fractions import Fraction
    ex = Fraction(0)
    floor_sum = 0
    cells = {}
    for i, c in enumerate(cell_in.tolist()):
        cells.setdefault(c, []).append(i)
    for members in cells.values():
        for d in range(3):
            vals = [P[i][d] for i in members]
            mean = Fraction(sum(vals), len(vals))
            ex += sum((Fraction(v) - mean) ** 2 for v in vals)
            floor_sum += sum(v * v for v in vals) - (sum(vals) ** 2) // len(vals)
    _, total = dynamics.dispersion(p, *dynamics.cell_means(cell_in, p, nc ** 3)[1:])
    assert total == floor_sum
    # the floor moves the sum by less than one unit per cell and axis
    assert 0 <= total - ex < 3 * len(cells)
    s2 = float(ex) * 2.0 ** -48 / (3 * N)
    assert abs(float(st.sigma) - math.sqrt(s2)) <= 1e-7 * math.sqrt(s2)
    # and sigma is close to the plain float64 dispersion about the stored means
    vcp = st.vc[cell_in]
    plain = math.sqrt(((p.astype(np.float64) - vcp) ** 2).sum() / (3 * N))
    assert abs(float(st.sigma) - plain) < 1e-6 * plain


def test_dispersion_moments_are_exact_for_large_momenta():
    # momenta near the 2^20 range limit: P^2 near 2^88, sums past 2^64 and
    # the per-cell floor(S^2/n), all against Python integers
    rng = np.random.default_rng(12)
    P = rng.integers(-(2 ** 44) + 1, 2 ** 44, size=(5000, 3))
    assert dynamics._sum_of_squares(P) == sum(int(v) * int(v) for v in P.ravel())
    p = (rng.normal(size=(2000, 3)) * 2e5).astype(np.float32)
    cell = rng.integers(0, 27, size=2000)
    vc, S, n = dynamics.cell_means(cell, p, 27)
    sig, total = dynamics.dispersion(p, S, n)
    Pf = [[int(round(float(v) * 2 ** 24)) for v in row] for row in p]
    T = sum(v * v for row in Pf for v in row)
    U = sum((int(S[c, d]) ** 2) // int(n[c]) for c in range(27) if n[c] for d in range(3))
    assert total == T - U and total > 2 ** 64
    # invariant under reordering the particles
    perm = rng.permutation(2000)
    _, S2, n2 = dynamics.cell_means(cell[perm], p[perm], 27)
    assert dynamics.dispersion(p[perm], S2, n2)[1] == total
