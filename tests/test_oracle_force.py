"""Pins of the oracle's force kernels and PM-PM force (Sec. II, Eq. 1)."""

import numpy as np
import pytest

from oracle import cic, codec, direct, force, kernels


def _cic_1d(pos, h, n):
    """Textbook CIC of a float position (fine units) on nodes at (i+1/2) h."""
    t = pos / h - 0.5
    i0 = int(np.floor(t))
    w1 = t - i0
    return [(i0 % n, 1.0 - w1), ((i0 + 1) % n, w1)]


def _cic_3d(x, h, n):
    out = []
    for iz, wz in _cic_1d(x[2], h, n):
        for iy, wy in _cic_1d(x[1], h, n):
            for ix, wx in _cic_1d(x[0], h, n):
                out.append(((iz, iy, ix), wx * wy * wz))
    return out


def test_coarse_kernel_is_odd():
    K = kernels.coarse_kernel_table(8)
    flip = K[:, (-np.arange(8)) % 8][:, :, (-np.arange(8)) % 8][:, :, :, (-np.arange(8)) % 8]
    np.testing.assert_array_equal(flip, -K)
    assert np.all(K[:, 0, 0, 0] == 0)


def test_periodic_pair_force_closed_forms():
    # Near the origin the periodic force of a unit mass with its images and
    # the removed mean is -x/|x|^3 + (4 pi / 3) x / L^3 (uniform negative
    # background; the cubic image lattice adds no linear term), up to
    # O(|x|^3 / L^5).  By symmetry it vanishes at the half-box points.
    x = np.array([[1.0, 0.3, -0.2], [0.5, 1.5, 0.1], [-2.0, 0.7, 1.1]])
    for L in (32.0, 64.0, 256.0):
        F = kernels.periodic_pair_kernel(x, L)
        approx = kernels.pair_kernel(x) + 4 * np.pi / 3 * x / L ** 3
        r = np.linalg.norm(x, axis=1)
        assert np.all(np.abs(F - approx).max(axis=1) < 20 * r ** 3 / L ** 5)
        half = kernels.periodic_pair_kernel(np.array([[L / 2, 0, 0], [L / 2, L / 2, L / 2],
                                                      [0, L / 2, L / 2]]), L)
        assert np.abs(half).max() < 1e-15


def test_coarse_table_equals_direct_ewald():
    # The table's band-limited Fourier part (inverse DFT on the mesh) plus its
    # real-space part must equal a direct Ewald evaluation with a different
    # screening length: Ewald sums are independent of the split.
    rng = np.random.default_rng(5)
    for nc in (8, 16, 64):
        T = kernels.coarse_kernel_table(nc)
        D = rng.integers(-nc // 2, nc // 2, size=(40, 3))
        direct = kernels.periodic_pair_kernel(4.0 * D, 4.0 * nc, h_max=6)
        tab = T[:, D[:, 2] % nc, D[:, 1] % nc, D[:, 0] % nc].T
        np.testing.assert_allclose(tab, direct, rtol=0, atol=1e-13 * np.abs(T).max())


def test_matching_force_odd_zero_and_newtonian_far_away():
    nc = 16
    d = kernels.fine_kernel_support()
    A = kernels.matching_force(d, nc)
    np.testing.assert_allclose(kernels.matching_force(-d, nc), -A, rtol=0, atol=1e-15)
    np.testing.assert_allclose(kernels.matching_force(np.zeros((1, 3), int), nc), 0, atol=1e-16)
    nc = 64
    far = np.array([[12, 0, 0], [0, -14, 0], [10, 10, 0], [-9, 9, 9], [16, 3, -5]])
    ref = kernels.periodic_pair_kernel(far.astype(float), 4.0 * nc)
    ratio = (kernels.matching_force(far, nc) * ref).sum(1) / (ref ** 2).sum(1)
    np.testing.assert_allclose(ratio, 1.0, atol=0.01)


def test_fine_kernel_support_and_matching():
    nc = 8
    nf = 32
    table = kernels.fine_kernel_table(nc)
    i = kernels.nearest_image(nf)
    dz, dy, dx = np.meshgrid(i, i, i, indexing="ij")
    r2 = dx * dx + dy * dy + dz * dz
    assert np.all(table[:, r2 >= kernels.R_CUT ** 2] == 0)
    assert np.all(table[:, r2 == 0] == 0)
    d, Ks = kernels.fine_kernel_values(nc)
    np.testing.assert_allclose(Ks + kernels.matching_force(d, nc),
                               kernels.periodic_pair_kernel(d.astype(float), 4.0 * nc),
                               rtol=0, atol=1e-15)


def test_coarse_fft_chain_reproduces_matching_force():
    # Unit source at each of the 64 fine-cell centres of one coarse cell,
    # coarse CIC -> FFT convolution with K_l -> coarse CIC gather at s + d,
    # averaged over s: must equal the direct-sum definition A(d).
    nc = 8
    op = force.ForceOperator(nc)
    Klh = op.Kl_hat()
    d = kernels.fine_kernel_support()
    acc = np.zeros((d.shape[0], 3))
    base = 4.0 * 3                      # coarse cell 3, away from nothing in particular
    for sx in range(4):
        for sy in range(4):
            for sz in range(4):
                s = base + np.array([sx, sy, sz]) + 0.5
                rho = np.zeros((nc, nc, nc))
                for idx, w in _cic_3d(s, 4.0, nc):
                    rho[idx] += w
                F = np.stack([np.fft.irfftn(np.fft.rfftn(rho) * Klh[c], s=rho.shape, axes=(0, 1, 2))
                              for c in range(3)])
                for k, dd in enumerate(d):
                    for idx, w in _cic_3d(s + dd, 4.0, nc):
                        acc[k] += w * F[(slice(None),) + idx]
    acc /= 64.0
    np.testing.assert_allclose(acc, kernels.matching_force(d, nc), rtol=0, atol=1e-13)


def test_fft_convolution_equals_direct_sum():
    rng = np.random.default_rng(0)
    nc = 8
    nf = 32
    op = force.ForceOperator(nc)
    Q = rng.integers(0, nc * 256, size=(300, 3))
    Fs = op.fine_field(Q)
    rho_f = op.fine_density(Q).astype(float) / 2.0 ** 21
    np.testing.assert_allclose(Fs, direct.fine_field_direct(rho_f, nc), rtol=0,
                               atol=1e-12 * np.abs(Fs).max())
    Fl = op.coarse_field(Q)
    rho_c = op.coarse_density(Q).astype(float) / 2.0 ** 27
    np.testing.assert_allclose(Fl, direct.coarse_field_direct(rho_c, nc), rtol=0,
                               atol=1e-12 * np.abs(Fl).max())


def test_zero_self_force_and_momentum_conservation():
    rng = np.random.default_rng(1)
    op = force.ForceOperator(8)
    for _ in range(5):
        Q = rng.integers(0, 8 * 256, size=(1, 3))
        assert np.abs(op.particle_force(Q)).max() < 1e-14
    Q = rng.integers(0, 8 * 256, size=(3000, 3))
    g = op.particle_force(Q)
    assert np.abs(g.sum(axis=0)).max() < 1e-12 * np.abs(g).max() * Q.shape[0] ** 0.5


def test_two_particle_force_is_newtonian():
    # Source field from one particle, gathered at test positions (test
    # particles do not deposit).  Beyond a few fine cells the radial force
    # must follow the periodic 1/r^2 force; the mean is within 2% for
    # 8 <= r <= nf/8 and within 5% for 2 <= r < 6.
    rng = np.random.default_rng(2)
    nc = 32
    nf = 4 * nc
    op = force.ForceOperator(nc)
    samples_r, samples_f = [], []
    for _ in range(6):
        Qs = rng.integers(0, nc * 256, size=(1, 3))
        Fs, Fl = op.fine_field(Qs), op.coarse_field(Qs)
        xs = codec.positions_from_codes(Qs)[0]
        r = rng.uniform(2.0, nf / 8.0, size=400)
        n = rng.normal(size=(400, 3))
        n /= np.linalg.norm(n, axis=1, keepdims=True)
        Qt = codec.codes_from_positions(xs[None, :] + r[:, None] * n, nc)
        dx = codec.positions_from_codes(Qt) - xs[None, :]
        dx -= nf * np.round(dx / nf)
        rr = np.linalg.norm(dx, axis=1)
        g = np.stack([cic.interpolate(Fs[c], Qt, 1) + cic.interpolate(Fl[c], Qt, 4)
                      for c in range(3)], axis=1)
        ref = kernels.periodic_pair_kernel(dx, float(nf))
        samples_r.append(rr)
        samples_f.append((g * dx).sum(1) / (ref * dx).sum(1))
    rr = np.concatenate(samples_r)
    f = np.concatenate(samples_f)
    far = (rr >= 8) & (rr <= nf / 8)
    assert far.sum() > 500
    assert abs(f[far].mean() - 1.0) < 0.02
    near = (rr >= 2) & (rr < 6)
    assert abs(f[near].mean() - 1.0) < 0.05


@pytest.mark.parametrize("T", [16, 20])
def test_tiling_invariance(T):
    # The derivation the GPU tiles rely on: a 32^3 periodic tile mesh holding
    # nodes [t0-6, t0+T+6) with every particle's CIC clipped to it gives the
    # full-mesh short-range field on the tile's nodes [t0-1, t0+T].
    rng = np.random.default_rng(3)
    nc = 16
    nf = 4 * nc
    M = 32
    op = force.ForceOperator(nc)
    Q = rng.integers(0, nc * 256, size=(6000, 3))
    full = op.fine_field(Q)
    t0 = np.array([8, 24, 44])
    origin = t0 - kernels.R_CUT
    node, w = cic.corners(Q, nf, 1)
    iz, iy, ix = node // (nf * nf), (node // nf) % nf, node % nf
    lx, ly, lz = (ix - origin[0]) % nf, (iy - origin[1]) % nf, (iz - origin[2]) % nf
    keep = (lx < M) & (ly < M) & (lz < M)
    rho = np.zeros((M, M, M))
    np.add.at(rho, (lz[keep], ly[keep], lx[keep]), w[keep] / 2.0 ** 21)
    Kt = kernels.fine_kernel_table(nc, M)
    tile = np.stack([np.fft.irfftn(np.fft.rfftn(rho) * np.fft.rfftn(Kt[c]), s=rho.shape, axes=(0, 1, 2))
                     for c in range(3)])
    sel = np.arange(-1, T + 1)
    a = tile[:, :, :, :][:, (sel + 6)[:, None, None], (sel + 6)[None, :, None],
                         (sel + 6)[None, None, :]]
    gz = (t0[2] + sel) % nf
    gy = (t0[1] + sel) % nf
    gx = (t0[0] + sel) % nf
    b = full[:, gz[:, None, None], gy[None, :, None], gx[None, None, :]]
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-12 * np.abs(full).max())


def test_sampled_force_equals_whole_mesh_force():
    # the large-box variant (chunked coarse density, direct short-range sums
    # near chosen particles) is the same force as the whole-mesh oracle
    from oracle import dynamics, force, ic
    st, _, _ = ic.zeldovich(7, 32, 16, 0.05, slope=-1.5, k_c=np.pi / 2, rms_disp=0.6)
    st = dynamics.Simulation(16, 0.05, 1.0, 6).run(st, 3)     # clustered
    Q = st.codes()
    op = force.ForceOperator(16)
    gs, gl = op.particle_force(Q, parts=True)
    rng = np.random.default_rng(0)
    idx = rng.choice(Q.shape[0], 40, replace=False)
    np.testing.assert_array_equal(force.coarse_density_chunked(Q, 16, chunk=1000),
                                  op.coarse_density(Q))
    fs = force.sampled_fine_force(Q, st.counts, 16, idx)
    np.testing.assert_allclose(fs, gs[idx], rtol=1e-9, atol=1e-12 * np.abs(gs).max())
    g = force.sampled_force(Q, st.counts, 16, idx)
    np.testing.assert_allclose(g, (gs + gl)[idx], rtol=1e-9, atol=1e-12 * np.abs(gs + gl).max())
