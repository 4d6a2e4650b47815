"""Pins of the oracle's integer cloud-in-cell assignment."""

import numpy as np

from oracle import cic, codec


def _float_cic_weight(x_nodeunits, node, n):
    # textbook CIC: weight max(0, 1 - |x - (node + 1/2)|) with periodic distance
    d = np.abs(x_nodeunits - (node + 0.5))
    d = np.minimum(d, n - d)
    return np.maximum(0.0, 1.0 - d)


def test_mass_conservation_exact():
    rng = np.random.default_rng(0)
    nc = 8
    Q = rng.integers(0, nc * 256, size=(5000, 3))
    for n, h in ((4 * nc, 1), (nc, 4), (2 * nc, 2)):
        U = cic.node_units(h)
        rho = cic.deposit(Q, n, h)
        assert rho.sum() == Q.shape[0] * (2 * U) ** 3
        assert rho.min() >= 0


def test_integer_weights_equal_textbook_cic():
    rng = np.random.default_rng(1)
    nc = 4
    Q = rng.integers(0, nc * 256, size=(400, 3))
    for n, h in ((4 * nc, 1), (nc, 4)):
        U = cic.node_units(h)
        node, w = cic.corners(Q, n, h)
        x = codec.positions_from_codes(Q) / h          # node units
        for c in range(8):
            iz = node[:, c] // (n * n)
            iy = (node[:, c] // n) % n
            ix = node[:, c] % n
            ref = (_float_cic_weight(x[:, 0], ix, n) * _float_cic_weight(x[:, 1], iy, n)
                   * _float_cic_weight(x[:, 2], iz, n))
            np.testing.assert_array_equal(w[:, c] / float((2 * U) ** 3), ref)


def test_interpolation_reproduces_linear_fields():
    # CIC gather is exact for fields linear in the node position (away from
    # the periodic seam); a shifted node convention would break this
    rng = np.random.default_rng(2)
    nc = 8
    n, h = 4 * nc, 1
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    field = 0.3 + 1.5 * (x + 0.5) - 0.25 * (y + 0.5) + 2.0 * (z + 0.5)
    Q = rng.integers(64 * 2, 64 * (n - 2), size=(1000, 3))
    xp = codec.positions_from_codes(Q)
    ref = 0.3 + 1.5 * xp[:, 0] - 0.25 * xp[:, 1] + 2.0 * xp[:, 2]
    np.testing.assert_allclose(cic.interpolate(field, Q, h), ref, rtol=0, atol=1e-12)


def test_two_byte_weights_are_rounded_exact_products():
    # 2-byte codes: every corner's exact 2^-45 (fine) / 2^-51 (coarse) product,
    # rounded half-even to the 1-byte unit, by Python integer arithmetic
    from fractions import Fraction
    rng = np.random.default_rng(11)
    Q = rng.integers(0, 8 * 65536, size=(300, 3))
    for h in (1, 4):
        U = cic.node_units(h, 2)
        node, w = cic.corners(Q, 8 * 4 // h, h, pos_bytes=2)
        for i in range(0, 300, 7):
            s = 2 * Q[i] + 1 - U
            i0 = s // (2 * U)
            w1 = s - 2 * U * i0
            k = 0
            for dz in (0, 1):
                for dy in (0, 1):
                    for dx in (0, 1):
                        exact = 1
                        for d, dd in ((0, dx), (1, dy), (2, dz)):
                            exact *= int(w1[d]) if dd else int(2 * U - w1[d])
                        f = Fraction(exact, 1 << 24)
                        fl = f.numerator // f.denominator
                        rem = f - fl
                        r = fl + (1 if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and fl % 2) else 0)
                        assert w[i, k] == r
                        k += 1
        # mass per particle: 1 within 4 units (eight roundings of at most 1/2)
        assert np.abs(w.sum(axis=1) - cic.weight_unit(h, 2)).max() <= 4


def test_two_byte_self_force_vanishes_and_mass_is_kept():
    from oracle import force
    rng = np.random.default_rng(13)
    Q = np.repeat(rng.integers(0, 8 * 65536, size=(1, 3)), 5, axis=0)
    g = force.ForceOperator(8, pos_bytes=2).particle_force(Q)
    assert np.abs(g).max() < 1e-12
    Q = rng.integers(0, 8 * 65536, size=(4000, 3))
    rho = cic.deposit(Q, 32, 1, pos_bytes=2)
    assert abs(int(rho.sum()) - 4000 * cic.weight_unit(1, 2)) <= 4 * 4000
