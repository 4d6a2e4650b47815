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
