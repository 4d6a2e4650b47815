"""Pins of the oracle's fixed-point codec (Eq. 2, Eq. 3, Eq. 4) against what
the paper and the mathematics fix."""

import numpy as np

from oracle import codec, dynamics


def test_paper_format_constants(golden):
    # Eq. 2: 256 bins per coarse cell; Sec. III-A: 6 bytes per particle.
    assert codec.bins_per_cell(1) == golden["bins_per_coarse_cell"]
    rng = np.random.default_rng(0)
    nc = 4
    Q = rng.integers(0, nc * 256, size=(50, 3))
    p = rng.normal(size=(50, 3)).astype(np.float32)
    st = dynamics.encode(Q, p, nc, 0.1)
    per_particle = st.m.dtype.itemsize * 3 + st.u.dtype.itemsize * 3
    assert per_particle == golden["bytes_per_particle"]
    assert per_particle * 4 == golden["float_bytes_per_particle"]


def test_position_roundtrip_exhaustive():
    # every bin of every cell of a small box decodes into its own cell, at the
    # bin centre, and re-encodes to the same code
    nc = 3
    B = 256
    m = np.arange(B)
    for c in range(nc):
        Q = c * B + m
        x = codec.positions_from_codes(Q)
        assert np.all((x >= 4 * c) & (x < 4 * (c + 1)))
        np.testing.assert_array_equal(codec.codes_from_positions(x, nc), Q)
        np.testing.assert_array_equal(x, 4 * c + (m + 0.5) * (4.0 / B))


def test_position_half_quantum_bound():
    rng = np.random.default_rng(1)
    nc = 16
    x = rng.uniform(0, 4 * nc, size=200000)
    xr = codec.positions_from_codes(codec.codes_from_positions(x, nc))
    d = np.abs(x - xr)
    d = np.minimum(d, 4 * nc - d)
    assert d.max() <= 0.5 * (4.0 / 256) + 1e-12


def test_cell_order_restores_cells():
    counts = np.array([0, 3, 0, 2, 1, 0, 0, 2], dtype=np.int32)   # nc = 2
    m = np.zeros((8, 3), dtype=np.uint8)
    Q = codec.decode_codes(counts, m, 2)
    cells = np.array([1, 1, 1, 3, 3, 4, 7, 7])
    c = codec.unflatten_cell(cells, 2)
    np.testing.assert_array_equal(Q, c * 256)


def test_velocity_tables_shape():
    T, E = codec.velocity_tables()
    assert np.all(np.diff(T) > 0)
    assert np.all(np.diff(E[1:]) > 0)
    # odd map: bin u and bin 255-u mirror each other
    np.testing.assert_array_equal(T[::-1], -T)
    # every centre lies strictly between its two edges
    assert np.all(T[1:255] > E[1:255]) and np.all(T[1:255] < E[2:256])
    assert T[0] < E[1] and T[255] > E[255]
    # the middle edge is tan(0) = 0
    assert E[128] == 0.0


def test_velocity_centres_roundtrip():
    T, _ = codec.velocity_tables()
    u = np.arange(256)
    for sigma in (1.0, 0.37, 12.5):
        for vc in (0.0, -3.25, 40.0):
            p = codec.decode_velocity(u, np.full(256, vc, np.float32), np.float32(sigma))
            u2 = codec.encode_velocity(p, np.full(256, vc, np.float32), np.float32(sigma))
            np.testing.assert_array_equal(u2, u)


def test_velocity_angle_bound():
    # |atan(t) - atan(T[u(t)])| <= half a bin width in angle, pi/512
    T, _ = codec.velocity_tables()
    rng = np.random.default_rng(2)
    t = np.concatenate([rng.standard_cauchy(300000), rng.normal(size=100000)]).astype(np.float32)
    u = codec.encode_velocity(t, np.zeros_like(t), np.float32(1.0))
    err = np.abs(np.arctan(t.astype(np.float64)) - np.arctan(T[u].astype(np.float64)))
    assert err.max() <= np.pi / 512 * (1 + 1e-6)


def test_eq4_max_error_is_the_papers(golden):
    x = np.concatenate([np.linspace(-40, 40, 4000001), np.logspace(-5, 5, 200001),
                        -np.logspace(-5, 5, 200001)])
    err = np.abs(codec.atan_eq4(x) - np.arctan(x)).max()
    assert err <= golden["eq4_max_abs_error_rad"]
    # and the bound is attained to the printed precision: the formula is the
    # paper's, not a better or worse one
    assert abs(err - golden["eq4_max_abs_error_rad"]) < 1e-4


def test_eq4_guess_plus_fixup_equals_definition():
    _, E = codec.velocity_tables()
    rng = np.random.default_rng(3)
    edges = E[1:]
    near = np.concatenate([edges, np.nextafter(edges, np.float32(np.inf)),
                           np.nextafter(edges, np.float32(-np.inf))])
    t = np.concatenate([near, rng.standard_cauchy(500000).astype(np.float32),
                        np.array([0, 1e30, -1e30, np.inf, -np.inf], dtype=np.float32)])
    t = t.astype(np.float32)
    z = np.zeros_like(t)
    np.testing.assert_array_equal(codec.encode_velocity_eq4(t, z, np.float32(1)),
                                  codec.encode_velocity(t, z, np.float32(1)))
