"""Integer cloud-in-cell mass assignment and interpolation (Sec. II, Eq. 1).

Test infrastructure only (see ``oracle/__init__``).

Reading (the paper names CIC, Sec. IV-D, but not its convention): mesh nodes
sit at cell centres (Hockney & Eastwood).  For a mesh of node spacing ``h``
fine cells and ``U = h * B / 4`` position codes per node spacing, a particle
with code ``Q`` (Eq. 2) sits at ``(Q + 1/2) / U`` node units, so
``s = 2Q + 1 - U`` is its offset from node 0's centre in units of 1/(2U).
Then ``i0 = floor(s / 2U)``, ``w1 = s - 2U*i0`` and ``w0 = 2U - w1``; the 3-D
weight is the product of the three 1-D weights, an exact integer in units of
``(2U)^-3``.  Fine mesh (h = 1, 1-byte): units 2^-21; coarse mesh (h = 4):
units 2^-27.  Because the weights are integers, the mesh density is an exact
integer and independent of summation order.

Reading for 2-byte positions (Sec. III-A, B = 65536): the exact 3-D product
is in units of 2^-45 (fine) and 2^-51 (coarse), too fine for the integer
meshes of a clustered box, so each corner's product is rounded half-even to
the 1-byte units (a factor 2^24 coarser: (256 / 65536 * ...)^3 = 2^-24 for
every mesh spacing), and the same rounded weights serve assignment and
interpolation.  A particle's mass is then 1 to within 4 units of 2^-21 (or
2^-27), and its force on itself stays exactly zero.
"""

import numpy as np

from .codec import bins_per_cell


def node_units(h, pos_bytes=1):
    """U: position codes per node spacing of a mesh with spacing h fine cells."""
    B = bins_per_cell(pos_bytes)
    U = h * B // 4
    if U * 4 != h * B:
        raise ValueError("node spacing must be a whole number of codes")
    return U


def weight_unit(h, pos_bytes=1):
    """Mesh density units per particle, (2U)^3 of the 1-byte format, which
    both formats use (see the module docstring)."""
    return (2 * node_units(h, 1)) ** 3


def round_half_even_shift(w, bits):
    """round-half-even(w / 2^bits) for non-negative int64 w."""
    w = np.asarray(w, dtype=np.int64)
    q = w >> bits
    r = w & ((1 << bits) - 1)
    half = 1 << (bits - 1)
    return q + ((r > half) | ((r == half) & ((q & 1) == 1))).astype(np.int64)


def weights_1d(Q, h, pos_bytes=1):
    """Per-axis CIC: (i0, w0, w1) with integer weights summing to 2U."""
    U = node_units(h, pos_bytes)
    s = 2 * np.asarray(Q, dtype=np.int64) + 1 - U
    i0 = np.floor_divide(s, 2 * U)
    w1 = s - 2 * U * i0
    w0 = 2 * U - w1
    return i0, w0, w1


def corners(Q, n, h, pos_bytes=1):
    """All 8 CIC corners of every particle.

    Returns (flat_node [N, 8] int64, weight [N, 8] int64); weights are in
    units of 1/weight_unit(h); for 1-byte positions each particle's 8
    weights sum to weight_unit(h) exactly, for 2-byte positions to within 4.
    """
    Q = np.asarray(Q, dtype=np.int64)
    i0, w0, w1 = weights_1d(Q, h, pos_bytes)
    nodes = []
    weights = []
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                ix = np.mod(i0[:, 0] + dx, n)
                iy = np.mod(i0[:, 1] + dy, n)
                iz = np.mod(i0[:, 2] + dz, n)
                wx = w1[:, 0] if dx else w0[:, 0]
                wy = w1[:, 1] if dy else w0[:, 1]
                wz = w1[:, 2] if dz else w0[:, 2]
                nodes.append(ix + n * (iy + n * iz))
                weights.append(wx * wy * wz)
    w = np.stack(weights, axis=1)
    if pos_bytes == 2:
        # (2U_2 / 2U_1)^3 = 256^3 = 2^24 for every mesh spacing
        w = round_half_even_shift(w, 24)
    return np.stack(nodes, axis=1), w


def deposit(Q, n, h, pos_bytes=1):
    """Integer CIC density on an n^3 periodic mesh, int64, units (2U)^-3.

    Index order of the returned array is [z, y, x] (x fastest in memory).
    """
    node, w = corners(Q, n, h, pos_bytes)
    rho = np.zeros(n * n * n, dtype=np.int64)
    np.add.at(rho, node.ravel(), w.ravel())
    return rho.reshape(n, n, n)


def interpolate(field, Q, h, pos_bytes=1):
    """CIC gather of a scalar mesh field [z, y, x] at the particles (float64)."""
    n = field.shape[0]
    node, w = corners(Q, n, h, pos_bytes)
    flat = np.asarray(field, dtype=np.float64).ravel()
    return (flat[node] * (w.astype(np.float64) / float(weight_unit(h, pos_bytes)))).sum(axis=1)
