"""Fixed-point particle codec (Sec. III-A, Eq. 2 and Eq. 3; Sec. III-B.2, Eq. 4).

Test infrastructure only (see ``oracle/__init__``).

Conventions (readings of the paper, stated once here):

* Lengths are in fine cells.  The box holds ``nc`` coarse cells per side and
  ``nf = 4 * nc`` fine cells (the coarse mesh is 4x coarser, Sec. II).
* Eq. 2 numbers cells from 1; here cell indices ``c`` are 0-based, so the
  paper's ``n_c - 1`` is ``c``.  Flat cell index is row-major with x fastest:
  ``flat = cx + nc * (cy + nc * cz)``.
* Each coarse cell is split into ``B`` bins per dimension (``B = 256`` for the
  1-byte format of Eq. 2; ``B = 65536`` for the 2-byte option the paper
  mentions in Sec. III-A).  The global position code is ``Q = c * B + m`` and
  the decoded position is ``x = (Q + 1/2) * q`` with quantum ``q = 4 / B``
  fine cells (the bin centre of Eq. 2).
* Eq. 3 leaves the nonlinear map ``f`` open (the paper likens it to an
  inverse error function, and Sec. III-B.2 works with an arctangent form).  Reading:
  a Cauchy-quantile map of scale sigma.  Bin ``u`` of 256 covers the angle
  interval [pi(u/256 - 1/2), pi((u+1)/256 - 1/2)); its decoded value is the
  tangent of the bin-centre angle, ``T[u] = tan(pi((u + 1/2)/256 - 1/2))``;
  the edges are ``E[k] = tan(pi(k/256 - 1/2))``, k = 1..255.  Both tables are
  float32 (the paper's particles are 32-bit floats, Sec. III-B.2).
* Velocity decode: ``p = fl32(v_c + fl32(sigma * T[u]))``.  Encode:
  ``t = fl32(fl32(p - v_c) / sigma)`` and ``u = #{k in 1..255 : E[k] <= t}``.
  All of these are IEEE float32 operations, so any implementation that uses
  the same tables reproduces them bit for bit.
"""

import numpy as np

NBINS_V = 256  # velocity bins (1-byte u), Eq. 3


def bins_per_cell(pos_bytes=1):
    """B of Eq. 2: 256 bins for 1-byte m, 65536 for 2-byte m (Sec. III-A)."""
    if pos_bytes == 1:
        return 256
    if pos_bytes == 2:
        return 65536
    raise ValueError("pos_bytes must be 1 or 2")


def code_units_per_fine_cell(pos_bytes=1):
    """Number of position codes per fine cell, 1/q = B/4."""
    return bins_per_cell(pos_bytes) // 4


# ---------------------------------------------------------------- positions

def cell_index_of_particles(counts):
    """Flat coarse-cell index of every particle of a cell-ordered store.

    Sec. III-A: particles are stored cell by cell, and the per-cell count field
    restores each particle's cell.
    """
    counts = np.asarray(counts, dtype=np.int64)
    return np.repeat(np.arange(counts.size, dtype=np.int64), counts)


def unflatten_cell(flat, nc):
    flat = np.asarray(flat, dtype=np.int64)
    cx = flat % nc
    cy = (flat // nc) % nc
    cz = flat // (nc * nc)
    return np.stack([cx, cy, cz], axis=-1)


def flatten_cell(c, nc):
    c = np.asarray(c, dtype=np.int64)
    return c[..., 0] + nc * (c[..., 1] + nc * c[..., 2])


def decode_codes(counts, m, nc, pos_bytes=1):
    """Eq. 2 as integers: Q = c * B + m, shape [N, 3], int64."""
    B = bins_per_cell(pos_bytes)
    cell = unflatten_cell(cell_index_of_particles(counts), nc)
    return cell * B + np.asarray(m, dtype=np.int64)


def positions_from_codes(Q, pos_bytes=1):
    """Eq. 2: x = (Q + 1/2) q in fine cells (float64, exact)."""
    U = code_units_per_fine_cell(pos_bytes)
    return (np.asarray(Q, dtype=np.float64) + 0.5) / U


def codes_from_positions(x, nc, pos_bytes=1):
    """Inverse of Eq. 2: Q = floor(x / q), wrapped into the periodic box."""
    U = code_units_per_fine_cell(pos_bytes)
    B = bins_per_cell(pos_bytes)
    Q = np.floor(np.asarray(x, dtype=np.float64) * U).astype(np.int64)
    return np.mod(Q, nc * B)


def split_codes(Q, pos_bytes=1):
    """Q -> (cell c, bin m) with Q = c * B + m (Eq. 2)."""
    B = bins_per_cell(pos_bytes)
    Q = np.asarray(Q, dtype=np.int64)
    return Q // B, Q % B


# ---------------------------------------------------------------- velocities

def velocity_tables():
    """float32 decode table T[u] (bin centres) and edge table E[k] (Eq. 3).

    E[0] is -inf so that ``u = #{k >= 1 : E[k] <= t}`` can be computed with a
    search over E[1:].
    """
    u = np.arange(NBINS_V, dtype=np.float64)
    T = np.tan(np.pi * ((u + 0.5) / NBINS_V - 0.5)).astype(np.float32)
    k = np.arange(1, NBINS_V, dtype=np.float64)
    E = np.empty(NBINS_V, dtype=np.float32)
    E[0] = -np.inf
    E[1:] = np.tan(np.pi * (k / NBINS_V - 0.5)).astype(np.float32)
    return T, E


def decode_velocity(u, vc, sigma32):
    """Eq. 3: p = v_c + f(u), with f(u) = sigma * T[u] (float32 IEEE ops)."""
    T, _ = velocity_tables()
    s = np.float32(sigma32)
    return (np.asarray(vc, dtype=np.float32)
            + (s * T[np.asarray(u, dtype=np.int64)]).astype(np.float32)).astype(np.float32)


def velocity_argument(p, vc, sigma32):
    """t = fl32(fl32(p - v_c) / sigma), the argument of the inverse map."""
    d = (np.asarray(p, dtype=np.float32) - np.asarray(vc, dtype=np.float32)).astype(np.float32)
    return (d / np.float32(sigma32)).astype(np.float32)


def encode_velocity(p, vc, sigma32):
    """Eq. 3 inverse by definition: u = #{k in 1..255 : E[k] <= t}."""
    _, E = velocity_tables()
    t = velocity_argument(p, vc, sigma32)
    return np.searchsorted(E[1:], t, side="right").astype(np.uint8)


def atan_eq4(x):
    """Eq. 4: the paper's fast arctangent (Rajan et al. form, domain extended
    to |x| > 1 through atan(x) = +-pi/2 - atan(1/x)).  float64."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    small = np.abs(x) <= 1.0
    xs = x[small]
    out[small] = np.pi / 4 * xs + 0.273 * xs * (1.0 - np.abs(xs))
    big = ~small
    xb = x[big]
    inv = 1.0 / xb
    core = np.pi / (4.0 * xb) + (0.273 / xb) * (1.0 - np.abs(inv))
    out[big] = np.where(xb > 0, np.pi / 2, -np.pi / 2) - core
    return out


def encode_velocity_eq4(p, vc, sigma32):
    """Encode through an Eq. 4 first guess plus one edge fix-up step.

    The guess is the bin of the approximate angle; because Eq. 4's error
    (0.0038 rad, Sec. III-B.2) is below one bin width (pi/256 = 0.0123 rad),
    the guess is off by at most one bin, and one comparison against the edge
    table on each side restores the exact bin of ``encode_velocity``.
    """
    _, E = velocity_tables()
    t = velocity_argument(p, vc, sigma32)
    theta = atan_eq4(t.astype(np.float64))
    u0 = np.floor((theta / np.pi + 0.5) * NBINS_V).astype(np.int64)
    u0 = np.clip(u0, 0, NBINS_V - 1)
    up = (u0 < NBINS_V - 1) & (E[np.minimum(u0 + 1, NBINS_V - 1)] <= t)
    down = (u0 > 0) & (E[u0] > t)
    u0 = u0 + up.astype(np.int64) - down.astype(np.int64)
    return u0.astype(np.uint8)
