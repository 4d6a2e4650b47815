"""Kick-drift step and cell-ordered re-encode (Sec. II, Sec. III-A).

Test infrastructure only (see ``oracle/__init__``).

Readings (the paper gives neither the integrator nor the units):

* Einstein-de Sitter background unless a ``cosmology.Cosmology`` is given
  (its LambdaCDM factors reduce to these), H0 = 1, time variable a, lengths in fine
  cells, particle mass 1, mean density rho_bar = N / nf^3.  Momentum
  p = a^2 dx/dt.  Poisson: lap(phi) = (3/2) delta / a, so the force is
  -grad(phi) = (3 / (8 pi rho_bar a)) g with g the unit-G field of ``force``.
* Time steps equal in log a: a_n = a_i (a_f / a_i)^(n / S); half steps
  a_{n+1/2} = sqrt(a_n a_{n+1}).  Momenta live at half steps; the state at
  step n holds x_n and p_{n-1/2} (p at a_0 before the first step).
* Kick from a_lo to a_hi: p += (3 / (8 pi rho_bar)) g * 2 (sqrt(a_hi) -
  sqrt(a_lo)).  Drift from a_n to a_{n+1}: dx = p * 2 (a_n^-1/2 -
  a_{n+1}^-1/2).
* The drift is integer: dQ = floor(fl32(p * c_d) + 1/2) with
  c_d = fl32(dx-factor / q), decided in float32 as the GPU does; Q wraps
  modulo nc * B.
* Re-encode (Sec. III-A): particles are re-grouped by new coarse cell in
  row-major x-fastest order (within-cell order is unspecified); counts are
  int32.  v_c is the cell mean of p: each p is rounded to a multiple of
  2^-24, the int64 sum S is exact, and v_c = fl32(fl32(S) 2^-24 / n), a
  float32 division of the rounded sum (the paper fixes v_c = <v>, not how
  its stored value is rounded).
  The isotropic dispersion sigma^2 is the variance of Delta v = v - <v>
  about the cell average <v> (Eq. 3 defines v_c as that average and the
  velocity map by the variance of Delta v), taken exactly over the same
  fixed-point momenta P = round(p 2^24) that give the cell sums S: per cell
  and axis sum_i (P_i - S/n)^2 = sum_i P_i^2 - S^2/n, so
  sigma^2 = (T - U) 2^-48 / (3N) with T = sum over particles and axes of P^2
  and U = sum over cells and axes of floor(S^2 / n) (integers; the floor
  moves sigma^2 by less than one unit of 2^-48 per cell and axis).  The
  128-bit integer T - U is converted as fl64(hi) 2^64 + fl64(lo), scaled by
  2^-48 and divided by 3N; sigma = fl32(sqrt(sigma^2)), or 2^-24 when
  T - U is 0.  u then follows ``codec.encode_velocity``.
"""

import math

import numpy as np

from . import codec, force as force_mod

P_FIX_BITS = 24      # p rounded to multiples of 2^-24 for the cell sums
SIGMA_FLOOR = 2.0 ** -24


def schedule(a_init, a_final, n_steps):
    n = np.arange(n_steps + 1, dtype=np.float64)
    return a_init * (a_final / a_init) ** (n / n_steps)


def step_factors(a_init, a_final, n_steps, n, n_particles, nf, cosmo=None):
    """(kick factor, drift factor) of step n, float64.

    kick: multiplies g; drift: multiplies p to give dx in fine cells.
    cosmo: a ``cosmology.Cosmology`` for a LambdaCDM background (its
    integrals over a); None is Einstein-de Sitter in closed form.
    """
    a = schedule(a_init, a_final, n_steps)
    a_lo = a[0] if n == 0 else math.sqrt(a[n - 1] * a[n])
    a_hi = math.sqrt(a[n] * a[n + 1])
    rho_bar = n_particles / float(nf) ** 3
    if cosmo is not None:
        kick = 3.0 * cosmo.om / (8.0 * math.pi * rho_bar) * cosmo.kick_integral(a_lo, a_hi)
        return kick, cosmo.drift_integral(a[n], a[n + 1])
    kick = 3.0 / (8.0 * math.pi * rho_bar) * 2.0 * (math.sqrt(a_hi) - math.sqrt(a_lo))
    drift = 2.0 * (1.0 / math.sqrt(a[n]) - 1.0 / math.sqrt(a[n + 1]))
    return kick, drift


class State:
    """Compressed particle store: counts, per-particle (m, u) in cell order,
    the coarse velocity field v_c and sigma (Sec. III-A)."""

    def __init__(self, nc, counts, m, u, vc, sigma, a, step=0, pos_bytes=1):
        self.nc = nc
        self.counts = np.asarray(counts, dtype=np.int32)
        self.m = np.asarray(m)
        self.u = np.asarray(u, dtype=np.uint8)
        self.vc = np.asarray(vc, dtype=np.float32)      # [nc^3, 3]
        self.sigma = np.float32(sigma)
        self.a = float(a)
        self.step = int(step)
        self.pos_bytes = pos_bytes

    @property
    def n(self):
        return int(self.counts.sum())

    def codes(self):
        return codec.decode_codes(self.counts, self.m, self.nc, self.pos_bytes)

    def momenta(self):
        cell = codec.cell_index_of_particles(self.counts)
        return codec.decode_velocity(self.u, self.vc[cell], self.sigma)

    def positions(self):
        return codec.positions_from_codes(self.codes(), self.pos_bytes)


def fixed_momenta(p32):
    """P = round(p 2^24) (half to even), int64, the fixed point of the cell sums."""
    P = np.rint(np.asarray(p32, dtype=np.float32).astype(np.float64) * 2.0 ** P_FIX_BITS)
    return P.astype(np.int64)


def cell_means(cell, p32, ncells):
    """v_c per cell from fixed-point sums (see module docstring)."""
    P = fixed_momenta(p32)
    S = np.zeros((ncells, 3), dtype=np.int64)
    np.add.at(S, cell, P)
    n = np.bincount(cell, minlength=ncells).astype(np.int64)
    vc = np.zeros((ncells, 3), dtype=np.float32)
    nz = n > 0
    Sf = (S[nz].astype(np.float32) * np.float32(2.0 ** -P_FIX_BITS)).astype(np.float32)
    vc[nz] = (Sf / n[nz, None].astype(np.float32)).astype(np.float32)
    return vc, S, n


def _sum_of_squares(P):
    """Exact sum of P^2 over an int64 array with |P| < 2^44 (Python integer):
    P = a 2^22 + b with 0 <= b < 2^22, each part's sum taken in int64 chunks."""
    P = np.asarray(P, dtype=np.int64).ravel()
    a = P >> 22
    b = P & ((1 << 22) - 1)
    total = 0
    for i in range(0, P.size, 1 << 16):
        aa, bb = a[i:i + (1 << 16)], b[i:i + (1 << 16)]
        total += (int((aa * aa).sum(dtype=np.int64)) << 44) + \
            (int((2 * aa * bb).sum(dtype=np.int64)) << 22) + int((bb * bb).sum(dtype=np.int64))
    return total


def dispersion(p32, S, n):
    """sigma (float32) and the exact integer T - U it comes from, from the
    momenta p32 [N, 3] and the cell sums S [C, 3] and counts n [C] of
    ``cell_means`` (see module docstring)."""
    P = fixed_momenta(p32)
    if P.size and np.abs(P).max() >= 2 ** 44:
        raise OverflowError("momentum too large for the fixed-point moments")
    T = _sum_of_squares(P)
    U = 0
    nz = np.nonzero(n > 0)[0]
    for srow, cnt in zip(S[nz].tolist(), n[nz].tolist()):
        for v in srow:
            U += (v * v) // cnt
    total = T - U
    n3 = 3 * P.shape[0]
    if total == 0 or n3 == 0:
        return np.float32(SIGMA_FLOOR), total
    hi, lo = total >> 64, total & ((1 << 64) - 1)
    s2 = (float(hi) * 2.0 ** 64 + float(lo)) * 2.0 ** -48 / float(n3)
    return np.float32(math.sqrt(s2)), total


def encode(Q, p32, nc, a, step=0, pos_bytes=1):
    """Build the compressed store from integer codes Q [N,3] and float32 p."""
    Q = np.asarray(Q, dtype=np.int64)
    p32 = np.asarray(p32, dtype=np.float32)
    B = codec.bins_per_cell(pos_bytes)
    c, m = codec.split_codes(Q, pos_bytes)
    cell = codec.flatten_cell(c, nc)
    ncells = nc ** 3
    counts = np.bincount(cell, minlength=ncells)
    vc, S, n = cell_means(cell, p32, ncells)
    sigma, _ = dispersion(p32, S, n)
    u = codec.encode_velocity(p32, vc[cell], sigma)
    order = np.argsort(cell, kind="stable")
    mdtype = np.uint8 if B == 256 else np.uint16
    return State(nc, counts.astype(np.int32), m[order].astype(mdtype), u[order],
                 vc, sigma, a, step, pos_bytes)


def kick_drift(Q, p32, g, kick, drift, nc, pos_bytes=1):
    """One kick (float64, rounded to float32) and one integer drift."""
    U = codec.code_units_per_fine_cell(pos_bytes)
    B = codec.bins_per_cell(pos_bytes)
    p_new = (np.asarray(p32, dtype=np.float32).astype(np.float64)
             + kick * np.asarray(g, dtype=np.float64)).astype(np.float32)
    cd = np.float32(drift * U)
    dq = np.floor((p_new * cd).astype(np.float32) + np.float32(0.5)).astype(np.int64)
    Q_new = np.mod(np.asarray(Q, dtype=np.int64) + dq, nc * B)
    return Q_new, p_new


class Simulation:
    """Plain PM-PM evolution of a compressed state (oracle)."""

    def __init__(self, nc, a_init, a_final, n_steps, pos_bytes=1, cosmo=None):
        self.nc = nc
        self.nf = 4 * nc
        self.a_init, self.a_final, self.n_steps = a_init, a_final, n_steps
        self.pos_bytes = pos_bytes
        self.cosmo = cosmo
        self.op = force_mod.ForceOperator(nc, pos_bytes)

    def forces(self, state):
        return self.op.particle_force(state.codes())

    def step(self, state):
        n = state.step
        if n >= self.n_steps:
            raise ValueError("schedule exhausted")
        a = schedule(self.a_init, self.a_final, self.n_steps)
        Q = state.codes()
        p = state.momenta()
        g = self.op.particle_force(Q)
        kick, drift = step_factors(self.a_init, self.a_final, self.n_steps, n,
                                   Q.shape[0], self.nf, self.cosmo)
        Q_new, p_new = kick_drift(Q, p, g, kick, drift, self.nc, self.pos_bytes)
        return encode(Q_new, p_new, self.nc, a[n + 1], n + 1, self.pos_bytes)

    def run(self, state, steps):
        for _ in range(steps):
            state = self.step(state)
        return state
