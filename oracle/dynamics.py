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
  The isotropic dispersion is sigma^2 = sum_i sum_d (p_id - v_c,d)^2 / (3N),
  with each squared float32 difference rounded to a multiple of 2^-32 and
  summed exactly; sigma^2 = fl64(hi) 2^64 + fl64(lo) in units of 2^-32 of the
  128-bit sum, divided by 3N, and sigma = fl32(sqrt(sigma^2)), or 2^-24 when
  the sum is 0.  u then follows ``codec.encode_velocity``.
"""

import math

import numpy as np

from . import codec, force as force_mod

P_FIX_BITS = 24      # p rounded to multiples of 2^-24 for the cell sums
D2_FIX_BITS = 32     # squared deviations rounded to multiples of 2^-32
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


def cell_means(cell, p32, ncells):
    """v_c per cell from fixed-point sums (see module docstring)."""
    P = np.rint(np.asarray(p32, dtype=np.float32).astype(np.float64) * 2.0 ** P_FIX_BITS)
    P = P.astype(np.int64)
    S = np.zeros((ncells, 3), dtype=np.int64)
    np.add.at(S, cell, P)
    n = np.bincount(cell, minlength=ncells).astype(np.int64)
    vc = np.zeros((ncells, 3), dtype=np.float32)
    nz = n > 0
    Sf = (S[nz].astype(np.float32) * np.float32(2.0 ** -P_FIX_BITS)).astype(np.float32)
    vc[nz] = (Sf / n[nz, None].astype(np.float32)).astype(np.float32)
    return vc, S, n


def dispersion(p32, vc_of_particle):
    """sigma (float32) and the exact 128-bit integer sum it comes from."""
    d = (np.asarray(p32, dtype=np.float32) - np.asarray(vc_of_particle, dtype=np.float32))
    d = d.astype(np.float32).astype(np.float64)
    D = np.rint(d * d * 2.0 ** D2_FIX_BITS)
    if D.size and D.max() >= 2.0 ** 64:
        raise OverflowError("velocity deviation too large for the dispersion sum")
    Du = D.astype(np.uint64).ravel()
    # exact 128-bit sum: split each term into 32-bit halves, sum each half in
    # int64 (no overflow below 2^31 terms), recombine with Python integers
    lo32 = (Du & np.uint64(0xFFFFFFFF)).astype(np.int64).sum(dtype=np.int64)
    hi32 = (Du >> np.uint64(32)).astype(np.int64).sum(dtype=np.int64)
    total = (int(hi32) << 32) + int(lo32)
    hi, lo = total >> 64, total & ((1 << 64) - 1)
    n3 = 3 * d.shape[0]
    if total == 0 or n3 == 0:
        return np.float32(SIGMA_FLOOR), total
    s2 = (float(hi) * 2.0 ** 64 + float(lo)) * 2.0 ** -D2_FIX_BITS / float(n3)
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
    vc, _, _ = cell_means(cell, p32, ncells)
    sigma, _ = dispersion(p32, vc[cell])
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
