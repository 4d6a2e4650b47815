"""Zel'dovich initial conditions (Sec. IV-A.2).

Test infrastructure only (see ``oracle/__init__``).

Sec. IV-A.2 sets particles at the start with the Zel'dovich approximation.
The synthetic workload replaces the paper's LCDM spectrum with a power law
P(k) = k^slope exp(-(k/k_c)^2).  Steps, in order:

1. White noise on the n_p^3 particle lattice, point i (flat, x fastest):
   Box-Muller of two uniforms drawn from the counter-based SplitMix64
   generator (Steele, Lea & Flood, OOPSLA 2014) at counters 2i and 2i+1.
   SplitMix64 output for counter j: z = seed + (j+1) * 0x9E3779B97F4A7C15,
   then z ^= z>>30, z *= 0xBF58476D1CE4E5B9, z ^= z>>27,
   z *= 0x94D049BB133111EB, z ^= z>>31 (all mod 2^64).
   u1 = ((z1 >> 11) + 1) 2^-53 in (0, 1], u2 = (z2 >> 11) 2^-53 in [0, 1),
   w = sqrt(-2 ln u1) cos(2 pi u2).
2. delta~ = DFT(w) sqrt(P(k)), k = 2 pi n / L, L = nf (fine cells).
3. Displacement Psi~ = i k / k^2 delta~ (so delta = -div Psi), with k = 0 and
   every mode on a Nyquist plane set to zero.
4. Psi = inverse DFT, scaled so that a_i sqrt(<|Psi|^2>) = rms_disp.
5. x = q + a_i Psi on the lattice q = (i + 1/2) nf / n_p, and the EdS growing
   mode p = a^2 dx/dt = a_i^(3/2) Psi.
6. Encode with Q = floor(x / q) (float64 decision) and ``dynamics.encode``.
"""

import numpy as np

from . import dynamics

GAMMA = np.uint64(0x9E3779B97F4A7C15)
MIX1 = np.uint64(0xBF58476D1CE4E5B9)
MIX2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed, counter):
    """SplitMix64 output at integer counters (numpy uint64, wrapping)."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (np.asarray(counter, dtype=np.uint64) + np.uint64(1)) * GAMMA
        z = (z ^ (z >> np.uint64(30))) * MIX1
        z = (z ^ (z >> np.uint64(27))) * MIX2
        return z ^ (z >> np.uint64(31))


def white_noise(seed, n_p):
    """Unit Gaussian field on the lattice, [z, y, x] float64."""
    i = np.arange(n_p ** 3, dtype=np.uint64)
    z1 = splitmix64(seed, 2 * i)
    z2 = splitmix64(seed, 2 * i + np.uint64(1))
    u1 = ((z1 >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53
    u2 = (z2 >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    w = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
    return w.reshape(n_p, n_p, n_p)


def power_law(k, slope, k_c):
    """P(k) = k^slope exp(-(k/k_c)^2); zero at k = 0."""
    k = np.asarray(k, dtype=np.float64)
    out = np.zeros_like(k)
    nz = k > 0
    out[nz] = k[nz] ** slope * np.exp(-(k[nz] / k_c) ** 2)
    return out


def lattice_frequencies(n_p):
    """Integer frequencies n in [-n_p/2, n_p/2) along one axis."""
    return np.rint(np.fft.fftfreq(n_p) * n_p).astype(np.int64)


def displacement(seed, n_p, nf, slope, k_c):
    """Unnormalised Zel'dovich displacement Psi [3, z, y, x] (steps 1-3)."""
    w = white_noise(seed, n_p)
    w_hat = np.fft.fftn(w)
    n = lattice_frequencies(n_p)
    nz_, ny_, nx_ = np.meshgrid(n, n, n, indexing="ij")
    kx = 2 * np.pi * nx_ / nf
    ky = 2 * np.pi * ny_ / nf
    kz = 2 * np.pi * nz_ / nf
    k2 = kx * kx + ky * ky + kz * kz
    delta_hat = w_hat * np.sqrt(power_law(np.sqrt(k2), slope, k_c))
    nyq = -(n_p // 2)
    zero = (k2 == 0) | (nx_ == nyq) | (ny_ == nyq) | (nz_ == nyq)
    inv_k2 = np.zeros_like(k2)
    inv_k2[~zero] = 1.0 / k2[~zero]
    psi = []
    for kd in (kx, ky, kz):
        psi_hat = 1j * kd * inv_k2 * delta_hat
        psi.append(np.fft.ifftn(psi_hat).real)
    return np.stack(psi)


def zeldovich(seed, n_p, nc, a_init, slope=-1.5, k_c=np.pi / 2, rms_disp=0.3, pos_bytes=1,
              cosmo=None):
    """Compressed initial state at a_init (steps 1-6).

    Returns (state, x float64 [N,3], p float64 [N,3]) with particles in
    lattice order for x and p.  cosmo: a ``cosmology.Cosmology``; the
    growing-mode momentum is then p = a^2 E f (x - q) instead of the
    Einstein-de Sitter sqrt(a) (x - q).
    """
    nf = 4 * nc
    psi = displacement(seed, n_p, nf, slope, k_c)
    psi = psi.reshape(3, -1).T                       # [N, 3], lattice order
    rms = np.sqrt((psi * psi).sum(axis=1).mean())
    psi = psi * (rms_disp / (a_init * rms))
    i = np.arange(n_p)
    qz, qy, qx = np.meshgrid(i, i, i, indexing="ij")
    spacing = nf / n_p
    q = (np.stack([qx.ravel(), qy.ravel(), qz.ravel()], axis=1) + 0.5) * spacing
    x = q + a_init * psi
    if cosmo is None:
        p = a_init ** 1.5 * psi
    else:
        p = cosmo.ic_momentum_factor(a_init) * (a_init * psi)
    U = 64 if pos_bytes == 1 else 16384
    B = 256 if pos_bytes == 1 else 65536
    Q = np.mod(np.floor(x * U).astype(np.int64), nc * B)
    state = dynamics.encode(Q, p.astype(np.float32), nc, a_init, 0, pos_bytes)
    return state, x, p
