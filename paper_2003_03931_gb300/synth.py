"""Seeded synthetic inputs shared by the tests, the smoke check and the bench.

Holds no arithmetic of the method: only random particle codes and momenta
with the shapes of the paper's workload (clustered positions, bulk flows
plus dispersion), and the workload table.  Lengths are in fine cells; a box
of nc coarse cells has 256 nc position codes per side.
"""

import numpy as np

# Workloads (particles per side, coarse cells per side, schedule)
WORKLOADS = {
    "c1_32": dict(np=32, nc=16, a_init=0.02, a_final=1.0, n_steps=10),
    "c2_128": dict(np=128, nc=64, a_init=0.02, a_final=1.0, n_steps=20),
    "c3_512": dict(np=512, nc=256, a_init=0.02, a_final=1.0, n_steps=20),
    "c4sub_256": dict(np=256, nc=128, a_init=0.02, a_final=1.0, n_steps=20),
    # the same box with 2-byte positions (Sec. III-A)
    "c4sub_256_pos2": dict(np=256, nc=128, a_init=0.02, a_final=1.0, n_steps=20, pos_bytes=2),
    # small ragged-tile case: 7 tiles of 4/5 coarse cells per side
    "ragged_32": dict(np=32, nc=32, a_init=0.02, a_final=1.0, n_steps=10),
    # the 512^3 box with the tile spectrum stored as FP16 (precision option)
    "c3_512_fp16": dict(np=512, nc=256, a_init=0.02, a_final=1.0, n_steps=20, fine_fp16=True),
    # the 256^3 box with the low-memory step (profiling its tile pass and re-encode)
    "c4sub_256_lowmem": dict(np=256, nc=128, a_init=0.02, a_final=1.0, n_steps=20, lowmem=True),
    # the paper's LambdaCDM background (Omega_m = 0.258, flat) from z = 99
    "lcdm_32": dict(np=32, nc=16, a_init=0.01, a_final=1.0, n_steps=10, omega_m=0.258,
                    omega_l=0.742),
    "lcdm_128": dict(np=128, nc=64, a_init=0.01, a_final=1.0, n_steps=20, omega_m=0.258,
                     omega_l=0.742),
    # 2048^3 particles (51.5 GB at 6 B/particle) on one GPU: low-memory step
    "c4_2048": dict(np=2048, nc=1024, a_init=0.02, a_final=1.0, n_steps=20, lowmem=True),
}

IC_SPECTRUM = dict(slope=-1.5, k_c=np.pi / 2, rms_disp=0.3)


def uniform_codes(rng, n, nc, bins=256):
    """Codes uniformly over the box, int32 [3, n] (bins per coarse cell: 256
    for 1-byte, 65536 for 2-byte positions)."""
    return rng.integers(0, nc * bins, size=(3, n)).astype(np.int32)


def clustered_codes(rng, n, nc, n_clusters=12, frac=0.6, width_fine=3.0, bins=256):
    """A fraction of the particles in Gaussian clumps (width in fine cells),
    the rest uniform; int32 [3, n]."""
    M = nc * bins
    Q = rng.integers(0, M, size=(3, n)).astype(np.int64)
    k = int(frac * n)
    centres = rng.integers(0, M, size=(3, n_clusters))
    which = rng.integers(0, n_clusters, size=k)
    off = rng.normal(scale=width_fine * bins / 4.0, size=(3, k))
    Q[:, :k] = np.mod(np.floor(centres[:, which] + off).astype(np.int64), M)
    return Q.astype(np.int32)


def momenta(rng, n, bulk=2.0, disp=0.5):
    """float32 [3, n]: a few large-scale bulk components plus dispersion."""
    p = rng.normal(scale=disp, size=(3, n)) + rng.normal(scale=bulk, size=(3, 1))
    return p.astype(np.float32)


def single_cell_codes(n, nc, cell=(3, 1, 2)):
    """Every particle in one coarse cell, spread over its bins, int32 [3, n]."""
    m = np.arange(n) % 256
    Q = np.stack([np.full(n, c * 256) for c in cell]) + np.stack([m, m[::-1], (m * 7) % 256])
    return (Q % (nc * 256)).astype(np.int32)
