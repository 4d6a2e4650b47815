"""Brute-force real-space convolutions, used only to pin the FFT path of
``oracle.force`` (Eq. 1 states the convolution; the FFT is one way to do it).

Test infrastructure only (see ``oracle/__init__``).
"""

import numpy as np

from . import kernels


def fine_field_direct(rho, nc):
    """F_s(j) = sum_d rho(j - d) K_s(d) over the compact support, by shifts.

    `rho` is a float64 [z, y, x] fine-mesh density (any units) of a box of
    nc coarse cells."""
    d, Ks = kernels.fine_kernel_values(nc)
    out = np.zeros((3,) + rho.shape)
    for (dx, dy, dz), k in zip(d, Ks):
        shifted = np.roll(rho, shift=(dz, dy, dx), axis=(0, 1, 2))
        for c in range(3):
            out[c] += k[c] * shifted
    return out


def coarse_field_direct(rho, nc):
    """F_l(b) = sum_a rho(a) K_l(b - a) by a double loop over all cell pairs."""
    K = kernels.coarse_kernel_table(nc)
    out = np.zeros((3, nc, nc, nc))
    idx = np.arange(nc)
    for az in range(nc):
        for ay in range(nc):
            for ax in range(nc):
                r = rho[az, ay, ax]
                if r == 0:
                    continue
                iz = np.mod(idx - az, nc)
                iy = np.mod(idx - ay, nc)
                ix = np.mod(idx - ax, nc)
                out += r * K[:, iz][:, :, iy][:, :, :, ix]
    return out


def pair_force_direct(x_src, x_tgt):
    """Newtonian K(x_tgt - x_src) summed over the source particles' nearest
    images only (no periodic sum); float64 [Nt, 3]."""
    x_src = np.asarray(x_src, dtype=np.float64)
    x_tgt = np.asarray(x_tgt, dtype=np.float64)
    r = x_tgt[:, None, :] - x_src[None, :, :]
    return kernels.pair_kernel(r).sum(axis=1)
