"""Per-particle PM-PM force on full periodic meshes (Sec. II, Eq. 1).

Test infrastructure only (see ``oracle/__init__``).

Eq. 1: each force component is the mesh density convolved with a component
kernel, done as a product in Fourier space.  The oracle applies it on two
whole periodic meshes, with no tiles:

* fine level: integer CIC density on the nf^3 fine mesh (units 2^-21 for the
  1-byte format) convolved with the short-range kernel K_s;
* coarse level: integer CIC density on the nc^3 coarse mesh (units 2^-27)
  convolved with the long-range kernel K_l.

The particle force is the CIC gather of both fields with the same weights
used for assignment: g = sum_b W_f(x)_b F_s(b) + sum_b W_c(x)_b F_l(b).  It is
the unit-G, unit-mass field g = sum_j K(x - x_j) in fine units; the
cosmological prefactor is applied by the integrator (``dynamics``).

Why no tiles: K_s vanishes for |d| >= r_cut, so the full-mesh convolution
equals the tile-by-tile one of Sec. II whenever the tile's FFT box holds the
tile plus a buffer of r_cut on each side.
"""

import numpy as np

from . import cic, kernels


class ForceOperator:
    """Caches the kernel spectra of one geometry (nc coarse cells per side)."""

    def __init__(self, nc, pos_bytes=1):
        self.nc = nc
        self.nf = kernels.RATIO * nc
        self.pos_bytes = pos_bytes
        self._Kl_hat = None
        self._Ks_hat = None

    # kernel spectra (DFT of the real-space tables)
    def Kl_hat(self):
        if self._Kl_hat is None:
            K = kernels.coarse_kernel_table(self.nc)
            self._Kl_hat = np.stack([np.fft.rfftn(K[c]) for c in range(3)])
        return self._Kl_hat

    def Ks_hat(self):
        if self._Ks_hat is None:
            K = kernels.fine_kernel_table(self.nc)
            self._Ks_hat = np.stack([np.fft.rfftn(K[c]) for c in range(3)])
        return self._Ks_hat

    # densities
    def fine_density(self, Q):
        return cic.deposit(Q, self.nf, 1, self.pos_bytes)

    def coarse_density(self, Q):
        return cic.deposit(Q, self.nc, kernels.RATIO, self.pos_bytes)

    # mesh forces (Eq. 1)
    def fine_field(self, Q):
        """F_s on the fine mesh, [3, z, y, x] float64."""
        U = cic.node_units(1, self.pos_bytes)
        rho = self.fine_density(Q).astype(np.float64) / float((2 * U) ** 3)
        rho_hat = np.fft.rfftn(rho)
        Kh = self.Ks_hat()
        return np.stack([np.fft.irfftn(rho_hat * Kh[c], s=rho.shape, axes=(0, 1, 2)) for c in range(3)])

    def coarse_field(self, Q):
        """F_l on the coarse mesh, [3, z, y, x] float64."""
        U = cic.node_units(kernels.RATIO, self.pos_bytes)
        rho = self.coarse_density(Q).astype(np.float64) / float((2 * U) ** 3)
        rho_hat = np.fft.rfftn(rho)
        Kh = self.Kl_hat()
        return np.stack([np.fft.irfftn(rho_hat * Kh[c], s=rho.shape, axes=(0, 1, 2)) for c in range(3)])

    def particle_force(self, Q, parts=False):
        """g per particle [N, 3] float64 (fine + coarse CIC gathers).

        With ``parts=True`` returns (g_fine, g_coarse) separately.
        """
        Fs = self.fine_field(Q)
        Fl = self.coarse_field(Q)
        gs = np.stack([cic.interpolate(Fs[c], Q, 1, self.pos_bytes) for c in range(3)], axis=1)
        gl = np.stack([cic.interpolate(Fl[c], Q, kernels.RATIO, self.pos_bytes)
                       for c in range(3)], axis=1)
        if parts:
            return gs, gl
        return gs + gl
