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

from . import cic, codec, kernels


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
        rho = self.fine_density(Q).astype(np.float64) / float(cic.weight_unit(1, self.pos_bytes))
        rho_hat = np.fft.rfftn(rho)
        Kh = self.Ks_hat()
        return np.stack([np.fft.irfftn(rho_hat * Kh[c], s=rho.shape, axes=(0, 1, 2)) for c in range(3)])

    def coarse_field(self, Q):
        """F_l on the coarse mesh, [3, z, y, x] float64."""
        rho = self.coarse_density(Q).astype(np.float64) / float(cic.weight_unit(kernels.RATIO, self.pos_bytes))
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


# ---------------------------------------------------------------- large boxes
# For boxes whose fine mesh is too large for a float64 FFT here, the same
# force at a few chosen particles.  Both follow the definitions above:
# the coarse density in chunks of particles (integer, so the sum is the
# same), and F_s at the chosen particles' CIC nodes by the direct sum
# F_s(b) = sum_{0 < |d| < r_cut} K_s(d) rho_f(b - d), K_s vanishing beyond
# r_cut (Sec. II), over the fine density of the particles near them.

def coarse_density_chunked(Q, nc, pos_bytes=1, chunk=1 << 22):
    """``cic.deposit`` on the coarse mesh, accumulated chunk by chunk."""
    Q = np.asarray(Q)
    n3 = nc ** 3
    rho = np.zeros(n3, dtype=np.int64)
    for s in range(0, Q.shape[0], chunk):
        node, w = cic.corners(Q[s:s + chunk], nc, kernels.RATIO, pos_bytes)
        # per-chunk node sums stay below 2^53, so float64 bincount is exact
        rho += np.rint(np.bincount(node.ravel(), weights=w.ravel().astype(np.float64),
                                   minlength=n3)).astype(np.int64)
    return rho.reshape(nc, nc, nc)


def coarse_field_from_density(rho_c, nc, pos_bytes=1):
    """F_l on the coarse mesh from a given integer coarse density."""
    rho = rho_c.astype(np.float64) / float(cic.weight_unit(kernels.RATIO, pos_bytes))
    rho_hat = np.fft.rfftn(rho)
    K = kernels.coarse_kernel_table(nc)
    return np.stack([np.fft.irfftn(rho_hat * np.fft.rfftn(K[c]), s=rho.shape, axes=(0, 1, 2))
                     for c in range(3)])


def sampled_fine_force(Q, counts, nc, idx, pos_bytes=1):
    """F_s gathered at particles ``idx`` of a cell-ordered store (codes Q
    [N, 3] in storage order, per-cell ``counts``), [len(idx), 3] float64.

    Every fine node within r_cut of a chosen particle's CIC nodes only
    receives mass from particles at most 8 fine cells (2 coarse cells) away,
    so the 5^3 coarse cells around the particle's own cell hold all of it.
    """
    Q = np.asarray(Q, dtype=np.int64)
    nf = kernels.RATIO * nc
    B = codec.bins_per_cell(pos_bytes)
    unit = float(cic.weight_unit(1, pos_bytes))
    d, Ks = kernels.fine_kernel_values(nc)
    offsets = np.concatenate([[0], np.cumsum(np.asarray(counts, dtype=np.int64))])
    r = np.arange(-2, 3)
    out = np.zeros((len(idx), 3))
    for k, i in enumerate(idx):
        c = Q[i] // B
        cz, cy, cx = np.meshgrid(r + c[2], r + c[1], r + c[0], indexing="ij")
        cells = np.mod(cx, nc) + nc * (np.mod(cy, nc) + nc * np.mod(cz, nc))
        near = np.concatenate([np.arange(offsets[j], offsets[j + 1]) for j in cells.ravel()])
        node, w = cic.corners(Q[near], nf, 1, pos_bytes)
        keys, inv = np.unique(node.ravel(), return_inverse=True)
        mass = np.bincount(inv, weights=w.ravel().astype(np.float64)) / unit
        bnode, bw = cic.corners(Q[i:i + 1], nf, 1, pos_bytes)
        for b, wb in zip(bnode[0], bw[0]):
            bx, by, bz = b % nf, (b // nf) % nf, b // (nf * nf)
            src = (np.mod(bx - d[:, 0], nf) + nf * (np.mod(by - d[:, 1], nf) +
                                                   nf * np.mod(bz - d[:, 2], nf)))
            pos = np.searchsorted(keys, src)
            pos[pos == len(keys)] = 0
            rho = np.where(keys[pos] == src, mass[pos], 0.0)
            out[k] += (wb / unit) * (Ks * rho[:, None]).sum(axis=0)
    return out


def sampled_force(Q, counts, nc, idx, Fl=None, pos_bytes=1):
    """g = F_s + F_l gathered at particles ``idx``; ``Fl`` is the coarse
    field (computed from the chunked coarse density when not given)."""
    Q = np.asarray(Q, dtype=np.int64)
    if Fl is None:
        Fl = coarse_field_from_density(coarse_density_chunked(Q, nc, pos_bytes), nc, pos_bytes)
    gl = np.stack([cic.interpolate(Fl[c], Q[idx], kernels.RATIO, pos_bytes) for c in range(3)], axis=1)
    return sampled_fine_force(Q, counts, nc, idx, pos_bytes) + gl

