"""Power spectrum of the particle density (Sec. IV-D).

Test infrastructure only (see ``oracle/__init__``).

Sec. IV-D defines delta = rho / rho_bar - 1 from the CIC density and the
power spectrum through <delta(k)^* delta(k')> = (2 pi)^3 P(k) delta_D(k - k'),
reported also as Delta^2(k) = k^3 P(k) / (2 pi^2).  On a periodic nmesh^3
mesh of side L this is P(k) = L^3 / nmesh^6 |DFT(delta)|^2.  Reading for the
binning: shell j = round(|n|) for integer frequency vectors n, j = 1..nbins;
each bin reports the mean |k| of its modes, the mean P and the mode count.  No
CIC-window deconvolution and no shot-noise subtraction (the paper states
neither).
"""

import numpy as np

from . import cic


def density_contrast(Q, nmesh, nf, pos_bytes=1):
    """delta on the nmesh^3 mesh from the integer CIC density."""
    h = nf // nmesh
    if h * nmesh != nf:
        raise ValueError("nmesh must divide the fine mesh")
    rho = cic.deposit(Q, nmesh, h, pos_bytes).astype(np.float64)
    return rho / rho.mean() - 1.0


def shells(nmesh):
    """(shell index j, |n|) of every mode of the full nmesh^3 DFT grid."""
    n = np.rint(np.fft.fftfreq(nmesh) * nmesh)
    nz_, ny_, nx_ = np.meshgrid(n, n, n, indexing="ij")
    r = np.sqrt(nx_ * nx_ + ny_ * ny_ + nz_ * nz_)
    return np.rint(r).astype(np.int64), r


def spectrum_from_delta(delta, L, nbins):
    nmesh = delta.shape[0]
    dk = np.fft.fftn(delta)
    P = (L ** 3 / float(nmesh) ** 6) * (dk.real ** 2 + dk.imag ** 2)
    j, r = shells(nmesh)
    k = 2 * np.pi * r / L
    sel = (j >= 1) & (j <= nbins)
    cnt = np.bincount(j[sel], minlength=nbins + 1)[1:]
    ksum = np.bincount(j[sel], weights=k[sel], minlength=nbins + 1)[1:]
    psum = np.bincount(j[sel], weights=P[sel], minlength=nbins + 1)[1:]
    with np.errstate(invalid="ignore", divide="ignore"):
        kmean = np.where(cnt > 0, ksum / np.maximum(cnt, 1), 0.0)
        pmean = np.where(cnt > 0, psum / np.maximum(cnt, 1), 0.0)
    return kmean, pmean, cnt.astype(np.int64)


def power_spectrum(Q, nmesh, nbins, nf, pos_bytes=1):
    """(k_j, P_j, nmodes_j) for j = 1..nbins (box side L = nf fine cells)."""
    delta = density_contrast(Q, nmesh, nf, pos_bytes)
    return spectrum_from_delta(delta, float(nf), nbins)


def dimensionless(k, P):
    """Delta^2(k) = k^3 P(k) / (2 pi^2) (Sec. IV-D)."""
    return np.asarray(k) ** 3 * np.asarray(P) / (2 * np.pi ** 2)
