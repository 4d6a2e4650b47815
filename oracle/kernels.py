"""Long- and short-range force kernels of the PM-PM split (Sec. II, Eq. 1).

Test infrastructure only (see ``oracle/__init__``).

Sec. II splits gravity into a long-range part computed on a 4x coarser mesh
and a short-range part with a cutoff, computed on the fine mesh; it defers
force matching to its references.  Reading used here (the PMFAST / CUBEP3M
idea those references describe):

* Unit-G pair kernel K(r) = -r / |r|^3 (force on a particle at separation r
  from a unit source; lengths in fine cells).  In the periodic box the
  gravity F_G that the long-range part must reproduce is the periodic pair
  force: a unit mass, all its images and the removed mean density, summed
  by the Ewald split (screened real-space images plus a Gaussian-damped
  Fourier sum).  A nearest-image truncated 1/r^2 under-forces box-scale
  modes by ~15%, which the linear-growth pin detects.
* Coarse kernel K_l on the nc^3 coarse mesh: the periodic pair force at the
  coarse separations 4D (fine units); zero at D = 0.  The table is exactly
  odd (the periodic force is odd and vanishes along an axis at L/2).
* Force matching A(d): the coarse-mesh force between two fine-cell centres a
  fine separation d apart, averaged over the 64 fine-cell centres s inside one
  coarse cell: A(d) = (1/64) sum_s sum_{a,b} W(s)_a W(s+d)_b K_l(b - a), with
  W the coarse CIC weights (nodes at coarse-cell centres).
* Fine kernel: K_s(d) = K_per(d) - A(d) for integer 0 < |d| < r_cut, else 0,
  with K_per the periodic pair force and
  r_cut equal to the 6-fine-cell tile buffer of Sec. IV-A.2.  So on average
  the fine and coarse parts together give K(d) inside the cutoff and the
  coarse part alone beyond it, F_s(r >= r_cut) = 0 as Sec. II requires.
"""

import functools

import numpy as np

R_CUT = 6  # fine cells; the tile buffer width of Sec. IV-A.2 (6 cells on each side)
RATIO = 4  # coarse / fine cell size, Sec. II


def pair_kernel(r):
    """K(r) = -r/|r|^3 for r [..., 3] float64, with K(0) = 0."""
    r = np.asarray(r, dtype=np.float64)
    r2 = (r * r).sum(axis=-1, keepdims=True)
    with np.errstate(divide="ignore", invalid="ignore"):
        out = -r / (r2 * np.sqrt(r2))
    out[np.broadcast_to(r2 == 0, out.shape)] = 0.0
    return out


# Ewald split: e^(-k^2/4 alpha^2) < e^-38 beyond the Fourier cutoff k_max,
# erfc-screened real-space terms negligible beyond alpha r = 6.5
EWALD_K_EXP = 38.0
EWALD_R_CUT = 6.5


def ewald_alpha(L, h_max):
    """Screening alpha for a Fourier cutoff |h| <= h_max (k = 2 pi h / L)."""
    return (2 * np.pi * h_max / L) / (2 * np.sqrt(EWALD_K_EXP))


def _ewald_images(L, alpha):
    n_img = int(np.ceil(EWALD_R_CUT / alpha / L + 0.5))
    r = np.arange(-n_img, n_img + 1)
    nz, ny, nx = np.meshgrid(r, r, r, indexing="ij")
    return L * np.stack([nx.ravel(), ny.ravel(), nz.ravel()], axis=1).astype(np.float64)


def _ewald_hvectors(h_max):
    r = np.arange(-h_max, h_max + 1)
    hz, hy, hx = np.meshgrid(r, r, r, indexing="ij")
    h = np.stack([hx.ravel(), hy.ravel(), hz.ravel()], axis=1)
    h2 = (h * h).sum(axis=1)
    return h[(h2 > 0) & (h2 <= h_max * h_max)]


def _ewald_real(x, L, alpha, skip_origin):
    """Real-space Ewald sum over periodic images, [M, 3]."""
    from math import sqrt, pi
    from scipy.special import erfc
    x = np.asarray(x, dtype=np.float64).reshape(-1, 3)
    out = np.zeros_like(x)
    rs = EWALD_R_CUT / alpha
    for shift in _ewald_images(L, alpha):
        rn = x + shift[None, :]
        r = np.sqrt((rn * rn).sum(axis=1))
        use = r <= rs
        if skip_origin:
            use &= r > 0
        if not use.any():
            continue
        rr = r[use]
        ar = alpha * rr
        screen = erfc(ar) + 2.0 / sqrt(pi) * ar * np.exp(-ar * ar)
        out[use] -= rn[use] / (rr ** 3)[:, None] * screen[:, None]
    return out


def periodic_pair_kernel(x, L, h_max=8):
    """Periodic (Ewald) unit-G pair force at separations x [..., 3]: the force
    of a unit mass and all its images, with the mean density removed, on a
    particle at separation x; zero at x = 0.  Direct evaluation."""
    x = np.asarray(x, dtype=np.float64)
    shape = x.shape
    xf = x.reshape(-1, 3)
    alpha = ewald_alpha(L, h_max)
    out = _ewald_real(xf, L, alpha, skip_origin=True)
    h = _ewald_hvectors(h_max).astype(np.float64)
    k = 2 * np.pi * h / L
    k2 = (k * k).sum(axis=1)
    coef = (4 * np.pi / L ** 3) * np.exp(-k2 / (4 * alpha * alpha)) / k2
    for lo in range(0, xf.shape[0], 256):
        xs = xf[lo:lo + 256]
        s = np.sin(xs @ k.T)                       # [m, nh]
        out[lo:lo + 256] -= (s * coef[None, :]) @ k
    zero = (xf * xf).sum(axis=1) == 0
    out[zero] = 0.0
    return out.reshape(shape)


def nearest_image(n):
    """Signed integer offsets of an n-periodic axis, in [-n/2, n/2)."""
    i = np.arange(n)
    return ((i + n // 2) % n) - n // 2


@functools.lru_cache(maxsize=8)
def coarse_kernel_table(nc):
    """K_l(D) on the nc^3 coarse mesh, array [3, z, y, x] float64 (fine units).

    K_l is the periodic (Ewald) pair force sampled at the coarse-cell
    separations 4D: a Fourier part band-limited to |h| <= h_max < nc/2,
    sampled exactly by an inverse DFT on the mesh, plus the real-space
    screened sum over images.
    """
    L = float(RATIO * nc)
    h_max = min(32, nc // 2 - 1)
    alpha = ewald_alpha(L, h_max)
    # Fourier part: T(D) = sum_h C(h) e^{2 pi i h.D / nc},
    # C(h) = (4 pi i / L^3) (k / k^2) e^{-k^2 / 4 alpha^2}
    h = _ewald_hvectors(h_max)
    k = 2 * np.pi * h.astype(np.float64) / L
    k2 = (k * k).sum(axis=1)
    g = np.exp(-k2 / (4 * alpha * alpha)) / k2
    table = np.zeros((3, nc, nc, nc))
    idx = (np.mod(h[:, 2], nc), np.mod(h[:, 1], nc), np.mod(h[:, 0], nc))
    for c in range(3):
        C = np.zeros((nc, nc, nc), dtype=np.complex128)
        C[idx] = (4j * np.pi / L ** 3) * k[:, c] * g
        table[c] = (np.fft.ifftn(C) * nc ** 3).real
    # real-space part at every lattice separation (nearest image of D)
    D = nearest_image(nc)
    Dz, Dy, Dx = np.meshgrid(D, D, D, indexing="ij")
    x = RATIO * np.stack([Dx.ravel(), Dy.ravel(), Dz.ravel()], axis=1).astype(np.float64)
    real = _ewald_real(x, L, alpha, skip_origin=True)
    table += np.moveaxis(real.reshape(nc, nc, nc, 3), -1, 0)
    # the periodic force is odd; remove the rounding-level asymmetry so the
    # table is exactly odd (zero self-force and momentum conservation then
    # hold to rounding of the convolution only)
    neg = (-np.arange(nc)) % nc
    table = 0.5 * (table - table[:, neg][:, :, neg][:, :, :, neg])
    table[:, 0, 0, 0] = 0.0
    table.setflags(write=False)
    return table


def _coarse_weights_1d(pos):
    """Coarse CIC weights of a point at `pos` (fine units, relative to the
    left edge of coarse cell 0); nodes at 4a + 2.  Returns (a0, w0, w1)."""
    t = (np.asarray(pos, dtype=np.float64) - RATIO / 2) / RATIO
    a0 = np.floor(t).astype(np.int64)
    w1 = t - a0
    return a0, 1.0 - w1, w1


def matching_force(d, nc):
    """A(d): sub-cell-averaged coarse-mesh pair force, float64 [..., 3].

    `d` is an integer array [..., 3] of fine separations; the coarse pair
    force K_l(b - a) is read from the periodic table of an nc^3 box.
    """
    table = coarse_kernel_table(nc)
    d = np.asarray(d, dtype=np.int64)
    shape = d.shape[:-1]
    dflat = d.reshape(-1, 3)
    out = np.zeros((dflat.shape[0], 3))
    sub = np.arange(RATIO) + 0.5  # fine-cell centres inside one coarse cell
    for sx in sub:
        for sy in sub:
            for sz in sub:
                s = np.array([sx, sy, sz])
                a0, aw0, aw1 = _coarse_weights_1d(s)
                b0, bw0, bw1 = _coarse_weights_1d(s[None, :] + dflat)
                for ax in (0, 1):
                    for ay in (0, 1):
                        for az in (0, 1):
                            wa = ((aw1[0] if ax else aw0[0]) * (aw1[1] if ay else aw0[1])
                                  * (aw1[2] if az else aw0[2]))
                            a = a0 + np.array([ax, ay, az])
                            for bx in (0, 1):
                                for by in (0, 1):
                                    for bz in (0, 1):
                                        wb = ((bw1[:, 0] if bx else bw0[:, 0])
                                              * (bw1[:, 1] if by else bw0[:, 1])
                                              * (bw1[:, 2] if bz else bw0[:, 2]))
                                        b = b0 + np.array([bx, by, bz])
                                        D = np.mod(b - a[None, :], nc)
                                        K = table[:, D[:, 2], D[:, 1], D[:, 0]].T
                                        out += (wa * wb)[:, None] * K
    out /= RATIO ** 3
    return out.reshape(shape + (3,))


def fine_kernel_support():
    """Integer offsets d with 0 < |d| < r_cut, shape [n, 3]."""
    r = np.arange(-R_CUT + 1, R_CUT)
    dz, dy, dx = np.meshgrid(r, r, r, indexing="ij")
    d = np.stack([dx.ravel(), dy.ravel(), dz.ravel()], axis=1)
    r2 = (d * d).sum(axis=1)
    keep = (r2 > 0) & (r2 < R_CUT * R_CUT)
    return d[keep]


def fine_kernel_values(nc):
    """(d [n, 3], K_s(d) [n, 3]) on the support 0 < |d| < r_cut of a box of
    nc coarse cells: the periodic pair force minus the matching force."""
    d = fine_kernel_support()
    Ks = periodic_pair_kernel(d.astype(np.float64), float(RATIO * nc)) - matching_force(d, nc)
    return d, Ks


def fine_kernel_table(nc, mesh=None):
    """K_s on a periodic mesh^3 fine mesh (default the whole box, 4 nc),
    array [3, z, y, x] float64."""
    nf = RATIO * nc if mesh is None else mesh
    if nf < 2 * R_CUT:
        raise ValueError("fine mesh too small for the kernel support")
    d, Ks = fine_kernel_values(nc)
    table = np.zeros((3, nf, nf, nf))
    ix = np.mod(d[:, 0], nf)
    iy = np.mod(d[:, 1], nf)
    iz = np.mod(d[:, 2], nf)
    for c in range(3):
        table[c, iz, iy, ix] = Ks[:, c]
    return table
