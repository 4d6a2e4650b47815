"""FP64 CPU oracle for the CUBE two-level particle-mesh (PMPM) step.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package; only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code with the CUDA library: it is written from the paper (Cheng et al.,
"CUBE -- Towards an Optimal Scaling of Cosmological N-body Simulations",
arXiv:2003.03931), in plain NumPy, float64 unless the method fixes a
precision, step by step in the paper's order, without tiling, fusion or
reordering.

Modules
-------
codec     fixed-point position (Eq. 2) and velocity (Eq. 3) codec, the fast
          arctangent of Eq. 4
cic       integer cloud-in-cell mass assignment / interpolation (Sec. II)
kernels   coarse (long-range) and fine (short-range) force kernels, Eq. 1
force     full-mesh PM-PM force per particle (Sec. II, Eq. 1)
dynamics  kick-drift step and the cell-ordered re-encode (Sec. III-A)
cosmology LambdaCDM background and linear growth (Sec. IV-A.2)
ic        Zel'dovich initial conditions (Sec. IV-A.2)
power     power spectrum (Sec. IV-D)
direct    brute-force convolutions used only to pin the FFT path

Readings of the paper where it is silent are listed in each function's
docstring.  Functions with no independent pin say "parity unpinned"; at the
time of writing there are none.
"""

from . import codec, cic, kernels, force, cosmology, dynamics, ic, power, direct  # noqa: F401
