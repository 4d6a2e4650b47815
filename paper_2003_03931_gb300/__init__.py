"""GB300-native two-level particle-mesh (PM-PM) step of CUBE (arXiv:2003.03931).

The compute lives in libpmpm.so (CUDA, sm_103a) behind the C ABI of
include/pmpm.h; this package holds its ctypes binding (``_lib``), a small
simulation handle (``sim``), the seeded input generators shared with the
tests (``synth``) and the build script (``build``).
"""

__all__ = ["sim", "synth", "build"]
