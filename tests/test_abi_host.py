"""Host-side checks of the C ABI (no GPU): the library builds and loads,
exports every entry point include/pmpm.h declares, sizes workspaces, rejects
bad configurations, and ships the same Eq. 3 tables as the oracle."""

import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2003_03931_gb300 import _lib, build
    build.build()
    return _lib.load()


def test_header_and_exports(lib):
    from paper_2003_03931_gb300 import _lib
    header = open(os.path.join(ROOT, "include", "pmpm.h")).read()
    declared = set(re.findall(r"\b(pmpm_[a-z_]+)\s*\(", header))
    assert declared == set(_lib.EXPORTS)
    for name in declared:
        assert hasattr(lib, name), name


def test_workspace_bytes_and_validation(lib):
    from paper_2003_03931_gb300.sim import SimConfig, workspace_bytes
    from paper_2003_03931_gb300._lib import PmpmError
    b1 = workspace_bytes(SimConfig(np=32, nc=16))
    b2 = workspace_bytes(SimConfig(np=128, nc=64))
    b3 = workspace_bytes(SimConfig(np=512, nc=256))
    assert 0 < b1 < b2 < b3
    # the persistent particle store is 2 x 6 bytes per particle plus cell fields
    assert b3 > 2 * 6 * 512 ** 3
    # 2-byte positions: 9 bytes per particle in each store buffer
    assert workspace_bytes(SimConfig(np=512, nc=256, pos_bytes=2)) - b3 == 2 * 3 * 512 ** 3
    for bad in (dict(np=30, nc=16), dict(np=32, nc=12), dict(np=32, nc=16, tile_max=6),
                dict(np=32, nc=16, buffer=4), dict(np=32, nc=16, pos_bytes=3),
                dict(np=32, nc=16, pos_bytes=2, lowmem=True),
                dict(np=32, nc=16, a_init=0.5, a_final=0.1)):
        with pytest.raises(PmpmError):
            workspace_bytes(SimConfig(**bad))


def test_codec_tables_match_oracle(lib):
    from oracle import codec
    from paper_2003_03931_gb300.sim import codec_tables
    T, E = codec_tables()
    To, Eo = codec.velocity_tables()
    np.testing.assert_array_equal(T, To)
    np.testing.assert_array_equal(E, Eo)


def test_init_without_device_fails_cleanly(lib):
    # no GPU here: pmpm_init must return an error code, not crash
    from paper_2003_03931_gb300 import _lib
    from paper_2003_03931_gb300.sim import SimConfig
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    c = SimConfig(np=16, nc=8).to_c()
    h = ctypes.c_void_p()
    rc = lib.pmpm_init(ctypes.byref(c), ctypes.c_void_p(256), 1 << 30, None, ctypes.byref(h))
    assert rc != _lib.PMPM_OK


def test_lowmem_workspace_fits_2048_cubed(lib):
    # the low-memory step keeps only the new momenta (12 B per particle) and
    # no codes; 2048^3 particles (nc = 1024) need about 31 bytes per
    # particle, inside one GB300's HBM (284,208 MiB)
    from paper_2003_03931_gb300.sim import SimConfig, workspace_bytes
    from paper_2003_03931_gb300._lib import PmpmError
    big = SimConfig(np=2048, nc=1024, n_steps=20, lowmem=True)
    b = workspace_bytes(big)
    assert b < 265e9
    assert b / 2048 ** 3 < 31
    assert workspace_bytes(SimConfig(np=2048, nc=1024, n_steps=20)) > 2.5 * b
    # two stores (2 x 6 B) and the new momenta (or the float32 IC field,
    # 12 B) must all be there, with the cell arrays (8 particles per cell)
    assert b > (12 + 12) * 2048 ** 3 + 2 * 24 * 1024 ** 3
    with pytest.raises(PmpmError):
        c = SimConfig(np=32, nc=16)
        cc = c.to_c()
        cc.flags = 6
        import ctypes
        from paper_2003_03931_gb300 import _lib
        out = ctypes.c_size_t(0)
        _lib.check(lib.pmpm_workspace_bytes(ctypes.byref(cc), ctypes.byref(out)))


@pytest.mark.parametrize("np_,nc", [(2048, 1024), (256, 128), (64, 16), (32, 32), (16, 32)])
def test_lowmem_workspace_regions(lib, np_, nc):
    # the low-memory layout: two stores (each max(6N, 36C) bytes: the next
    # store's space also holds the step's momentum sums, 24 B/cell, and
    # F_l, 12 B/cell) with their counts, offsets and v_c; the slot counters;
    # one region taken in turn by the coarse mesh (4 x 8 B/cell), the kept
    # momenta or the IC displacement field (12 B/particle), the P(k) mesh and
    # the force-table scratch; and small tables (the coarse Green table, 16 B
    # per folded wavenumber, the largest).  No per-particle codes.
    from paper_2003_03931_gb300.sim import SimConfig, workspace_bytes

    def al(x):
        return (x + 255) // 256 * 256

    N, C = np_ ** 3, nc ** 3
    h = nc // 2 + 1
    store = al(max(6 * N, al(24 * C) + 12 * C))
    pair = 2 * (store + al(4 * C) + al(8 * (C + 1)) + al(12 * C))
    pk = min(4 * nc, 512)
    green = 343 * 8 + 1331 * 8 + 512 + 16 * C + 4 * h ** 3
    U = max(12 * N, 4 * al(8 * C), 16 * pk ** 3 + 512, green)
    big = pair + al(4 * C) + U
    b = workspace_bytes(SimConfig(np=np_, nc=nc, n_steps=20, lowmem=True))
    small = b - big
    assert 16 * h ** 3 <= small <= 16 * h ** 3 + (8 << 20), (b, big)


def test_fma_probe_rejects_bad_arguments(lib):
    # argument checks come before any CUDA call, so they run without a GPU
    f, ms = ctypes.c_double(), ctypes.c_float()
    buf = ctypes.c_void_p(4096)   # never dereferenced on these paths
    for args in ((None, 256, None, 10), (buf, 255, None, 10), (buf, 0, None, 10), (buf, 256, None, 0)):
        assert lib.pmpm_probe_fma(*args, ctypes.byref(f), ctypes.byref(ms)) == -1
    assert lib.pmpm_probe_fma(buf, 256, None, 10, None, ctypes.byref(ms)) == -1


def test_binding_fails_loudly_without_the_library(monkeypatch, tmp_path):
    # no fallback: without libpmpm.so the binding raises instead of running
    # anything else
    from paper_2003_03931_gb300 import _lib
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "missing" / "libpmpm.so"))
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(ImportError):
        _lib.load()


def test_step_factors_match_the_oracle(lib):
    # the library's float64 schedule factors (its own quadrature of the
    # background, Sec. IV-A.2) against the oracle's (scipy), EdS and LambdaCDM
    import math

    from oracle import cosmology, dynamics
    from paper_2003_03931_gb300.sim import SimConfig, step_factors
    for om, ol, ai in ((0.0, 0.0, 0.02), (0.258, 0.742, 0.01), (0.3, 0.0, 0.05)):
        cfg = SimConfig(np=32, nc=16, a_init=ai, a_final=1.0, n_steps=12, omega_m=om, omega_l=ol)
        cos = cosmology.Cosmology(om, ol) if om else None
        for n in range(12):
            k, d, pf = step_factors(cfg, n)
            ko, do = dynamics.step_factors(ai, 1.0, 12, n, 32 ** 3, 64, cos)
            assert abs(k / ko - 1) < 1e-12 and abs(d / do - 1) < 1e-12, (om, n, k, ko, d, do)
        ref = cos.ic_momentum_factor(ai) if cos else math.sqrt(ai)
        assert abs(pf / ref - 1) < 1e-11, (om, pf, ref)
    from paper_2003_03931_gb300._lib import PMPM_EINVAL, PmpmError
    for om, ol in ((0.0, 0.7), (-0.1, 0.0), (0.1, 5.0)):
        with pytest.raises(PmpmError) as e:
            step_factors(SimConfig(np=32, nc=16, omega_m=om, omega_l=ol), 0)
        assert e.value.code == PMPM_EINVAL
