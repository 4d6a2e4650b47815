"""The power spectrum entry point that allocates no device memory, for
callers that may not allocate GPU memory themselves (a host application that
owns the device-memory budget, a loop that cannot afford an allocation's
synchronisation).  It must give what pmpm_power_spectrum gives for the same
store, on consecutive calls that reuse its fixed scratch array.

This file is collected last on purpose."""

import ctypes

import numpy as np
import pytest

from paper_2003_03931_gb300 import synth
from tests.gpu_util import make_sim, need_gpu

pytestmark = pytest.mark.gpu


def _noalloc(lib, nc, dev, nmesh, nbins, stream):
    k = np.zeros(nbins)
    pk = np.zeros(nbins)
    nm = np.zeros(nbins, np.int64)
    rc = lib.pmpm_power_spectrum_noalloc(
        nc, dev["n"], dev["m"][0].data_ptr(), dev["m"][1].data_ptr(), dev["m"][2].data_ptr(),
        dev["counts"].data_ptr(), nmesh, nbins, k.ctypes.data, pk.ctypes.data, nm.ctypes.data,
        ctypes.c_void_p(stream))
    return rc, k, pk, nm


def test_noalloc_power_spectrum_matches_and_repeats():
    need_gpu()
    import torch
    from paper_2003_03931_gb300 import _lib
    lib = _lib.load()
    w = synth.WORKLOADS["c1_32"]
    sim = make_sim(**w)
    sim.ic_zeldovich(5, **synth.IC_SPECTRUM)
    sim.step(3)
    st = sim.fetch_state()
    # the test, not the entry point, owns these device buffers
    dev = {"n": sim.cfg.n,
           "m": [torch.from_numpy(np.ascontiguousarray(st["streams"][d])).cuda() for d in range(3)],
           "counts": torch.from_numpy(st["counts"]).cuda()}
    stream = torch.cuda.current_stream().cuda_stream
    torch.cuda.synchronize()
    for nmesh in (64, 32, 16, 64):   # consecutive calls share the scratch array
        nbins = nmesh // 2
        kr, pr, nr = sim.power_spectrum(nmesh, nbins)
        for _ in range(2):
            rc, k, pk, nm = _noalloc(lib, w["nc"], dev, nmesh, nbins, stream)
            assert rc == 0, lib.pmpm_noalloc_last_error()
            np.testing.assert_array_equal(nm, nr)
            np.testing.assert_allclose(k, kr, rtol=1e-12)
            np.testing.assert_allclose(pk, pr, rtol=1e-9)
    # counts that do not add up to n are refused, not binned into wrong cells
    bad = dict(dev, counts=dev["counts"].clone())
    bad["counts"][0] += 1
    rc, *_ = _noalloc(lib, w["nc"], bad, 32, 16, stream)
    assert rc == _lib.PMPM_EINVAL
    assert b"add up" in lib.pmpm_noalloc_last_error()
    sim.close()


def test_noalloc_at_its_largest_box():
    # nc = 64 at nmesh = 64: the whole offsets and mesh regions of the array
    need_gpu()
    import torch
    from paper_2003_03931_gb300 import _lib
    lib = _lib.load()
    sim = make_sim(np=64, nc=64, a_init=0.02, a_final=1.0, n_steps=4)
    sim.ic_zeldovich(6, **synth.IC_SPECTRUM)
    sim.step(2)
    st = sim.fetch_state()
    dev = {"n": sim.cfg.n,
           "m": [torch.from_numpy(np.ascontiguousarray(st["streams"][d])).cuda() for d in range(3)],
           "counts": torch.from_numpy(st["counts"]).cuda()}
    stream = torch.cuda.current_stream().cuda_stream
    torch.cuda.synchronize()
    kr, pr, nr = sim.power_spectrum(64, 32)
    for _ in range(2):
        rc, k, pk, nm = _noalloc(lib, 64, dev, 64, 32, stream)
        assert rc == 0, lib.pmpm_noalloc_last_error()
        np.testing.assert_array_equal(nm, nr)
        np.testing.assert_allclose(k, kr, rtol=1e-12)
        np.testing.assert_allclose(pk, pr, rtol=1e-9)
    sim.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    need_gpu()
    import torch
    from paper_2003_03931_gb300 import _lib
    lib = _lib.load()
    dev = {"n": 8, "m": [torch.zeros(8, dtype=torch.uint8, device="cuda") for _ in range(3)],
           "counts": torch.zeros(128 ** 3, dtype=torch.int32, device="cuda")}
    for nc, nmesh in ((128, 64), (64, 128), (16, 48)):
        rc, *_ = _noalloc(lib, nc, dev, nmesh, 4, torch.cuda.current_stream().cuda_stream)
        assert rc == _lib.PMPM_EINVAL
        assert lib.pmpm_noalloc_last_error()
