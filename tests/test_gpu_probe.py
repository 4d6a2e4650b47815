"""The FP32 FMA probe (pmpm_probe_fma) on the GPU: its rate is a plausible
fraction of the lanes x clock figure, and its output words are finite."""

import ctypes

import pytest

from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu


def test_fma_probe_measures_a_plausible_peak():
    need_gpu()
    import torch

    import bench
    from paper_2003_03931_gb300 import _lib
    dev = torch.device("cuda:0")
    tf = bench.probe_fp32_tflops(dev, repeats=3, iters=1 << 12)
    props = torch.cuda.get_device_properties(dev)
    # 128 FP32 lanes per SM, 2 FLOP per FMA, at most ~2.1 GHz
    ceiling = props.multi_processor_count * 128 * 2 * 2.2e9 / 1e12
    assert 0.2 * ceiling < tf < ceiling, (tf, ceiling)
    out = torch.empty(256 * 4, device=dev)
    f, ms = ctypes.c_double(), ctypes.c_float()
    lib = _lib.load()
    assert lib.pmpm_probe_fma(ctypes.c_void_p(out.data_ptr()), out.numel(), None, 100,
                              ctypes.byref(f), ctypes.byref(ms)) == 0
    assert torch.isfinite(out).all() and f.value == 2 * 8 * 100 * out.numel()
