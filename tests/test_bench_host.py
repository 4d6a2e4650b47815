"""Host logic of bench.py: the kernel-source hash that keys the recorded
tile-pass traffic, and the FP32 roofline peak."""

import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _hash_of(tmp_path, text):
    p = tmp_path / "k.cu"
    p.write_text(text)
    old = bench.ROOT
    bench.ROOT = str(tmp_path)
    try:
        return bench.source_hash(["k.cu"])
    finally:
        bench.ROOT = old


def test_source_hash_ignores_comments_but_not_code(tmp_path):
    base = "int f(int x) {\n    return x + 1;   // add one\n}\n"
    same = "/* a block\n   comment */\nint f(int x) {\n  return x + 1;\n}  // trailing\n"
    other = "int f(int x) {\n    return x + 2;\n}\n"
    assert _hash_of(tmp_path, base) == _hash_of(tmp_path, same)
    assert _hash_of(tmp_path, base) != _hash_of(tmp_path, other)


def test_fp32_peak_is_lanes_times_clock():
    # 152 SMs x 128 lanes x 2 FLOP x 2070 MHz
    assert abs(bench.fp32_peak_tflops(2070.0) - 80.54784) < 1e-6
