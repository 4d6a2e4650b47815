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


def test_pinned_state_bytes_round_each_buffer_up():
    # the end-to-end leg pins the store, counts and v_c; the pinned-memory
    # cache rounds each to a power of two (2048^3: 64 + 4 + 16 GiB)
    from paper_2003_03931_gb300.sim import SimConfig
    big = SimConfig(np=2048, nc=1024, n_steps=20, lowmem=True)
    assert bench.pinned_state_bytes(big) == (64 + 4 + 16) << 30
    small = SimConfig(np=64, nc=32, n_steps=20)
    n, c = 64 ** 3, 32 ** 3
    got = bench.pinned_state_bytes(small)
    assert 6 * n + 16 * c <= got < 2 * (6 * n + 16 * c)


def test_host_memory_available_is_positive_or_unknown():
    avail = bench.host_memory_available()
    assert avail is None or avail > 0
