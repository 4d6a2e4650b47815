"""Host-side checks of the serving layer (no GPU): the arena allocator
against a model of first fit with merging, the ctypes structs against the C
ABI's sizes, engine argument checks, and the seeded mixed request stream."""

import ctypes

import numpy as np
import pytest


@pytest.fixture(scope="module")
def lib():
    from paper_2003_03931_gb300 import _lib, build
    build.build()
    return _lib.load()


def test_binding_structs_match_c_sizes(lib):
    from paper_2003_03931_gb300 import _lib
    n = len(_lib.ABI_STRUCTS)
    sizes = (ctypes.c_int64 * n)()
    assert lib.pmpm_abi_sizes(sizes, n) == 0
    assert list(sizes) == [ctypes.sizeof(s) for s in _lib.ABI_STRUCTS]
    assert lib.pmpm_abi_sizes(sizes, n - 1) == _lib.PMPM_EINVAL


class ModelArena:
    """First fit in address order over 256-byte units; merged free list."""

    def __init__(self, size):
        self.size = size // 256 * 256
        self.free = [(0, self.size)]
        self.live = {}

    def alloc(self, b):
        if b > self.size:
            return None
        b = max(256, -(-b // 256) * 256)
        for i, (o, ln) in enumerate(self.free):
            if ln >= b:
                self.free[i:i + 1] = [(o + b, ln - b)] if ln > b else []
                self.live[o] = b
                return o
        return None

    def release(self, o):
        ln = self.live.pop(o)
        self.free.append((o, ln))
        self.free.sort()
        merged = []
        for a, l in self.free:
            if merged and merged[-1][0] + merged[-1][1] == a:
                merged[-1] = (merged[-1][0], merged[-1][1] + l)
            else:
                merged.append((a, l))
        self.free = merged


def test_arena_matches_first_fit_model(lib):
    from paper_2003_03931_gb300 import _lib
    rng = np.random.default_rng(3)
    for size in (1 << 20, 12345678):
        h = ctypes.c_void_p()
        assert lib.pmpm_arena_create(size, ctypes.byref(h)) == 0
        model = ModelArena(size)
        live = []
        for it in range(3000):
            if live and rng.random() < 0.45:
                o = live.pop(int(rng.integers(len(live))))
                assert lib.pmpm_arena_free(h, o) == 0
                model.release(o)
            else:
                b = int(rng.choice([0, 1, 255, 256, 257, int(rng.integers(1, size // 8))]))
                off = ctypes.c_size_t()
                rc = lib.pmpm_arena_alloc(h, b, ctypes.byref(off))
                mo = model.alloc(b)
                if mo is None:
                    assert rc == _lib.PMPM_ENOMEM
                else:
                    assert rc == 0 and off.value == mo and off.value % 256 == 0
                    live.append(off.value)
            used, largest, nlive = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_int64()
            assert lib.pmpm_arena_stats(h, ctypes.byref(used), ctypes.byref(largest),
                                        ctypes.byref(nlive)) == 0
            assert used.value == sum(model.live.values())
            assert largest.value == max([ln for _, ln in model.free], default=0)
            assert nlive.value == len(live)
        # double free and unknown offsets are refused; everything freed merges back
        if live:
            o = live[0]
            assert lib.pmpm_arena_free(h, o + 256) == _lib.PMPM_EINVAL or (o + 256) in live
        for o in live:
            assert lib.pmpm_arena_free(h, o) == 0
        assert lib.pmpm_arena_free(h, 0) == _lib.PMPM_EINVAL
        largest = ctypes.c_size_t()
        lib.pmpm_arena_stats(h, None, ctypes.byref(largest), None)
        assert largest.value == size // 256 * 256
        lib.pmpm_arena_destroy(h)
    h = ctypes.c_void_p()
    assert lib.pmpm_arena_create(100, ctypes.byref(h)) == _lib.PMPM_EINVAL


def test_batch_create_rejects_bad_arguments(lib):
    from paper_2003_03931_gb300 import _lib
    h = ctypes.c_void_p()
    good = _lib.BatchConfig(4, 1, 0, 1, 2, 2)
    assert lib.pmpm_batch_create(ctypes.byref(good), None, 1 << 20, ctypes.byref(h)) == _lib.PMPM_EINVAL
    for bad in (_lib.BatchConfig(0, 1, 0, 1, 2, 2), _lib.BatchConfig(4, 1, 0, 1, 0, 2),
                _lib.BatchConfig(4, 1, 0, 1, 2, 0), _lib.BatchConfig(4, 1, 0, 3, 2, 2),
                _lib.BatchConfig(4, 1, 0, -1, 2, 2), _lib.BatchConfig(4, 1, 0, 1, 2, 2, -1, 1),
                _lib.BatchConfig(4, 1, 0, 1, 2, 2, 256, -1)):
        assert lib.pmpm_batch_create(ctypes.byref(bad), ctypes.c_void_p(1 << 20), 1 << 20,
                                     ctypes.byref(h)) == _lib.PMPM_EINVAL
        assert b"max_active" in lib.pmpm_batch_last_error(None)
    # misaligned arena
    assert lib.pmpm_batch_create(ctypes.byref(good), ctypes.c_void_p((1 << 20) + 8), 1 << 20,
                                 ctypes.byref(h)) == _lib.PMPM_EINVAL


def test_mixed_request_stream():
    from paper_2003_03931_gb300.serve import MIX_SIZES, mixed_requests, with_arrivals
    a = mixed_requests(4000, seed=5)
    b = mixed_requests(4000, seed=5)
    assert a == b
    assert a != mixed_requests(4000, seed=6)
    sizes = np.array([r.np for r in a])
    frac = [(sizes == s).mean() for s in MIX_SIZES]
    np.testing.assert_allclose(frac, [0.4, 0.3, 0.2, 0.1], atol=0.03)
    steps = np.array([r.n_steps for r in a])
    assert steps.min() == 10 and steps.max() == 40
    slopes = np.array([r.slope for r in a])
    assert slopes.min() >= -2 and slopes.max() <= -1
    assert all(r.nc == r.np // 2 and r.arrival == 0 for r in a)
    assert len({r.seed for r in a}) == len(a)
    t = np.array([r.arrival for r in with_arrivals(a, rate=50.0, seed=1)])
    assert t[0] == 0 and np.all(np.diff(t) > 0)
    # Poisson process: mean gap 1/rate, exponential gaps (cv ~ 1)
    g = np.diff(t)
    assert abs(g.mean() * 50 - 1) < 0.05 and abs(g.std() / g.mean() - 1) < 0.06


def test_latency_summary():
    from paper_2003_03931_gb300.serve import Request, Result, latency_summary
    req = Request(np=32, nc=16, n_steps=10, seed=1)
    res = [Result(i, 0, float(i), float(i), float(i) + 1 + i % 3, 1.0, 1.0, 100, req,
                  None, None, None) for i in range(100)]
    res.append(Result(100, -3, 0.0, 0.0, 0.5, 0, 0, 0, req, None, None, None))
    s = latency_summary(res)
    assert s["requests"] == 101 and s["failed"] == 1
    lat = np.array([1 + i % 3 for i in range(100)], float)
    assert s["p50_s"] == np.percentile(lat, 50) and s["p99_s"] == np.percentile(lat, 99)
    assert s["makespan_s"] == max(i + 1 + i % 3 for i in range(100))
    assert s["particle_steps_per_s"] == 100 * 100 / s["makespan_s"]
