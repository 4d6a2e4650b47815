"""The autotuner on the GPU: it times both tile edges and a small grid of
serving-engine settings through the public API, keeps the fastest, and
answers the second call from its cache."""

import pytest

from paper_2003_03931_gb300 import autotune, serve
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu


def test_tile_edge_is_measured_and_cached(tmp_path):
    need_gpu()
    cache = str(tmp_path / "tune.json")
    out = autotune.tune_tile(32, 32, cache_path=cache, repeats=1, steps=2)
    assert out.best in autotune.TILE_CANDIDATES and not out.cached
    assert all(t["error"] is None and t["seconds"] > 0 for t in out.trials), out.trials
    again = autotune.tune_tile(32, 32, cache_path=cache, repeats=1, steps=2)
    assert again.cached and again.best == out.best


def test_serving_settings_are_measured(tmp_path):
    need_gpu()
    reqs = [serve.Request(np=32, nc=16, n_steps=2, seed=100 + i) for i in range(3)]
    cands = autotune.serving_candidates(max_active=(1, 4), steps_per_chunk=(2,), graphs=(False,))
    out = autotune.tune_serving(reqs, 1 << 28, candidates=cands, cache_path=str(tmp_path / "t.json"))
    assert out.best in cands and not out.cached
    assert all(t["error"] is None and t["seconds"] > 0 for t in out.trials), out.trials
