"""Host logic of the autotuner (paper_2003_03931_gb300/autotune.py) with a
fake timer: the fastest candidate wins, the winner is cached per key and
reused without measuring, failing candidates lose, ties keep the candidate
order, and a new key (another GPU, library or workload) measures again."""

import json

import pytest

from paper_2003_03931_gb300 import autotune, serve


class FakeTimer:
    def __init__(self, seconds, fail=()):
        self.seconds = seconds
        self.fail = fail
        self.calls = []

    def __call__(self, cand):
        self.calls.append(dict(cand))
        k = json.dumps(cand, sort_keys=True)
        if k in self.fail:
            raise RuntimeError("cannot run")
        return self.seconds[k]


def _k(**c):
    return json.dumps(c, sort_keys=True)


def test_fastest_wins_and_is_cached(tmp_path):
    cache = str(tmp_path / "tune.json")
    cands = [{"a": 1}, {"a": 2}, {"a": 3}]
    t = FakeTimer({_k(a=1): 3.0, _k(a=2): 1.0, _k(a=3): 2.0})
    out = autotune.tune({"w": 1}, cands, t, cache, repeats=3)
    assert out.best == {"a": 2} and not out.cached
    assert len(t.calls) == 9 and [tr["seconds"] for tr in out.trials] == [3.0, 1.0, 2.0]
    again = autotune.tune({"w": 1}, cands, t, cache, repeats=3)
    assert again.best == {"a": 2} and again.cached and len(t.calls) == 9
    forced = autotune.tune({"w": 1}, cands, t, cache, repeats=1, force=True)
    assert not forced.cached and len(t.calls) == 12
    # another key measures again; the file keeps both
    autotune.tune({"w": 2}, cands, t, cache, repeats=1)
    assert len(t.calls) == 15 and len(json.load(open(cache))) == 2


def test_median_not_minimum_decides(tmp_path):
    runs = {"a": [0.5, 9.0, 9.0], "b": [2.0, 2.0, 2.0]}   # a has the single best run, b the median
    it = {k: iter(v) for k, v in runs.items()}
    out = autotune.tune({"m": 1}, [{"c": "a"}, {"c": "b"}], lambda c: next(it[c["c"]]),
                        str(tmp_path / "t.json"), repeats=3)
    assert out.best == {"c": "b"}


def test_failures_lose_and_all_failing_raises(tmp_path):
    cache = str(tmp_path / "tune.json")
    cands = [{"a": 1}, {"a": 2}]
    t = FakeTimer({_k(a=1): 1.0, _k(a=2): 2.0}, fail={_k(a=1)})
    out = autotune.tune({"w": 1}, cands, t, cache)
    assert out.best == {"a": 2}
    assert out.trials[0]["seconds"] is None and "cannot run" in out.trials[0]["error"]
    t2 = FakeTimer({}, fail={_k(a=1), _k(a=2)})
    with pytest.raises(RuntimeError):
        autotune.tune({"w": 9}, cands, t2, cache)
    with pytest.raises(ValueError):
        autotune.tune({"w": 9}, [], t2, cache)


def test_ties_keep_candidate_order(tmp_path):
    t = FakeTimer({_k(a=1): 1.0, _k(a=2): 1.0})
    out = autotune.tune({"w": 1}, [{"a": 2}, {"a": 1}], t, str(tmp_path / "t.json"), repeats=1)
    assert out.best == {"a": 2}


def test_cached_winner_outside_candidates_remeasures(tmp_path):
    cache = str(tmp_path / "t.json")
    t = FakeTimer({_k(a=1): 1.0, _k(a=2): 2.0, _k(a=3): 0.5})
    autotune.tune({"w": 1}, [{"a": 1}, {"a": 2}], t, cache, repeats=1)
    out = autotune.tune({"w": 1}, [{"a": 2}, {"a": 3}], t, cache, repeats=1)
    assert out.best == {"a": 3} and not out.cached


def test_corrupt_cache_is_ignored(tmp_path):
    cache = tmp_path / "t.json"
    cache.write_text("{not json")
    t = FakeTimer({_k(a=1): 1.0})
    assert autotune.tune({"w": 1}, [{"a": 1}], t, str(cache), repeats=1).best == {"a": 1}
    assert json.loads(cache.read_text())


def test_tile_and_serving_keys(tmp_path):
    cache = str(tmp_path / "t.json")
    t = FakeTimer({_k(tile_max=5): 1.0, _k(tile_max=4): 1.5})
    out = autotune.tune_tile(32, 16, cache_path=cache, measure=t, gpu_name="GPU-A", repeats=1)
    assert out.best == {"tile_max": 5}
    assert autotune.tune_tile(32, 16, cache_path=cache, measure=t, gpu_name="GPU-A").cached
    assert not autotune.tune_tile(32, 16, cache_path=cache, measure=t, gpu_name="GPU-B",
                                  repeats=1).cached
    assert not autotune.tune_tile(64, 32, cache_path=cache, measure=t, gpu_name="GPU-A",
                                  repeats=1).cached
    keys = [json.loads(k) for k in json.load(open(cache))]
    assert all(k["lib"] == autotune.library_version() for k in keys)
    # serving: the mix is part of the key
    cands = autotune.serving_candidates()
    assert len(cands) == 12 and len({json.dumps(c, sort_keys=True) for c in cands}) == 12
    secs = {json.dumps(c, sort_keys=True): 1.0 + 0.01 * i for i, c in enumerate(cands)}
    secs[json.dumps(cands[7], sort_keys=True)] = 0.1
    ts = FakeTimer(secs)
    reqs = serve.mixed_requests(6, seed=3)
    out = autotune.tune_serving(reqs, 1 << 30, cache_path=cache, measure=ts, gpu_name="GPU-A")
    assert out.best == cands[7] and len(ts.calls) == 12
    assert autotune.tune_serving(reqs, 1 << 30, cache_path=cache, measure=ts, gpu_name="GPU-A").cached
    autotune.tune_serving(serve.mixed_requests(7, seed=3), 1 << 30, cache_path=cache, measure=ts,
                          gpu_name="GPU-A")
    assert len(ts.calls) == 24


def test_library_version_is_stable():
    v = autotune.library_version()
    assert len(v) == 16 and int(v, 16) >= 0 and v == autotune.library_version()


def test_default_cache_path_honours_environment(monkeypatch, tmp_path):
    monkeypatch.setenv("PMPM_TUNE_CACHE", str(tmp_path / "x.json"))
    assert autotune.default_cache_path() == str(tmp_path / "x.json")
    monkeypatch.delenv("PMPM_TUNE_CACHE")
    monkeypatch.setenv("XDG_CACHE_HOME", str(tmp_path))
    assert autotune.default_cache_path() == str(tmp_path / "pmpm_gb300" / "tune.json")
