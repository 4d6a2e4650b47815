"""Autotuner for the choices the library leaves to its caller.

The step itself has no free launch shape: the tile FFT box is 32^3 (one
CTA of 512 threads per tile, the whole box in one SM's shared memory), and
the tile buffer equals the short-range cutoff of 6 fine cells (Sec. IV-A.2),
which the force split fixes.  What remains open, and what this module tunes
by measurement on the GPU at hand, is

- the tile edge (``tile_max``, 4 or 5 coarse cells): how the coarse mesh is
  cut into tiles, i.e. the number of 32^3 tile transforms per step against
  the particles each tile deposits and gathers;
- the serving engine's concurrency and chunking (``max_active``,
  ``steps_per_chunk``, ``chunks_in_flight``, CUDA graphs on or off) for a
  given request mix.

Each candidate runs a short calibration through the public API and is
timed with a device synchronisation on both sides; the median of a few
repeats decides, ties going to the earlier candidate.  The winner is
cached in a JSON file keyed by the GPU's name, the workload and a hash of
the library's sources, so a rebuilt library or another GPU measures again.
"""

import dataclasses
import hashlib
import json
import os
import statistics
import time

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = [os.path.join(HERE, "csrc"), os.path.join(os.path.dirname(HERE), "include")]


def default_cache_path():
    base = os.environ.get("PMPM_TUNE_CACHE")
    if base:
        return base
    root = os.environ.get("XDG_CACHE_HOME") or os.path.join(os.path.expanduser("~"), ".cache")
    return os.path.join(root, "pmpm_gb300", "tune.json")


def library_version():
    """Hash of the library's CUDA sources and C header (the cache is stale
    once they change)."""
    h = hashlib.sha256()
    for d in SOURCES:
        for name in sorted(os.listdir(d)):
            if name.endswith((".cu", ".cuh", ".h")):
                h.update(name.encode())
                with open(os.path.join(d, name), "rb") as f:
                    h.update(f.read())
    return h.hexdigest()[:16]


def _key_string(key):
    return json.dumps(key, sort_keys=True, separators=(",", ":"))


def _load(path):
    try:
        with open(path) as f:
            data = json.load(f)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}


def _store(path, data):
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    tmp = f"{path}.{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


@dataclasses.dataclass
class Outcome:
    best: dict                 # the chosen candidate
    cached: bool               # taken from the cache without measuring
    trials: list               # [{"params", "seconds" (median) or None, "runs", "error"}]


def tune(key, candidates, measure, cache_path=None, repeats=3, force=False):
    """Return the candidate with the smallest median of ``measure(candidate)``
    (seconds) over ``repeats`` runs.

    key: JSON-serialisable dict naming the workload (the GPU name and the
    library version are added by the callers below).  A cached winner for the
    same key is returned without measuring, unless ``force`` or it is no
    longer among ``candidates``.  A candidate whose measurement raises is
    skipped (its error is recorded); if all fail, RuntimeError."""
    if not candidates:
        raise ValueError("no candidates")
    path = cache_path or default_cache_path()
    ks = _key_string(key)
    data = _load(path)
    hit = data.get(ks)
    if not force and hit and hit.get("best") in candidates:
        return Outcome(best=hit["best"], cached=True, trials=hit.get("trials", []))
    trials = []
    for cand in candidates:
        runs, error = [], None
        for _ in range(repeats):
            try:
                runs.append(float(measure(cand)))
            except Exception as e:   # a candidate that cannot run loses
                error = f"{type(e).__name__}: {e}"
                break
        med = statistics.median(runs) if runs and error is None else None
        trials.append({"params": cand, "seconds": med, "runs": runs, "error": error})
    ok = [t for t in trials if t["seconds"] is not None]
    if not ok:
        raise RuntimeError("every candidate failed: " + "; ".join(str(t["error"]) for t in trials))
    best = min(ok, key=lambda t: t["seconds"])["params"]   # min keeps the first of equals
    data = _load(path)   # re-read: another process may have added keys meanwhile
    data[ks] = {"best": best, "trials": trials, "when": time.time()}
    _store(path, data)
    return Outcome(best=best, cached=False, trials=trials)


# --------------------------------------------------------------- the tile edge

TILE_CANDIDATES = [{"tile_max": 5}, {"tile_max": 4}]


def _gpu_name(device):
    import torch
    return torch.cuda.get_device_name(torch.device(device))


def measure_tile_step(cfg, steps=3, warmup=1, seed=1, device="cuda:0"):
    """Seconds per step of one box with configuration ``cfg`` (a SimConfig):
    Zel'dovich initial conditions, ``warmup`` untimed steps, then ``steps``
    steps between two device synchronisations."""
    from .sim import Simulation
    sim = Simulation(cfg, device=device)
    try:
        sim.ic_zeldovich(seed)
        sim.step(warmup)
        sim.sync()
        t0 = time.perf_counter()
        sim.step(steps)
        sim.sync()
        return (time.perf_counter() - t0) / steps
    finally:
        sim.close()


def tune_tile(np_, nc, pos_bytes=1, lowmem=False, cache_path=None, repeats=3, force=False,
              device="cuda:0", steps=3, measure=None, gpu_name=None):
    """Pick ``tile_max`` for boxes of np_^3 particles on an nc^3 coarse mesh.
    Returns an Outcome whose ``best`` is {"tile_max": 4 or 5}."""
    from .sim import SimConfig

    def run(cand):
        cfg = SimConfig(np=np_, nc=nc, a_init=0.02, a_final=1.0, n_steps=max(steps + 1, 2),
                        pos_bytes=pos_bytes, lowmem=lowmem, **cand)
        return measure_tile_step(cfg, steps=steps, device=device)

    key = {"what": "tile", "np": np_, "nc": nc, "pos_bytes": pos_bytes, "lowmem": bool(lowmem),
           "gpu": gpu_name or _gpu_name(device), "lib": library_version()}
    return tune(key, TILE_CANDIDATES, measure or run, cache_path, repeats, force)


# ----------------------------------------------------------- the serving engine

def serving_candidates(max_active=(8, 32), steps_per_chunk=(1, 2, 4), graphs=(False, True),
                       chunks_in_flight=(2,)):
    return [{"max_active": a, "steps_per_chunk": s, "graphs": g, "chunks_in_flight": c}
            for a in max_active for s in steps_per_chunk for g in graphs for c in chunks_in_flight]


def measure_serving(params, reqs, arena_bytes, device="cuda:0", timeout=600.0):
    """Makespan in seconds of the request list ``reqs`` (serve.Request, all
    arriving at once) on a fresh engine with ``params``; a failed request
    makes the candidate fail."""
    from . import serve
    eng = serve.Engine(arena_bytes, device=device, **params)
    try:
        t0 = time.perf_counter()
        res = serve.run_stream(eng, reqs, timeout)
        dt = time.perf_counter() - t0
    finally:
        eng.close()
    bad = [r for r in res if r.status != 0]
    if bad:
        raise RuntimeError(f"{len(bad)} request(s) failed, first status {bad[0].status}")
    return dt


def tune_serving(reqs, arena_bytes, candidates=None, cache_path=None, repeats=1, force=False,
                 device="cuda:0", measure=None, gpu_name=None):
    """Pick the serving engine's parameters for a request mix.  The key holds
    a digest of the mix (sizes, steps, mesh of each request), so another mix
    measures again."""
    cands = candidates or serving_candidates()
    mix = hashlib.sha256(json.dumps([[r.np, r.nc, r.n_steps, r.pk_nmesh] for r in reqs]).encode())
    key = {"what": "serving", "mix": mix.hexdigest()[:16], "requests": len(reqs),
           "arena": int(arena_bytes), "gpu": gpu_name or _gpu_name(device), "lib": library_version()}
    run = measure or (lambda p: measure_serving(p, reqs, arena_bytes, device))
    return tune(key, cands, run, cache_path, repeats, force)
