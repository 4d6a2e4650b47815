"""Many simulations on one GPU: a thin wrapper over the pmpm_batch_* calls
of include/pmpm.h, plus the seeded request streams used to measure it.

The engine itself (admission, streams, table cache, stepping) is native code
in libpmpm; this module marshals requests and results.  Each request is one
whole box: Zel'dovich initial conditions (Sec. IV-A.2), n_steps PM-PM steps
(Sec. II), and the power spectrum of the final particles (Sec. IV-D).
"""

import ctypes
import math
from dataclasses import dataclass

import numpy as np

from . import _lib


@dataclass
class Request:
    np: int                      # particles per side
    nc: int                      # coarse cells per side
    n_steps: int
    seed: int
    slope: float = -1.5          # P(k) ~ k^slope exp(-(k/k_c)^2)
    k_c: float = math.pi / 2     # half the fine-mesh Nyquist wavenumber
    rms_disp: float = 0.3        # fine cells at a_init
    a_init: float = 0.02
    a_final: float = 1.0
    arrival: float = 0.0         # engine-clock seconds
    pk_nmesh: int = 0            # 0: min(np, 4 nc)
    pk_nbins: int = 0            # 0: pk_nmesh / 2
    want_state: bool = False     # also return the final store (streams, counts)
    lowmem: bool = False         # the low-memory step (PMPM_FLAG_LOWMEM)

    @property
    def n(self):
        return self.np ** 3

    def mesh(self):
        m = self.pk_nmesh or min(self.np, 4 * self.nc)
        return m, self.pk_nbins or m // 2


@dataclass
class Result:
    id: int
    status: int
    t_arrival: float
    t_admit: float
    t_done: float
    a: float
    sigma: float
    particle_steps: int
    request: Request
    k: np.ndarray
    pk: np.ndarray
    nmodes: np.ndarray
    streams: np.ndarray = None   # uint8 [6][N] when requested
    counts: np.ndarray = None    # int32 [nc^3] when requested

    @property
    def latency(self):
        return self.t_done - self.t_arrival


class Engine:
    """A batch engine over one device arena (a torch uint8 tensor)."""

    def __init__(self, arena_bytes, max_active=32, share_tables=True, graphs=False,
                 priorities=True, steps_per_chunk=2, chunks_in_flight=2, device="cuda:0",
                 large_np=0, max_large=0):
        import torch
        self.lib = _lib.load()
        self.device = torch.device(device)
        self.arena = torch.empty(int(arena_bytes), dtype=torch.uint8, device=self.device)
        c = _lib.BatchConfig(max_active, int(share_tables), int(graphs), int(priorities),
                             steps_per_chunk, chunks_in_flight, large_np, max_large)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            rc = self.lib.pmpm_batch_create(ctypes.byref(c), ctypes.c_void_p(self.arena.data_ptr()),
                                            self.arena.numel(), ctypes.byref(h))
        if rc != _lib.PMPM_OK:
            raise _lib.PmpmError(rc, self.lib.pmpm_batch_last_error(None).decode())
        self.h = h
        self._pending = {}

    def _check(self, rc):
        if rc != _lib.PMPM_OK:
            raise _lib.PmpmError(rc, self.lib.pmpm_batch_last_error(self.h).decode())

    def clock(self):
        return self.lib.pmpm_batch_clock(self.h)

    def submit(self, req):
        m, nb = req.mesh()
        out = dict(k=np.zeros(nb), pk=np.zeros(nb), nmodes=np.zeros(nb, np.int64))
        if req.want_state:
            out["streams"] = np.zeros((6, req.n), np.uint8)
            out["counts"] = np.zeros(req.nc ** 3, np.int32)
        r = _lib.Request(req.np, req.nc, req.n_steps, req.pk_nmesh, req.pk_nbins,
                         _lib.FLAG_LOWMEM if req.lowmem else 0,
                         req.a_init, req.a_final, req.seed, req.slope, req.k_c, req.rms_disp,
                         req.arrival, out["k"].ctypes.data, out["pk"].ctypes.data,
                         out["nmodes"].ctypes.data,
                         out["streams"].ctypes.data if req.want_state else None,
                         out["counts"].ctypes.data if req.want_state else None)
        rid = ctypes.c_int64()
        self._check(self.lib.pmpm_batch_submit(self.h, ctypes.byref(r), ctypes.byref(rid)))
        self._pending[rid.value] = (req, out)
        return rid.value

    def progress(self):
        n = ctypes.c_int32()
        self._check(self.lib.pmpm_batch_progress(self.h, ctypes.byref(n)))
        return n.value

    def run(self, timeout=3600.0):
        self._check(self.lib.pmpm_batch_run(self.h, float(timeout)))

    def poll(self):
        buf = (_lib.Result * 64)()
        n = ctypes.c_int32()
        got = []
        while True:
            self._check(self.lib.pmpm_batch_poll(self.h, buf, 64, ctypes.byref(n)))
            for r in buf[:n.value]:
                req, out = self._pending.pop(r.id)
                got.append(Result(r.id, r.status, r.t_arrival, r.t_admit, r.t_done, r.a, r.sigma,
                                  r.particle_steps, req, out["k"], out["pk"], out["nmodes"],
                                  out.get("streams"), out.get("counts")))
            if n.value < 64:
                return got

    def stats(self):
        s = _lib.BatchStats()
        self._check(self.lib.pmpm_batch_get_stats(self.h, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in _lib.BatchStats._fields_}

    def last_error(self):
        return self.lib.pmpm_batch_last_error(self.h).decode()

    def close(self):
        if getattr(self, "h", None):
            self.lib.pmpm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------ request streams
# Mixed-size workload: particle counts 32^3 / 64^3 / 128^3 / 256^3 with
# weights 0.4 / 0.3 / 0.2 / 0.1, 10-40 steps each, power-law slopes in
# [-2, -1], independent seeds, Poisson arrivals.
MIX_SIZES = (32, 64, 128, 256)
MIX_WEIGHTS = (0.4, 0.3, 0.2, 0.1)


def mixed_requests(count, seed=0, rate=None, steps=(10, 40), sizes=MIX_SIZES, weights=MIX_WEIGHTS,
                   slopes=(-2.0, -1.0), seed_base=1000):
    """`count` requests; arrivals at 0 when rate is None, else a Poisson
    process of `rate` requests per second starting at 0."""
    rng = np.random.default_rng(seed)
    idx = rng.choice(len(sizes), size=count, p=np.asarray(weights) / np.sum(weights))
    n_steps = rng.integers(steps[0], steps[1] + 1, size=count)
    slope = rng.uniform(slopes[0], slopes[1], size=count)
    if rate is None:
        t = np.zeros(count)
    else:
        t = np.cumsum(rng.exponential(1.0 / rate, size=count))
        t -= t[0]
    out = []
    for i in range(count):
        n_p = int(sizes[idx[i]])
        out.append(Request(np=n_p, nc=n_p // 2, n_steps=int(n_steps[i]), seed=seed_base + i,
                           slope=float(slope[i]), arrival=float(t[i])))
    return out


def with_arrivals(reqs, rate, seed=0):
    """The same requests on a Poisson arrival process of `rate` per second."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=len(reqs)))
    t -= t[0]
    return [Request(**{**r.__dict__, "arrival": float(ti)}) for r, ti in zip(reqs, t)]


def latency_summary(results):
    """p50/p99/mean latency (s), makespan and throughput of a finished run."""
    ok = [r for r in results if r.status == 0]
    lat = np.array([r.latency for r in ok])
    t_first = min(r.t_arrival for r in results)
    t_last = max(r.t_done for r in results)
    span = t_last - t_first
    ps = sum(r.particle_steps for r in ok)
    return {
        "requests": len(results),
        "failed": len(results) - len(ok),
        "p50_s": float(np.percentile(lat, 50)) if len(lat) else None,
        "p99_s": float(np.percentile(lat, 99)) if len(lat) else None,
        "mean_s": float(lat.mean()) if len(lat) else None,
        "makespan_s": span,
        "requests_per_s": len(ok) / span if span > 0 else None,
        "particle_steps_per_s": ps / span if span > 0 else None,
    }


def run_stream(engine, reqs, timeout=3600.0):
    """Submit `reqs` with arrivals offset to now, run them all, return results
    in submission order."""
    t0 = engine.clock() + 1e-3
    ids = [engine.submit(Request(**{**r.__dict__, "arrival": r.arrival + t0})) for r in reqs]
    engine.run(timeout)
    res = {r.id: r for r in engine.poll()}
    return [res[i] for i in ids]
