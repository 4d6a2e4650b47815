"""Helpers shared by the GPU tests: sims, and conversion of fetched stores
into oracle states.  Comparisons are per cell where within-cell order is
unspecified (Sec. III-A fixes only the cell order)."""

import numpy as np
import pytest

from oracle import dynamics
from paper_2003_03931_gb300.sim import join_store, split_store


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_03931_gb300 import build
    build.build()


def make_sim(**kw):
    from paper_2003_03931_gb300.sim import SimConfig, Simulation
    return Simulation(SimConfig(**kw), device="cuda:0")


def oracle_state(sim):
    """The sim's current store as an oracle State (same storage order)."""
    st = sim.fetch_state()
    pb = sim.cfg.pos_bytes
    m, u = split_store(st["streams"], sim.cfg.n, pb)
    return dynamics.State(sim.cfg.nc, st["counts"], m.T, u.T, st["vc"].T,
                          np.float32(st["scalars"]["sigma"]), st["scalars"]["a"],
                          st["scalars"]["step"], pos_bytes=pb)


def load_oracle_state(sim, ost):
    m = np.ascontiguousarray(ost.m.T).astype(np.uint8 if sim.cfg.pos_bytes == 1 else np.uint16)
    raw = join_store(m, ost.u.T)
    if sim.cfg.pos_bytes == 1:
        raw = raw.reshape(6, -1)
    sim.load_state({"streams": raw, "counts": ost.counts, "vc": ost.vc.T,
                    "scalars": {"a": ost.a, "sigma": float(ost.sigma), "step": ost.step}})


def cell_sorted_records(counts, recs):
    """Sort records [N, k] within each cell (cell order kept) for multiset
    comparison."""
    cell = np.repeat(np.arange(counts.size), counts)
    keys = [recs[:, j] for j in range(recs.shape[1] - 1, -1, -1)] + [cell]
    order = np.lexsort(keys)
    return recs[order]


def vector_rel_err(g, ref, floor=1e-3):
    """max |g - ref| / |ref| over particles with |ref| > floor * max |ref|
    (vectors [3, N])."""
    nrm = np.linalg.norm(ref, axis=0)
    sel = nrm > floor * nrm.max()
    return (np.linalg.norm(g - ref, axis=0)[sel] / nrm[sel]).max()
