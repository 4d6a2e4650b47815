"""Parity at the full 512^3 size, in the launch configuration bench.py times
(one CTA per tile, 52^3 tiles; encode kernels over all 134M particles), on
inputs from the shared seeded generators:

* encode and cell sort (Sec. III-A) of every particle: per-cell counts, v_c
  and sigma bit for bit, and each cell's multiset of records (within-cell
  order is unspecified) through per-cell sums of a 64-bit record hash;
* decode (Eq. 2-3) of every particle, bit for bit;
* the integer coarse CIC density (units 2^-27), bit for bit;
* the force at sampled particles against the oracle's direct short-range
  sums plus its coarse field, max relative error 1e-4 where |g| exceeds
  1e-3 of the largest |g|.
"""

import numpy as np
import pytest

from oracle import codec, dynamics, force
from paper_2003_03931_gb300 import synth
from tests.gpu_util import make_sim, need_gpu, oracle_state

pytestmark = pytest.mark.gpu

NP, NC = 512, 256


def _record_hash(st):
    """64-bit mix of each particle's six stored bytes (storage order)."""
    m = np.asarray(st.m, dtype=np.uint64)
    u = np.asarray(st.u, dtype=np.uint64)
    x = np.zeros(m.shape[0], dtype=np.uint64)
    for k, col in enumerate([m[:, 0], m[:, 1], m[:, 2], u[:, 0], u[:, 1], u[:, 2]]):
        x |= col << np.uint64(8 * k)
    # SplitMix64 finaliser (Steele, Lea & Flood 2014)
    x = (x ^ (x >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    x = (x ^ (x >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return x ^ (x >> np.uint64(31))


def _cell_hash_sums(st):
    h = _record_hash(st)
    starts = np.concatenate([[0], np.cumsum(st.counts.astype(np.int64))[:-1]])
    nz = st.counts > 0
    out = np.zeros(st.counts.size, dtype=np.uint64)
    with np.errstate(over="ignore"):
        out[nz] = np.add.reduceat(h, starts[nz])
    return out


@pytest.fixture(scope="module")
def full():
    need_gpu()
    rng = np.random.default_rng(512)
    n = NP ** 3
    Q = synth.clustered_codes(rng, n, NC, n_clusters=4096, frac=0.5, width_fine=8.0)
    P = synth.momenta(rng, n)
    w = dict(synth.WORKLOADS["c3_512"])
    sim = make_sim(**w)
    sim.load_qp(Q, P, 0.3)
    ref = dynamics.encode(Q.T, P.T, NC, 0.3)
    del Q, P
    got = oracle_state(sim)
    yield sim, ref, got
    sim.close()


def test_encode_and_sort_full_size(full):
    sim, ref, got = full
    np.testing.assert_array_equal(got.counts, ref.counts)
    np.testing.assert_array_equal(got.vc, ref.vc)
    assert np.float32(got.sigma) == np.float32(ref.sigma)
    np.testing.assert_array_equal(_cell_hash_sums(got), _cell_hash_sums(ref))


def test_decode_full_size(full):
    sim, ref, got = full
    Qg, Pg = sim.fetch_decoded()
    np.testing.assert_array_equal(Qg.T.astype(np.int64), got.codes())
    np.testing.assert_array_equal(Pg.T, got.momenta())


def test_coarse_density_full_size(full):
    sim, ref, got = full
    rho = sim.fetch_coarse_density()
    np.testing.assert_array_equal(rho, force.coarse_density_chunked(ref.codes(), NC).ravel())


def test_force_sampled_full_size(full):
    sim, ref, got = full
    g = sim.fetch_force()                        # GPU store order
    Qr = ref.codes()
    rng = np.random.default_rng(7)
    idx = np.sort(rng.choice(Qr.shape[0], 96, replace=False))
    go = force.sampled_force(Qr, ref.counts, NC, idx)
    # the same particle in the GPU store: same cell, same position bins
    offs = np.concatenate([[0], np.cumsum(got.counts.astype(np.int64))])
    cell = codec.flatten_cell(Qr[idx] // 256, NC)
    mg = np.asarray(got.m, dtype=np.int64)
    mr = np.asarray(ref.m, dtype=np.int64)
    gg = np.zeros((len(idx), 3))
    for k, (i, c) in enumerate(zip(idx, cell)):
        lo, hi = offs[c], offs[c + 1]
        j = lo + int(np.flatnonzero((mg[lo:hi] == mr[i]).all(axis=1))[0])
        gg[k] = g[:, j]
    peak = np.linalg.norm(g, axis=0).max()
    norm = np.linalg.norm(go, axis=1)
    sel = norm > 1e-3 * peak
    assert sel.sum() > 48
    err = (np.linalg.norm(gg - go, axis=1)[sel] / norm[sel]).max()
    assert err <= 1e-4, err
