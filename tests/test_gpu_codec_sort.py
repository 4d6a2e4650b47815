"""GPU parity of the codec and the cell-ordered re-encode (Sec. III-A,
Eq. 2-4) against the oracle on identical inputs: bit-exact."""

import numpy as np
import pytest

from oracle import cic, dynamics
from paper_2003_03931_gb300 import synth
from tests.gpu_util import cell_sorted_records, make_sim, need_gpu

pytestmark = pytest.mark.gpu


def _compare_encode(sim, Q, P, a=0.3):
    sim.load_qp(Q, P, a)
    got = sim.fetch_state()
    ref = dynamics.encode(Q.T.astype(np.int64), P.T, sim.cfg.nc, a)
    np.testing.assert_array_equal(got["counts"], ref.counts)
    np.testing.assert_array_equal(got["vc"], ref.vc.T)
    assert np.float32(got["scalars"]["sigma"]) == ref.sigma
    rec_g = np.concatenate([got["streams"][:3], got["streams"][3:]]).T
    rec_o = np.concatenate([ref.m.T, ref.u.T]).T
    np.testing.assert_array_equal(cell_sorted_records(ref.counts, rec_g),
                                  cell_sorted_records(ref.counts, rec_o))
    return got, ref


@pytest.mark.parametrize("kind", ["uniform", "clustered", "one_cell"])
def test_encode_bit_exact(kind):
    need_gpu()
    rng = np.random.default_rng({"uniform": 1, "clustered": 2, "one_cell": 3}[kind])
    sim = make_sim(np=16, nc=8, a_init=0.1, a_final=0.5, n_steps=4)
    n = sim.cfg.n
    if kind == "uniform":
        Q = synth.uniform_codes(rng, n, 8)
    elif kind == "clustered":
        Q = synth.clustered_codes(rng, n, 8, width_fine=1.0)
    else:
        Q = synth.single_cell_codes(n, 8)
    P = synth.momenta(rng, n)
    _compare_encode(sim, Q, P)
    sim.close()


def test_encode_spans_scan_blocks_and_empty_cells():
    # 64^3 cells: several scan blocks; a clustered load leaves most cells empty
    need_gpu()
    rng = np.random.default_rng(5)
    sim = make_sim(np=64, nc=64, a_init=0.1, a_final=0.5, n_steps=4)
    Q = synth.clustered_codes(rng, sim.cfg.n, 64, frac=0.9, width_fine=6.0)
    P = synth.momenta(rng, sim.cfg.n, bulk=20.0, disp=3.0)
    got, ref = _compare_encode(sim, Q, P)
    assert (ref.counts == 0).mean() > 0.3
    sim.close()


def test_decode_bit_exact():
    need_gpu()
    rng = np.random.default_rng(6)
    sim = make_sim(np=16, nc=8, a_init=0.1, a_final=0.5, n_steps=4)
    Q = synth.clustered_codes(rng, sim.cfg.n, 8)
    sim.load_qp(Q, synth.momenta(rng, sim.cfg.n), 0.3)
    st = sim.fetch_state()
    Qd, Pd = sim.fetch_decoded()
    ost = dynamics.State(8, st["counts"], st["streams"][:3].T, st["streams"][3:].T, st["vc"].T,
                         np.float32(st["scalars"]["sigma"]), 0.3)
    np.testing.assert_array_equal(Qd.T, ost.codes())
    np.testing.assert_array_equal(Pd.T, ost.momenta())
    sim.close()


@pytest.mark.parametrize("nc,np_", [(8, 16), (32, 32)])
def test_coarse_density_bit_exact(nc, np_):
    need_gpu()
    rng = np.random.default_rng(7)
    sim = make_sim(np=np_, nc=nc, a_init=0.1, a_final=0.5, n_steps=4)
    Q = synth.clustered_codes(rng, sim.cfg.n, nc)
    sim.load_qp(Q, synth.momenta(rng, sim.cfg.n), 0.3)
    rho = sim.fetch_coarse_density()
    ref = cic.deposit(Q.T.astype(np.int64), nc, 4)
    np.testing.assert_array_equal(rho, ref.ravel())
    assert rho.sum() == sim.cfg.n * 2 ** 27
    sim.close()


def test_coarse_density_crowded_cell():
    # every particle in one coarse cell: the deposit's 32-bit per-cell sums
    # are flushed every 31 particles
    need_gpu()
    sim = make_sim(np=16, nc=8, a_init=0.1, a_final=0.5, n_steps=4)
    rng = np.random.default_rng(8)
    Q = synth.single_cell_codes(sim.cfg.n, 8)
    sim.load_qp(Q, synth.momenta(rng, sim.cfg.n), 0.3)
    rho = sim.fetch_coarse_density()
    ref = cic.deposit(Q.T.astype(np.int64), 8, 4)
    np.testing.assert_array_equal(rho, ref.ravel())
    assert rho.sum() == sim.cfg.n * 2 ** 27
    sim.close()
