"""GPU parity of the 2-byte position format (Sec. III-A, B = 65536 bins per
coarse cell; CIC weight products rounded to the 1-byte units): encode, cell
sort and decode bit for bit, integer coarse density bit for bit, force
within 1e-4, initial conditions, one step, and P(k) within 0.5% per bin
after the 10 steps of the 32^3 workload."""

import numpy as np
import pytest

from oracle import dynamics, force, ic, power
from paper_2003_03931_gb300 import synth
from tests.gpu_util import (cell_sorted_records, load_oracle_state, make_sim, need_gpu,
                            oracle_state, vector_rel_err)

pytestmark = pytest.mark.gpu

B2 = 65536


def _records(st):
    return cell_sorted_records(st.counts, np.concatenate([st.m, st.u], axis=1).astype(np.int64))


@pytest.mark.parametrize("kind", ["uniform", "clustered"])
def test_encode_decode_bit_exact_2byte(kind):
    need_gpu()
    rng = np.random.default_rng(21)
    nc = 16
    sim = make_sim(np=32, nc=nc, a_init=0.1, a_final=0.5, n_steps=2, pos_bytes=2)
    n = sim.cfg.n
    Q = (synth.uniform_codes(rng, n, nc, bins=B2) if kind == "uniform"
         else synth.clustered_codes(rng, n, nc, n_clusters=6, frac=0.5, width_fine=2.0, bins=B2))
    P = synth.momenta(rng, n)
    sim.load_qp(Q, P, 0.3)
    got = oracle_state(sim)
    ref = dynamics.encode(Q.T, P.T, nc, 0.3, pos_bytes=2)
    np.testing.assert_array_equal(got.counts, ref.counts)
    np.testing.assert_array_equal(got.vc, ref.vc)
    assert np.float32(got.sigma) == np.float32(ref.sigma)
    assert got.m.dtype == np.uint16
    np.testing.assert_array_equal(_records(got), _records(ref))
    Qg, Pg = sim.fetch_decoded()
    np.testing.assert_array_equal(Qg.T.astype(np.int64), got.codes())
    np.testing.assert_array_equal(Pg.T, got.momenta())
    sim.close()


def test_coarse_density_and_force_2byte():
    need_gpu()
    rng = np.random.default_rng(22)
    nc = 16
    sim = make_sim(np=32, nc=nc, a_init=0.1, a_final=0.5, n_steps=2, pos_bytes=2)
    n = sim.cfg.n
    Q = synth.clustered_codes(rng, n, nc, n_clusters=8, frac=0.4, width_fine=3.0, bins=B2)
    sim.load_qp(Q, synth.momenta(rng, n), 0.3)
    st = oracle_state(sim)
    op = force.ForceOperator(nc, pos_bytes=2)
    np.testing.assert_array_equal(sim.fetch_coarse_density(), op.coarse_density(st.codes()).ravel())
    g = sim.fetch_force()
    ref = op.particle_force(st.codes()).T
    assert vector_rel_err(g, ref) <= 1e-4
    sim.close()


def test_initial_conditions_and_power_spectrum_2byte():
    need_gpu()
    w = synth.WORKLOADS["c1_32"]
    sim = make_sim(**w, pos_bytes=2)
    sim.ic_zeldovich(5, **synth.IC_SPECTRUM)
    got = oracle_state(sim)
    ref, _, _ = ic.zeldovich(5, w["np"], w["nc"], w["a_init"], pos_bytes=2, **synth.IC_SPECTRUM)
    # float64 on both sides: codes equal up to a rare rounding of floor(16384 x)
    assert np.abs(got.counts.astype(int) - ref.counts).sum() <= 2
    if (got.counts == ref.counts).all():
        a = cell_sorted_records(got.counts, got.codes())
        b = cell_sorted_records(ref.counts, ref.codes())
        assert (np.abs(a - b) > 1).sum() == 0 and (a != b).mean() < 1e-4
    np.testing.assert_allclose(float(got.sigma), float(ref.sigma), rtol=1e-6)
    for nmesh in (64, 32):
        kg, pg, ng = sim.power_spectrum(nmesh, nmesh // 2)
        ko, po, no = power.power_spectrum(got.codes(), nmesh, nmesh // 2, 64, pos_bytes=2)
        np.testing.assert_array_equal(ng, no)
        np.testing.assert_allclose(pg, po, rtol=2e-5)
    sim.close()


def test_steps_and_power_spectrum_after_ten_steps_2byte():
    need_gpu()
    w = synth.WORKLOADS["c1_32"]
    sim = make_sim(**w, pos_bytes=2)
    sim.ic_zeldovich(5, **synth.IC_SPECTRUM)
    ost = oracle_state(sim)
    oref = dynamics.Simulation(w["nc"], w["a_init"], w["a_final"], w["n_steps"], pos_bytes=2)
    # one step from the same state
    sim.step(1)
    one = oracle_state(sim)
    ref1 = oref.step(ost)
    assert np.abs(one.counts.astype(int) - ref1.counts).sum() <= 0.002 * sim.cfg.n
    np.testing.assert_allclose(float(one.sigma), float(ref1.sigma), rtol=1e-4)
    # ten steps: P(k) within 0.5% per bin
    load_oracle_state(sim, ost)
    sim.step(10)
    ost10 = oref.run(ost, 10)
    kg, pg, ng = sim.power_spectrum(64, 32)
    ko, po, no = power.power_spectrum(ost10.codes(), 64, 32, 64, pos_bytes=2)
    np.testing.assert_array_equal(ng, no)
    assert (np.abs(pg / po - 1)).max() < 5e-3
    sim.close()
