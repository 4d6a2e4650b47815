"""GPU parity of whole PM-PM steps: one step from an identical state, the
power spectrum after the 10-step 32^3 run (within 0.5% per k-bin), the
Zel'dovich initial conditions, determinism and checkpoint/resume."""

import numpy as np
import pytest

from oracle import codec, dynamics, ic, power
from paper_2003_03931_gb300 import synth
from tests.gpu_util import cell_sorted_records, load_oracle_state, make_sim, need_gpu, oracle_state

pytestmark = pytest.mark.gpu


def _codes(sim):
    Q, _ = sim.fetch_decoded()
    return Q.T.astype(np.int64)


def test_initial_conditions_match_oracle():
    need_gpu()
    w = synth.WORKLOADS["c1_32"]
    sim = make_sim(**w)
    sim.ic_zeldovich(5, **synth.IC_SPECTRUM)
    got = oracle_state(sim)
    ref, _, _ = ic.zeldovich(5, w["np"], w["nc"], w["a_init"], **synth.IC_SPECTRUM)
    # decoded positions: identical up to a rare float64 rounding of floor(64 x)
    a = cell_sorted_records(got.counts, got.codes())
    b = cell_sorted_records(ref.counts, ref.codes())
    assert np.abs(got.counts.astype(int) - ref.counts).sum() <= 2
    if a.shape == b.shape and (got.counts == ref.counts).all():
        assert (np.abs(a - b) > 1).sum() == 0
        assert (a != b).mean() < 1e-4
    np.testing.assert_allclose(float(got.sigma), float(ref.sigma), rtol=1e-6)
    sim.close()


def test_one_step_matches_oracle():
    need_gpu()
    w = synth.WORKLOADS["c1_32"]
    sim = make_sim(**w)
    sim.ic_zeldovich(5, **synth.IC_SPECTRUM)
    ost = oracle_state(sim)
    oref = dynamics.Simulation(w["nc"], w["a_init"], w["a_final"], w["n_steps"])
    ost = oref.run(ost, 3)
    load_oracle_state(sim, ost)
    sim.step(1)
    got = oracle_state(sim)
    ref = oref.step(ost)
    # new codes: float32 force differences flip at most a few drift roundings
    diff = (np.abs(got.counts.astype(int) - ref.counts)).sum()
    assert diff <= 0.002 * sim.cfg.n
    assert got.step == ref.step and abs(got.a - ref.a) < 1e-15
    np.testing.assert_allclose(float(got.sigma), float(ref.sigma), rtol=1e-4)
    sim.close()


def test_power_spectrum_after_ten_steps():
    # 32^3 particles, 10 steps a = 0.02 -> 1: P(k) within 0.5% per k-bin
    need_gpu()
    w = synth.WORKLOADS["c1_32"]
    sim = make_sim(**w)
    sim.ic_zeldovich(5, **synth.IC_SPECTRUM)
    ost = oracle_state(sim)
    sim.step(10)
    ost = dynamics.Simulation(w["nc"], w["a_init"], w["a_final"], w["n_steps"]).run(ost, 10)
    nf = 4 * w["nc"]
    kg, pg, ng = sim.power_spectrum(nf, nf // 2)
    ko, po, no = power.power_spectrum(ost.codes(), nf, nf // 2, nf)
    np.testing.assert_array_equal(ng, no)
    rel = np.abs(pg / po - 1)
    assert rel.max() < 5e-3, rel
    sim.close()


def test_power_spectrum_kernel_matches_oracle():
    need_gpu()
    rng = np.random.default_rng(9)
    sim = make_sim(np=32, nc=16, a_init=0.1, a_final=0.5, n_steps=2)
    Q = synth.clustered_codes(rng, sim.cfg.n, 16)
    sim.load_qp(Q, synth.momenta(rng, sim.cfg.n), 0.3)
    for nmesh in (64, 32, 16):
        kg, pg, ng = sim.power_spectrum(nmesh, nmesh // 2)
        ko, po, no = power.power_spectrum(Q.T.astype(np.int64), nmesh, nmesh // 2, 64)
        np.testing.assert_array_equal(ng, no)
        np.testing.assert_allclose(kg, ko, rtol=1e-12)
        np.testing.assert_allclose(pg, po, rtol=2e-5)
    sim.close()


def _state_bytes(sim):
    st = sim.fetch_state()
    rec = np.concatenate([st["streams"][:3], st["streams"][3:]]).T
    return (st["counts"].copy(), st["vc"].copy(), st["scalars"]["sigma"],
            cell_sorted_records(st["counts"], rec))


def test_runs_are_bitwise_deterministic_and_resume():
    need_gpu()
    w = synth.WORKLOADS["ragged_32"]
    outs = []
    for _ in range(2):
        sim = make_sim(**w)
        sim.ic_zeldovich(3, **synth.IC_SPECTRUM)
        sim.step(6)
        outs.append(_state_bytes(sim))
        sim.close()
    for a, b in zip(outs[0], outs[1]):
        np.testing.assert_array_equal(a, b)
    # 3 steps, checkpoint to host, new sim, load, 3 steps == 6 steps
    sim = make_sim(**w)
    sim.ic_zeldovich(3, **synth.IC_SPECTRUM)
    sim.step(3)
    ck = sim.fetch_state()
    sim.close()
    sim = make_sim(**w)
    sim.load_state(ck)
    sim.step(3)
    for a, b in zip(outs[0], _state_bytes(sim)):
        np.testing.assert_array_equal(a, b)
    sim.close()


def test_graph_mode_and_shared_tables_are_bitwise_identical():
    # a sim that copies its force tables from a donor and replays captured
    # steps must evolve exactly like an eager sim that built its own tables
    need_gpu()
    from paper_2003_03931_gb300.sim import SimConfig, Simulation
    w = synth.WORKLOADS["ragged_32"]
    eager = make_sim(**w)
    eager.ic_zeldovich(9, **synth.IC_SPECTRUM)
    eager.step(5)
    ref = _state_bytes(eager)
    import torch
    with pytest.raises(Exception, match="created stream"):
        eager.graph_mode(True)     # eager runs on the default stream
    graph = Simulation(SimConfig(**w), device="cuda:0", stream=torch.cuda.Stream("cuda:0"),
                       donor=eager)
    graph.graph_mode(True)
    graph.ic_zeldovich(9, **synth.IC_SPECTRUM)
    graph.step(2)
    graph.step(3)
    for a, b in zip(ref, _state_bytes(graph)):
        np.testing.assert_array_equal(a, b)
    assert graph.fetch_scalars()["step"] == 5
    # loading a checkpoint resets the replayed step counter
    ck = eager.fetch_state()
    graph.load_state(ck)
    graph.step(2)
    eager.step(2)
    for a, b in zip(_state_bytes(eager), _state_bytes(graph)):
        np.testing.assert_array_equal(a, b)
    eager.close()
    graph.close()


def test_refused_counts_leave_no_state():
    # counts are checked on the host before any kernel indexes with them; a
    # refused load leaves the sim without a state until a valid one is loaded
    need_gpu()
    from paper_2003_03931_gb300 import _lib
    from paper_2003_03931_gb300._lib import PMPM_EINVAL, PMPM_ESTATE, PmpmError
    w = synth.WORKLOADS["c1_32"]
    sim = make_sim(**w)
    sim.ic_zeldovich(3, **synth.IC_SPECTRUM)
    st = sim.fetch_state()
    bad = st["counts"].copy()
    bad[0] += 1                                   # adds up to N + 1
    neg = st["counts"].copy()
    neg[0] = -1                                   # adds up to N, one negative
    neg[1] += st["counts"][0] + 1
    for counts in (bad, neg):
        with pytest.raises(PmpmError) as e:
            sim._load(_lib.COUNTS, counts)
        assert e.value.code == PMPM_EINVAL
        with pytest.raises(PmpmError) as e:
            sim.step(1)
        assert e.value.code == PMPM_ESTATE
    sim.load_state(st)
    sim.step(1)
    sim.close()
