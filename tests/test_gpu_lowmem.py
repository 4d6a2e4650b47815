"""GPU checks of the low-memory step (PMPM_FLAG_LOWMEM): from the same state
it writes the same store as the default step (cell-sorted records, counts,
v_c, sigma bit for bit), also at 256^3 where each warp of the re-encode takes
several rows of cells; its float32 initial conditions match the oracle's like
the default ones; and the per-particle fetches it cannot serve fail cleanly."""

import numpy as np
import pytest

from oracle import ic
from paper_2003_03931_gb300 import synth
from tests.gpu_util import cell_sorted_records, make_sim, need_gpu, oracle_state

pytestmark = pytest.mark.gpu


def _state(sim):
    st = sim.fetch_state()
    rec = np.concatenate([st["streams"][:3], st["streams"][3:]]).T
    return (st["counts"].copy(), st["vc"].copy(), np.float32(st["scalars"]["sigma"]),
            cell_sorted_records(st["counts"], rec))


@pytest.mark.parametrize("name,steps", [("c1_32", 5), ("ragged_32", 4), ("c2_128", 3), ("c4sub_256", 1)])
def test_lowmem_steps_equal_default_steps(name, steps):
    need_gpu()
    w = synth.WORKLOADS[name]
    ref = make_sim(**w)
    ref.ic_zeldovich(4, **synth.IC_SPECTRUM)
    ref.step(2)
    low = make_sim(**w, lowmem=True)
    low.load_state(ref.fetch_state())
    for _ in range(steps):
        ref.step(1)
        low.step(1)
        for a, b in zip(_state(ref), _state(low)):
            np.testing.assert_array_equal(a, b)
    assert low.fetch_scalars()["step"] == ref.fetch_scalars()["step"]
    nf = 4 * w["nc"]
    for a, b in zip(ref.power_spectrum(nf // 2, nf // 4), low.power_spectrum(nf // 2, nf // 4)):
        np.testing.assert_allclose(a, b, rtol=1e-12)
    ref.close()
    low.close()


def test_lowmem_graph_replay_equals_eager():
    need_gpu()
    import torch
    from paper_2003_03931_gb300.sim import SimConfig, Simulation
    w = synth.WORKLOADS["c1_32"]
    eager = make_sim(**w, lowmem=True)
    eager.ic_zeldovich(6, **synth.IC_SPECTRUM)
    g = Simulation(SimConfig(**w, lowmem=True), device="cuda:0", stream=torch.cuda.Stream("cuda:0"))
    g.graph_mode(True)
    g.load_state(eager.fetch_state())
    eager.step(4)
    g.step(4)
    for a, b in zip(_state(eager), _state(g)):
        np.testing.assert_array_equal(a, b)
    eager.close()
    g.close()


def test_lowmem_initial_conditions_match_oracle():
    need_gpu()
    w = synth.WORKLOADS["c1_32"]
    sim = make_sim(**w, lowmem=True)
    sim.ic_zeldovich(5, **synth.IC_SPECTRUM)
    got = oracle_state(sim)
    ref, _, _ = ic.zeldovich(5, w["np"], w["nc"], w["a_init"], **synth.IC_SPECTRUM)
    # float32 transforms: codes within one quantum, rarely different
    assert np.abs(got.counts.astype(int) - ref.counts).sum() <= 4
    if (got.counts == ref.counts).all():
        a = cell_sorted_records(got.counts, got.codes())
        b = cell_sorted_records(ref.counts, ref.codes())
        assert (np.abs(a - b) > 1).sum() == 0
        assert (a != b).mean() < 1e-3
    np.testing.assert_allclose(float(got.sigma), float(ref.sigma), rtol=1e-5)
    sim.close()


def test_lowmem_refuses_per_particle_fetches():
    need_gpu()
    from paper_2003_03931_gb300._lib import PMPM_EINVAL, PmpmError
    w = synth.WORKLOADS["c1_32"]
    sim = make_sim(**w, lowmem=True)
    sim.ic_zeldovich(5, **synth.IC_SPECTRUM)
    for call in (sim.fetch_force, sim.fetch_decoded):
        with pytest.raises(PmpmError) as e:
            call()
        assert e.value.code == PMPM_EINVAL
    rng = np.random.default_rng(1)
    with pytest.raises(PmpmError) as e:
        sim.load_qp(synth.uniform_codes(rng, sim.cfg.n, w["nc"]), synth.momenta(rng, sim.cfg.n), 0.1)
    assert e.value.code == PMPM_EINVAL
    sim.step(1)     # still usable
    sim.close()
