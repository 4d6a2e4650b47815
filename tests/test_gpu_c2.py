"""The 128^3-particle workload against the oracle (64^3 coarse cells, 256^3
fine cells, 8^3 tiles, seeded power-law Zel'dovich ICs, 20 steps a = 0.02 ->
1 equal in log a): the whole-box force per particle at the start and at the
end (Sec. II, Eq. 1), and the power spectrum after the 20 steps (Sec. IV-D)
within 0.5% per k-bin.  Both sides start from the oracle's initial
conditions; the oracle takes about 12 s per step on one core."""

import numpy as np
import pytest

from oracle import dynamics, force, ic, power
from paper_2003_03931_gb300 import synth
from tests.gpu_util import load_oracle_state, make_sim, need_gpu, vector_rel_err

pytestmark = pytest.mark.gpu


def test_c2_128_force_and_power_spectrum_after_20_steps():
    need_gpu()
    w = synth.WORKLOADS["c2_128"]
    nc, n_steps = w["nc"], w["n_steps"]
    st, _, _ = ic.zeldovich(3, w["np"], nc, w["a_init"], **synth.IC_SPECTRUM)
    sim = make_sim(**w)
    load_oracle_state(sim, st)
    orc = dynamics.Simulation(nc, w["a_init"], w["a_final"], n_steps)
    # whole-box force at the initial state
    err0 = vector_rel_err(sim.fetch_force(), orc.op.particle_force(st.codes()).T)
    assert err0 <= 1e-4, err0
    sim.step(n_steps)
    ost = orc.run(st, n_steps)
    nf = 4 * nc
    kg, pg, ng = sim.power_spectrum(nf, nf // 2)
    ko, po, no = power.power_spectrum(ost.codes(), nf, nf // 2, nf)
    np.testing.assert_array_equal(ng, no)
    np.testing.assert_allclose(kg, ko, rtol=1e-12)
    rel = np.abs(pg / po - 1)
    assert rel.max() < 5e-3, (rel.max(), int(rel.argmax()))
    # whole-box force at the clustered end state (the oracle's, loaded)
    load_oracle_state(sim, ost)
    err1 = vector_rel_err(sim.fetch_force(), force.ForceOperator(nc).particle_force(ost.codes()).T)
    assert err1 <= 1e-4, err1
    sim.close()
