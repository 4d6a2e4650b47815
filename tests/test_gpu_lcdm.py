"""GPU parity in the paper's LambdaCDM background (Sec. IV-A.2: Omega_m =
0.258, flat, from z = 99): the Zel'dovich initial conditions, one step
particle by particle, and the power spectrum after 10 steps to a = 1, each
against the oracle with the same background."""

import numpy as np
import pytest

from oracle import cosmology, dynamics, ic, power
from paper_2003_03931_gb300 import synth
from tests.gpu_util import cell_sorted_records, load_oracle_state, make_sim, need_gpu, oracle_state

pytestmark = pytest.mark.gpu


def _setup(name="lcdm_32"):
    w = synth.WORKLOADS[name]
    cos = cosmology.Cosmology(w["omega_m"], w["omega_l"])
    orc = dynamics.Simulation(w["nc"], w["a_init"], w["a_final"], w["n_steps"], cosmo=cos)
    return w, cos, orc


def test_lcdm_initial_conditions_match_oracle():
    need_gpu()
    w, cos, _ = _setup()
    sim = make_sim(**w)
    sim.ic_zeldovich(5, **synth.IC_SPECTRUM)
    got = oracle_state(sim)
    ref, _, p = ic.zeldovich(5, w["np"], w["nc"], w["a_init"], cosmo=cos, **synth.IC_SPECTRUM)
    assert np.abs(got.counts.astype(int) - ref.counts).sum() <= 2
    if (got.counts == ref.counts).all():
        a = cell_sorted_records(got.counts, got.codes())
        b = cell_sorted_records(ref.counts, ref.codes())
        assert (np.abs(a - b) > 1).sum() == 0
    # sigma scales with the growing mode's momentum factor a^2 E f
    np.testing.assert_allclose(float(got.sigma), float(ref.sigma), rtol=1e-6)
    eds, _, _ = ic.zeldovich(5, w["np"], w["nc"], w["a_init"], **synth.IC_SPECTRUM)
    ratio = cos.ic_momentum_factor(w["a_init"]) / np.sqrt(w["a_init"])
    np.testing.assert_allclose(float(ref.sigma) / float(eds.sigma), ratio, rtol=1e-5)
    sim.close()


def test_lcdm_step_per_particle_matches_oracle():
    need_gpu()
    w, cos, orc = _setup()
    st, _, _ = ic.zeldovich(6, w["np"], w["nc"], w["a_init"], cosmo=cos, **synth.IC_SPECTRUM)
    st = orc.run(st, 5)
    sim = make_sim(**w)
    load_oracle_state(sim, st)
    g_gpu = sim.fetch_force().T
    sim.step(1)
    Qg, pg = sim.fetch_step_qp()
    Qg, pg = Qg.T.astype(np.int64), pg.T
    Q, p = st.codes(), st.momenta()
    g = orc.op.particle_force(Q)
    kick, drift = dynamics.step_factors(w["a_init"], w["a_final"], w["n_steps"], st.step,
                                        Q.shape[0], 4 * w["nc"], cos)
    # the device's kick with its own force, exactly
    np.testing.assert_array_equal(pg, (p + (np.float32(kick) * g_gpu).astype(np.float32))
                                  .astype(np.float32))
    Qo, po = dynamics.kick_drift(Q, p, g, kick, drift, w["nc"])
    gn = np.linalg.norm(g, axis=1)
    tol = (kick * 1e-4 * np.maximum(gn, 1e-3 * gn.max()))[:, None] + \
        4 * np.spacing(np.abs(po).astype(np.float32))
    assert (np.abs(pg.astype(np.float64) - po) <= tol).all()
    M = w["nc"] * 256
    dq = np.mod(Qg - Qo + M // 2, M) - M // 2
    assert np.abs(dq).max() <= 1 and (dq != 0).mean() < 1e-3
    sim.close()


def test_lcdm_power_spectrum_after_ten_steps():
    need_gpu()
    w, cos, orc = _setup()
    st, _, _ = ic.zeldovich(5, w["np"], w["nc"], w["a_init"], cosmo=cos, **synth.IC_SPECTRUM)
    sim = make_sim(**w)
    load_oracle_state(sim, st)
    sim.step(10)
    st = orc.run(st, 10)
    nf = 4 * w["nc"]
    kg, pg, ng = sim.power_spectrum(nf, nf // 2)
    ko, po, no = power.power_spectrum(st.codes(), nf, nf // 2, nf)
    np.testing.assert_array_equal(ng, no)
    rel = np.abs(pg / po - 1)
    assert rel.max() < 5e-3, rel
    sim.close()
