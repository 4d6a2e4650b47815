"""The FP16 tile-spectrum storage option (PMPM_FLAG_FINE_FP16; Sec. III-A's
compact storage carried over to the fine-mesh field, float32 arithmetic)
against the oracle: it is exempt from the 1e-4 force bar, so the test
states the error it reaches (max and rms over the whole box, 32^3 on a
clustered state and 64^3 at the start) and P(k) after 10 steps.  It must also leave the
particle format untouched: decode, encode and the integer densities are the
default step's."""

import numpy as np
import pytest

from oracle import dynamics, force, ic, power
from paper_2003_03931_gb300 import synth
from tests.gpu_util import load_oracle_state, make_sim, need_gpu, vector_rel_err

pytestmark = pytest.mark.gpu

# Stated error of the option, from GB300 runs: the force is off by 2e-4 to
# 3e-4 of itself in the rms and by up to about 1e-2 at single particles with
# small forces (1.15e-2 at 64^3 from the ICs, 3.4e-3 on the clustered 32^3
# state, 3.8e-2 at 256^3 from the ICs); P(k) after 10 steps within 5e-3.
FORCE_TOL_FP16 = 2.5e-2
FORCE_RMS_TOL_FP16 = 1e-3
PK_TOL_FP16 = 1e-2


def _rms_rel(g, ref):
    nrm = np.linalg.norm(ref, axis=0)
    return np.sqrt((np.linalg.norm(g - ref, axis=0) ** 2).mean() / (nrm ** 2).mean())


@pytest.mark.parametrize("np_,nc,evolve", [(32, 16, 6), (64, 32, 0)])
def test_fp16_tile_storage_force_error(np_, nc, evolve):
    need_gpu()
    st, _, _ = ic.zeldovich(11, np_, nc, 0.02, **synth.IC_SPECTRUM)
    if evolve:
        st = dynamics.Simulation(nc, 0.02, 1.0, 10).run(st, evolve)
    ref = force.ForceOperator(nc).particle_force(st.codes()).T
    errs, rms = {}, {}
    for fp16 in (False, True):
        sim = make_sim(np=np_, nc=nc, a_init=0.02, a_final=1.0, n_steps=10, fine_fp16=fp16)
        load_oracle_state(sim, st)
        g = sim.fetch_force()
        errs[fp16] = vector_rel_err(g, ref)
        rms[fp16] = _rms_rel(g, ref)
        sim.close()
    print("force max / rms rel err: fp32 %.2e / %.2e, fp16 storage %.2e / %.2e"
          % (errs[False], rms[False], errs[True], rms[True]))
    assert errs[False] <= 1e-4
    assert errs[True] <= FORCE_TOL_FP16
    assert rms[True] <= FORCE_RMS_TOL_FP16


def test_fp16_tile_storage_power_spectrum_after_ten_steps():
    need_gpu()
    w = synth.WORKLOADS["c1_32"]
    st, _, _ = ic.zeldovich(5, w["np"], w["nc"], w["a_init"], **synth.IC_SPECTRUM)
    sim = make_sim(**w, fine_fp16=True)
    load_oracle_state(sim, st)
    sim.step(10)
    ost = dynamics.Simulation(w["nc"], w["a_init"], w["a_final"], w["n_steps"]).run(st, 10)
    nf = 4 * w["nc"]
    kg, pg, ng = sim.power_spectrum(nf, nf // 2)
    ko, po, no = power.power_spectrum(ost.codes(), nf, nf // 2, nf)
    np.testing.assert_array_equal(ng, no)
    rel = np.abs(pg / po - 1)
    print("P(k) after 10 steps, fp16 storage: max rel %.2e" % rel.max())
    assert rel.max() < PK_TOL_FP16, rel
    # the coarse density (the particle format) is untouched by the option
    ref = make_sim(**w)
    ref.load_state(sim.fetch_state())
    np.testing.assert_array_equal(ref.fetch_coarse_density(), sim.fetch_coarse_density())
    ref.close()
    sim.close()


def test_fp16_with_lowmem_is_refused():
    need_gpu()
    from paper_2003_03931_gb300._lib import PMPM_EINVAL, PmpmError
    with pytest.raises(PmpmError) as e:
        make_sim(np=32, nc=16, lowmem=True, fine_fp16=True)
    assert e.value.code == PMPM_EINVAL
