"""GPU parity of the PM-PM force (Sec. II, Eq. 1): tiled fine mesh + coarse
mesh on the GPU vs the oracle's whole-box meshes, identical compressed state.
Bar: max |g - g_oracle| / |g_oracle| <= 1e-4 over particles whose |g| exceeds
1e-3 of the peak (vectors)."""

import numpy as np
import pytest

from oracle import dynamics, force
from tests.gpu_util import load_oracle_state, make_sim, need_gpu, oracle_state, vector_rel_err

pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.mark.parametrize("np_,nc,evolve", [(32, 16, 0), (32, 16, 6), (32, 32, 4), (64, 32, 3), (64, 64, 1)])
def test_force_matches_oracle(np_, nc, evolve):
    # (32, 16): 4 tiles of 16 per side; (32, 32) and (64, 32): 7 ragged tiles
    # of 16/20; evolved states are clustered; (64, 64): the coarse mesh goes
    # through the two-step register FFT (64 = 8 x 8 points)
    need_gpu()
    sim = make_sim(np=np_, nc=nc, a_init=0.02, a_final=1.0, n_steps=10)
    sim.ic_zeldovich(11)
    ost = oracle_state(sim)
    if evolve:
        ost = dynamics.Simulation(nc, 0.02, 1.0, 10).run(ost, evolve)
        load_oracle_state(sim, ost)
    g = sim.fetch_force()
    ref = force.ForceOperator(nc).particle_force(ost.codes()).T
    err = vector_rel_err(g, ref)
    assert err <= TOL, err
    # momentum: the net force vanishes up to float32 rounding
    assert np.abs(g.sum(axis=1)).max() < 1e-4 * np.abs(g).max() * np.sqrt(g.shape[1])
    sim.close()


def test_single_particle_has_no_self_force():
    need_gpu()
    sim = make_sim(np=4, nc=8, a_init=0.1, a_final=0.5, n_steps=2)
    rng = np.random.default_rng(3)
    Q = np.zeros((3, sim.cfg.n), np.int32)
    # all 64 particles at one position: the force on each is the self force, 0
    Q[:] = rng.integers(0, 8 * 256, size=(3, 1))
    sim.load_qp(Q, np.zeros((3, sim.cfg.n), np.float32), 0.3)
    g = sim.fetch_force()
    assert np.abs(g).max() < 1e-4
    sim.close()


@pytest.mark.parametrize("np_,nc,evolve", [(32, 32, 2), (64, 32, 0)])
def test_force_with_four_cell_tiles(np_, nc, evolve):
    # tile_max = 4: eight tiles of 16 fine cells per side where tile_max = 5
    # gives seven ragged ones; the force must not depend on the tiling
    need_gpu()
    sim = make_sim(np=np_, nc=nc, a_init=0.02, a_final=1.0, n_steps=10, tile_max=4)
    sim.ic_zeldovich(5)
    ost = oracle_state(sim)
    if evolve:
        ost = dynamics.Simulation(nc, 0.02, 1.0, 10).run(ost, evolve)
        load_oracle_state(sim, ost)
    g = sim.fetch_force()
    ref = force.ForceOperator(nc).particle_force(ost.codes()).T
    err = vector_rel_err(g, ref)
    assert err <= TOL, err
    sim.close()
