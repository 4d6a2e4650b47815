"""Element-wise GPU parity of one PM-PM step against the oracle (Sec. II,
Sec. III-A), from states the oracle generated and evolved itself:

* every particle's drifted code Q' and kicked momentum p' (fetched before the
  re-encode) against the oracle's kick and drift of the same particle;
* the re-encoded store of the default and of the low-memory step against the
  oracle's re-encode: counts, v_c, sigma and cell-sorted records;
* one tile's integer fine density, node by node, against the oracle's
  whole-mesh CIC deposit (a bit-exact gate), in an ordinary, a crowded and a
  16-cell tile.

Tolerances follow from the force bar (a force within 1e-4 of the oracle's,
relative to max(|g|, 1e-3 max|g|)): the kick moves p by kick * g, so p' may
differ by kick times that bound plus float32 rounding, and a drift rounding
floor(p' c + 1/2) may differ by one code only where the oracle's value lies
within that tolerance of a tie."""

import numpy as np
import pytest

from oracle import cic, codec, dynamics, ic
from paper_2003_03931_gb300 import synth
from tests.gpu_util import cell_sorted_records, load_oracle_state, make_sim, need_gpu, oracle_state

pytestmark = pytest.mark.gpu

FORCE_TOL = 1e-4
A_INIT, A_FINAL, N_STEPS = 0.02, 1.0, 10


def _oracle_start(np_, nc, evolve, seed=7):
    """Oracle ICs (Sec. IV-A.2) evolved `evolve` oracle steps."""
    st, _, _ = ic.zeldovich(seed, np_, nc, A_INIT, **synth.IC_SPECTRUM)
    orc = dynamics.Simulation(nc, A_INIT, A_FINAL, N_STEPS)
    return orc.run(st, evolve), orc


def _oracle_kick_drift(orc, st):
    """The oracle's step of `st` before the re-encode: codes, momenta, force,
    the factors, and the per-component momentum tolerance of the force bar."""
    Q, p = st.codes(), st.momenta()
    g = orc.op.particle_force(Q)
    n = Q.shape[0]
    kick, drift = dynamics.step_factors(A_INIT, A_FINAL, N_STEPS, st.step, n, 4 * st.nc)
    Qo, po = dynamics.kick_drift(Q, p, g, kick, drift, st.nc)
    gn = np.linalg.norm(g, axis=1)
    gref = np.maximum(gn, 1e-3 * gn.max())
    # force bar times the kick, the float32 product and sum (a few ulp)
    tolp = (kick * FORCE_TOL * gref)[:, None] + 4 * np.spacing(np.abs(po).astype(np.float32))
    return Qo, po, tolp, drift


def _near_ties(po, tolp, drift):
    """Components whose drift rounding floor(fl32(p' c) + 1/2) lies within
    the momentum tolerance of a tie (c the drift factor in codes)."""
    cd = np.float32(drift * codec.code_units_per_fine_cell(1))
    xq = (po * cd).astype(np.float32).astype(np.float64) + 0.5
    dist = np.abs(xq - np.rint(xq))
    return dist <= abs(float(cd)) * tolp + 4 * np.spacing(np.abs(xq))


def _touched_cells(Qo, ties, nc):
    """Cells a near-tie particle may end in: its oracle cell and the cell of
    its code moved one quantum either way on the tied axis."""
    B = 256
    M = nc * B
    cells = set()
    for i, d in zip(*np.nonzero(ties)):
        for delta in (-1, 0, 1):
            q = Qo[i].copy()
            q[d] = (q[d] + delta) % M
            cells.add(int(codec.flatten_cell(q // B, nc)))
    return np.array(sorted(cells), dtype=np.int64)


def _compare_store(got, ref, touched, tolp_cell, flips_max):
    """The re-encoded store `got` (sim) against the oracle's `ref`: counts
    equal outside the touched cells (and within 2 flips_max overall); in every
    untouched cell the same position bins, v_c within the momentum tolerance,
    and velocity bins within one bin (rarely different)."""
    ncell = ref.counts.size
    free = np.ones(ncell, bool)
    free[touched] = False
    dc = got.counts.astype(np.int64) - ref.counts
    assert np.abs(dc).sum() <= 2 * flips_max
    assert (dc[free] == 0).all()
    # velocity scale: every p' within tolerance
    np.testing.assert_allclose(float(got.sigma), float(ref.sigma), rtol=2e-5)
    # v_c of untouched cells: a mean of momenta within tolerance each
    dv = np.abs(got.vc.astype(np.float64) - ref.vc.astype(np.float64))
    bound = tolp_cell + 4 * np.spacing(np.abs(ref.vc).astype(np.float32)) + 2.0 ** -23
    assert (dv[free] <= bound[free]).all(), dv[free].max()
    # records of untouched cells, sorted within the cell by (m, u)
    cg = codec.cell_index_of_particles(got.counts)
    cr = codec.cell_index_of_particles(ref.counts)
    sg = free[cg]
    sr = free[cr]
    rg = np.concatenate([np.asarray(got.m, np.int64)[sg], np.asarray(got.u, np.int64)[sg]], axis=1)
    rr = np.concatenate([np.asarray(ref.m, np.int64)[sr], np.asarray(ref.u, np.int64)[sr]], axis=1)
    kg = got.counts.copy()
    kg[~free] = 0
    kr = ref.counts.copy()
    kr[~free] = 0
    a = cell_sorted_records(kg, rg)
    b = cell_sorted_records(kr, rr)
    np.testing.assert_array_equal(a[:, :3], b[:, :3])
    du = np.abs(a[:, 3:] - b[:, 3:])
    assert du.max() <= 1
    assert (du > 0).mean() < 1e-3
    return int(free.sum())


def _cell_tolerance(Qo, tolp, nc):
    """Largest momentum tolerance of the particles of each new cell, [C, 3]."""
    cell = codec.flatten_cell(Qo // 256, nc)
    out = np.zeros((nc ** 3, 3))
    np.maximum.at(out, cell, tolp)
    return out


@pytest.mark.parametrize("np_,nc,evolve", [(32, 16, 4), (64, 32, 5)])
def test_kick_and_drift_per_particle_match_oracle(np_, nc, evolve):
    need_gpu()
    st, orc = _oracle_start(np_, nc, evolve)
    sim = make_sim(np=np_, nc=nc, a_init=A_INIT, a_final=A_FINAL, n_steps=N_STEPS)
    load_oracle_state(sim, st)
    g_gpu = sim.fetch_force().T
    sim.step(1)
    Qg, pg = sim.fetch_step_qp()
    Qg = Qg.T.astype(np.int64)
    pg = pg.T
    Qo, po, tolp, drift = _oracle_kick_drift(orc, st)
    # the kick and drift arithmetic itself, exact given the device's own force:
    # p' = fl32(p + fl32(fl32(kick) g)), Q' = Q + floor(fl32(p' fl32(64 drift)) + 1/2)
    Q, p = st.codes(), st.momenta()
    kick, _ = dynamics.step_factors(A_INIT, A_FINAL, N_STEPS, st.step, Q.shape[0], 4 * nc)
    p_exp = (p + (np.float32(kick) * g_gpu).astype(np.float32)).astype(np.float32)
    np.testing.assert_array_equal(pg, p_exp)
    cd = np.float32(drift * 64)
    step_q = np.floor((pg * cd).astype(np.float32) + np.float32(0.5)).astype(np.int64)
    np.testing.assert_array_equal(Qg, np.mod(Q + step_q, nc * 256))
    # momenta, particle by particle in storage order
    dp = np.abs(pg.astype(np.float64) - po.astype(np.float64))
    assert (dp <= tolp).all(), (dp / tolp).max()
    # codes: equal except a drift rounding at a tie, by one code
    M = nc * 256
    dq = np.mod(Qg - Qo + M // 2, M) - M // 2
    assert np.abs(dq).max() <= 1
    ties = _near_ties(po, tolp, drift)
    assert (ties | (dq == 0)).all()
    assert (dq != 0).mean() < 1e-3
    # the re-encoded store against the oracle's re-encode of its own Q', p'
    ref = dynamics.encode(Qo, po, nc, sim.fetch_scalars()["a"], st.step + 1)
    got = oracle_state(sim)
    touched = _touched_cells(Qo, ties, nc)
    free = _compare_store(got, ref, touched, _cell_tolerance(Qo, tolp, nc), int(ties.sum()))
    assert free > 0.8 * nc ** 3
    # the per-particle buffer is gone once a later call reuses it
    sim.power_spectrum(4 * nc // 2, 4)
    from paper_2003_03931_gb300._lib import PMPM_ESTATE, PmpmError
    with pytest.raises(PmpmError) as e:
        sim.fetch_step_qp()
    assert e.value.code == PMPM_ESTATE
    sim.close()


@pytest.mark.parametrize("np_,nc,evolve", [(32, 16, 4), (64, 32, 5)])
def test_lowmem_step_matches_oracle(np_, nc, evolve):
    # the low-memory step (new momenta kept, new codes derived again)
    # against the oracle's step directly
    need_gpu()
    st, orc = _oracle_start(np_, nc, evolve, seed=8)
    sim = make_sim(np=np_, nc=nc, a_init=A_INIT, a_final=A_FINAL, n_steps=N_STEPS, lowmem=True)
    load_oracle_state(sim, st)
    sim.step(1)
    Qo, po, tolp, drift = _oracle_kick_drift(orc, st)
    ref = dynamics.encode(Qo, po, nc, sim.fetch_scalars()["a"], st.step + 1)
    ties = _near_ties(po, tolp, drift)
    got = oracle_state(sim)
    assert got.step == ref.step
    touched = _touched_cells(Qo, ties, nc)
    free = _compare_store(got, ref, touched, _cell_tolerance(Qo, tolp, nc), int(ties.sum()))
    assert free > 0.8 * nc ** 3
    sim.close()


def _tile_index(t, nt):
    return t[0] + nt * (t[1] + nt * t[2])


def _check_tile_density(sim, Q, nc, tile):
    box, org, edge = sim.fetch_tile_density(tile)
    nf = 4 * nc
    ref = cic.deposit(Q, nf, 1)               # int64 [z, y, x], units 2^-21
    idx = [np.mod(org[d] + np.arange(32), nf) for d in range(3)]
    sub = ref[np.ix_(idx[2], idx[1], idx[0])]
    # nodes i <= T + 12 of each axis receive every particle that reaches them
    lim = [min(32, int(edge[d]) + 13) for d in range(3)]
    np.testing.assert_array_equal(box[:lim[2], :lim[1], :lim[0]].astype(np.int64),
                                  sub[:lim[2], :lim[1], :lim[0]])
    return box, lim


@pytest.mark.parametrize("nc", [16, 32])
def test_tile_fine_density_matches_oracle(nc):
    # nc = 16: tiles of 4 coarse cells (16 fine); nc = 32: 7 tiles of 4/5 per
    # side.  A clustered state; the tile holding the densest coarse cell is
    # checked along with a corner tile and, for nc = 32, a 16-cell tile.
    need_gpu()
    rng = np.random.default_rng(21)
    np_ = 2 * nc
    n = np_ ** 3
    sim = make_sim(np=np_, nc=nc, a_init=A_INIT, a_final=A_FINAL, n_steps=N_STEPS)
    # clumps of a few thousand particles, one fine cell wide: several
    # hundred particles' weight on the densest nodes (a node overflows at 2048)
    Q = synth.clustered_codes(rng, n, nc, n_clusters=6 if nc == 16 else 24, frac=0.7, width_fine=1.0)
    sim.load_qp(Q, synth.momenta(rng, n), 0.1)
    Qn = Q.T.astype(np.int64)
    nt = -(-nc // 5)
    bounds = [(t * nc) // nt for t in range(nt + 1)]
    cells = codec.flatten_cell(Qn // 256, nc)
    dense = np.bincount(cells, minlength=nc ** 3).argmax()
    dc = codec.unflatten_cell(np.array([dense]), nc)[0]
    tdense = [int(np.searchsorted(bounds, dc[d], side="right") - 1) for d in range(3)]
    tiles = {_tile_index(tdense, nt), 0, nt ** 3 - 1}
    if nc == 32:
        small = [t for t in range(nt) if bounds[t + 1] - bounds[t] == 4]
        tiles.add(_tile_index([small[0], 0, small[-1]], nt))
    crowded = 0
    for t in sorted(tiles):
        box, lim = _check_tile_density(sim, Qn, nc, t)
        crowded = max(crowded, int(box.max()))
    # the crowded tile's densest node holds a hundred particles' weight or more
    assert crowded > 100 * 2 ** 21
    from paper_2003_03931_gb300._lib import PMPM_EINVAL, PmpmError
    with pytest.raises(PmpmError) as e:
        sim.fetch_tile_density(nt ** 3)
    assert e.value.code == PMPM_EINVAL
    sim.close()
