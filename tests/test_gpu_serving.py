"""GPU checks of the serving engine: each box of a mixed batch ends exactly
where it ends when run alone (same cell-sorted store, counts, sigma and
scale factor; P(k) within 1e-12, the shell sums being float64 atomics), in
every engine configuration; FIFO admission within a tight arena; and the
engine's argument and time-limit errors."""

import numpy as np
import pytest

from tests.gpu_util import cell_sorted_records, need_gpu

pytestmark = pytest.mark.gpu


def _solo(req):
    from paper_2003_03931_gb300.sim import SimConfig, Simulation
    m, nb = req.mesh()
    sim = Simulation(SimConfig(np=req.np, nc=req.nc, a_init=req.a_init, a_final=req.a_final,
                               n_steps=req.n_steps, pk_mesh_max=m, lowmem=req.lowmem),
                     device="cuda:0")
    sim.ic_zeldovich(req.seed, req.slope, req.k_c, req.rms_disp)
    sim.step(req.n_steps)
    k, pk, nm = sim.power_spectrum(m, nb)
    st = sim.fetch_state()
    sim.close()
    return k, pk, nm, st


def _mix():
    from paper_2003_03931_gb300.serve import Request
    return [Request(np=32, nc=16, n_steps=6, seed=11, slope=-1.2, want_state=True),
            Request(np=32, nc=8, n_steps=4, seed=12, slope=-1.5, want_state=True),
            Request(np=64, nc=32, n_steps=5, seed=13, slope=-1.8, want_state=True),
            Request(np=32, nc=16, n_steps=3, seed=14, slope=-1.0, want_state=True),
            Request(np=64, nc=32, n_steps=2, seed=15, slope=-2.0, want_state=True),
            Request(np=32, nc=16, n_steps=7, seed=16, slope=-1.5, pk_nmesh=64, pk_nbins=20,
                    want_state=True)]


def _large_mix():
    # the large boxes of the serving mix (128^3, 256^3 particles) next to
    # small ones, and low-memory boxes (new codes derived again by the re-encode) among them
    from paper_2003_03931_gb300.serve import Request
    return [Request(np=256, nc=128, n_steps=3, seed=21, slope=-1.5, want_state=True),
            Request(np=32, nc=16, n_steps=5, seed=22, slope=-1.2, want_state=True),
            Request(np=128, nc=64, n_steps=4, seed=23, slope=-1.8, want_state=True),
            Request(np=64, nc=32, n_steps=3, seed=24, slope=-1.5, want_state=True, lowmem=True),
            Request(np=128, nc=64, n_steps=2, seed=25, slope=-2.0, want_state=True, lowmem=True),
            Request(np=64, nc=32, n_steps=4, seed=26, slope=-1.0, want_state=True)]


def _check_against_solo(reqs, res):
    for req, r in zip(reqs, res):
        assert r.status == 0
        k, pk, nm, st = _solo(req)
        np.testing.assert_array_equal(r.nmodes, nm)
        np.testing.assert_allclose(r.k, k, rtol=1e-12)
        np.testing.assert_allclose(r.pk, pk, rtol=1e-12)
        np.testing.assert_array_equal(r.counts, st["counts"])
        a = cell_sorted_records(r.counts, r.streams.T)
        b = cell_sorted_records(st["counts"], st["streams"].T)
        np.testing.assert_array_equal(a, b)
        assert np.float32(r.sigma) == np.float32(st["scalars"]["sigma"])
        assert r.a == st["scalars"]["a"]
        assert r.particle_steps == req.n * req.n_steps
        assert r.t_arrival <= r.t_admit <= r.t_done


@pytest.mark.parametrize("kw", [
    dict(max_active=6, share_tables=True, graphs=True, priorities=True, steps_per_chunk=2),
    dict(max_active=3, share_tables=False, graphs=False, priorities=True, steps_per_chunk=1),
    dict(max_active=4, share_tables=True, graphs=True, priorities=2, steps_per_chunk=3),
])
def test_large_and_lowmem_boxes_equal_solo_runs(kw):
    need_gpu()
    from paper_2003_03931_gb300.serve import Engine, run_stream
    reqs = _large_mix()
    eng = Engine(8 << 30, **kw)
    res = run_stream(eng, reqs, timeout=600)
    stats = eng.stats()
    eng.close()
    assert stats["completed"] == len(reqs) and stats["failed"] == 0
    _check_against_solo(reqs, res)


def test_large_box_limit():
    # large_np = 128, max_large = 1: two 128^3 boxes are never resident
    # together, later small requests pass a waiting large one, and every box
    # still ends as it does alone
    need_gpu()
    from paper_2003_03931_gb300.serve import Engine, Request, run_stream
    reqs = [Request(np=128, nc=64, n_steps=4, seed=31, want_state=True),
            Request(np=128, nc=64, n_steps=3, seed=32, want_state=True),
            Request(np=32, nc=16, n_steps=3, seed=33, want_state=True),
            Request(np=64, nc=32, n_steps=2, seed=34, want_state=True),
            Request(np=128, nc=64, n_steps=2, seed=35, want_state=True),
            Request(np=32, nc=16, n_steps=4, seed=36, want_state=True)]
    eng = Engine(4 << 30, max_active=4, share_tables=True, graphs=False, priorities=1,
                 steps_per_chunk=1, large_np=128, max_large=1)
    res = run_stream(eng, reqs, timeout=600)
    eng.close()
    big = sorted((r.t_admit, r.t_done) for r in res if r.request.np == 128)
    for (a0, d0), (a1, d1) in zip(big, big[1:]):
        assert a1 >= d0 - 1e-3
    # the small requests behind the second large one did not wait for it
    second_big_admit = big[1][0]
    assert min(r.t_admit for r in res if r.request.seed in (33, 34)) < second_big_admit
    _check_against_solo(reqs, res)


def test_request_flags_are_checked():
    need_gpu()
    from paper_2003_03931_gb300 import _lib
    from paper_2003_03931_gb300.serve import Engine, Request
    eng = Engine(1 << 28, max_active=2)
    req = Request(np=32, nc=16, n_steps=2, seed=3)
    nb = req.mesh()[1]
    k, pk, nm = np.zeros(nb), np.zeros(nb), np.zeros(nb, np.int64)
    import ctypes
    r = _lib.Request(32, 16, 2, 0, 0, 2, 0.02, 1.0, 3, -1.5, np.pi / 2, 0.3, 0.0,
                     k.ctypes.data, pk.ctypes.data, nm.ctypes.data, None, None)
    rid = ctypes.c_int64()
    rc = eng.lib.pmpm_batch_submit(eng.h, ctypes.byref(r), ctypes.byref(rid))
    assert rc == _lib.PMPM_EINVAL
    eng.close()


@pytest.mark.parametrize("kw", [
    dict(max_active=4, share_tables=True, graphs=True, priorities=True, steps_per_chunk=2),
    dict(max_active=6, share_tables=True, graphs=False, priorities=False, steps_per_chunk=1,
         chunks_in_flight=3),
    dict(max_active=1, share_tables=False, graphs=False, priorities=False, steps_per_chunk=3),
])
def test_mixed_batch_equals_solo_runs(kw):
    need_gpu()
    from paper_2003_03931_gb300.serve import Engine, run_stream
    reqs = _mix()
    eng = Engine(1 << 30, **kw)
    res = run_stream(eng, reqs, timeout=300)
    stats = eng.stats()
    eng.close()
    assert stats["completed"] == len(reqs) and stats["failed"] == 0
    assert stats["table_builds"] == (3 if kw["share_tables"] else len(reqs))
    assert stats["launches"] > 0
    _check_against_solo(reqs, res)


def test_admission_within_a_tight_arena():
    need_gpu()
    from paper_2003_03931_gb300._lib import PMPM_EINVAL, PMPM_ENOMEM, PmpmError
    from paper_2003_03931_gb300.serve import Engine, Request, run_stream
    from paper_2003_03931_gb300.sim import SimConfig, workspace_bytes
    big = workspace_bytes(SimConfig(np=64, nc=32, n_steps=3, pk_mesh_max=64))
    arena = big + (4 << 20)       # one 64^3 box and its tables at a time
    reqs = [Request(np=64, nc=32, n_steps=3, seed=40 + i) for i in range(3)]
    reqs += [Request(np=32, nc=16, n_steps=3, seed=50 + i) for i in range(2)]
    eng = Engine(arena, max_active=8)
    with pytest.raises(PmpmError) as e:
        eng.submit(Request(np=128, nc=64, n_steps=3, seed=1))
    assert e.value.code == PMPM_ENOMEM
    with pytest.raises(PmpmError) as e:
        eng.submit(Request(np=32, nc=16, n_steps=3, seed=1, pk_nmesh=48))
    assert e.value.code == PMPM_EINVAL
    res = run_stream(eng, reqs, timeout=300)
    st = eng.stats()
    assert all(r.status == 0 for r in res)
    assert st["arena_peak"] <= arena and st["arena_used"] > 0   # tables stay
    # first in, first admitted
    t = [r.t_admit for r in res]
    assert t == sorted(t)
    # two 64^3 boxes never resident together
    big_runs = sorted((r.t_admit, r.t_done) for r in res if r.request.np == 64)
    for (a0, d0), (a1, d1) in zip(big_runs, big_runs[1:]):
        assert a1 >= d0 - 1e-3
    eng.close()


def test_time_limit_and_teardown_with_queued_work():
    need_gpu()
    from paper_2003_03931_gb300._lib import PMPM_ETIMEOUT, PmpmError
    from paper_2003_03931_gb300.serve import Engine, Request
    eng = Engine(1 << 28, max_active=2)
    eng.submit(Request(np=32, nc=16, n_steps=2, seed=3, arrival=eng.clock() + 3600))
    eng.submit(Request(np=32, nc=16, n_steps=2, seed=4))
    with pytest.raises(PmpmError) as e:
        eng.run(0.5)
    assert e.value.code == PMPM_ETIMEOUT
    done = eng.poll()
    assert len(done) == 1 and done[0].status == 0 and done[0].request.seed == 4
    eng.close()     # the far-future request is dropped with the engine
