"""The plain float32 PM comparator that bench.py times beside the library
(bench.PlainPM), run on CPU tensors: the pair force follows the periodic
1/r^2 force of the oracle beyond a few cells, the net force vanishes, and a
uniform lattice streams freely under the library's kick-drift schedule."""

import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import bench
from oracle import dynamics, kernels


def _pm(x, p=None, nf=64, n_steps=4):
    x = torch.tensor(np.asarray(x, np.float32))
    p = torch.zeros_like(x) if p is None else torch.tensor(np.asarray(p, np.float32))
    return bench.PlainPM(x, p, nf, 0.1, 1.0, n_steps)


def test_kernel_is_the_periodic_pair_force():
    # the sampled kernel behind the spectra: the oracle's Ewald sum of the
    # periodic pair force at every separation of the mesh, to 1e-9
    nf = 64
    S = bench.periodic_kernel_spectra(nf, "cpu", dtype=torch.float64)
    K = np.stack([torch.fft.irfftn(1j * S[d], s=(nf, nf, nf)).numpy() for d in range(3)])
    rng = np.random.default_rng(3)
    d = rng.integers(-nf // 2, nf // 2, size=(400, 3))
    d[:6] = [[1, 0, 0], [0, 2, 0], [0, 0, -3], [nf // 2, 5, 1], [7, -9, 11], [0, 0, 0]]
    got = K[:, d[:, 2] % nf, d[:, 1] % nf, d[:, 0] % nf].T
    ref = kernels.periodic_pair_kernel(d.astype(np.float64), float(nf))
    assert np.abs(got - ref).max() < 1e-9 * np.abs(ref).max()
    # the float32 spectra the step uses reproduce it to float32 resolution
    S32 = bench.periodic_kernel_spectra(nf, "cpu")
    K32 = torch.fft.irfftn(1j * S32[0].to(torch.float64), s=(nf, nf, nf)).numpy()
    assert np.abs(K32 - K[0]).max() < 1e-6 * np.abs(K[0]).max()


def test_pair_force_is_the_periodic_newtonian_force():
    # the same kernel on one mesh with CIC both ways reaches the periodic
    # pair force to a per cent or two beyond 4 cells
    rng = np.random.default_rng(5)
    nf = 64
    S = bench.periodic_kernel_spectra(nf, "cpu")
    rs, errs = [], []
    for _ in range(60):
        x0 = rng.uniform(0, nf, 3)
        r = rng.uniform(4.0, 16.0)
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        x1 = np.mod(x0 + r * n, nf)
        pm = bench.PlainPM(torch.tensor(np.stack([x0, x1], axis=1).astype(np.float32)),
                           torch.zeros(3, 2), nf, 0.1, 1.0, 4, spectra=S)
        g = pm.force().numpy().astype(np.float64)
        dx = x1 - x0
        dx -= nf * np.round(dx / nf)
        ref = kernels.periodic_pair_kernel(dx[None, :], float(nf))[0]
        rs.append(r)
        errs.append(np.linalg.norm(g[:, 1] - ref) / np.linalg.norm(ref))
        # the source feels the opposite force
        assert np.allclose(g[:, 0], -g[:, 1], rtol=1e-3, atol=1e-6 * np.abs(g).max())
    rs, errs = np.array(rs), np.array(errs)
    print("max rel err r>=8: %.4f, r<8: %.4f" % (errs[rs >= 8].max(), errs[rs < 8].max()))
    assert errs[rs >= 8].max() < 0.02, errs[rs >= 8].max()
    assert errs[rs < 8].max() < 0.06, errs[rs < 8].max()


def test_net_force_vanishes():
    rng = np.random.default_rng(6)
    g = _pm(rng.uniform(0, 64, (3, 2000))).force().numpy().astype(np.float64)
    assert np.abs(g.sum(axis=1)).max() < 1e-5 * np.abs(g).sum(axis=1).max()


def test_uniform_lattice_streams_freely():
    nf, n_steps = 32, 4
    q = (np.arange(nf) + 0.5).astype(np.float32)
    x = np.stack(np.meshgrid(q, q, q, indexing="ij")).reshape(3, -1)
    v = np.array([0.3, -0.2, 0.1], np.float32)
    pm = _pm(x, np.repeat(v[:, None], x.shape[1], axis=1), nf=nf, n_steps=n_steps)
    assert np.abs(pm.force().numpy()).max() < 1e-4
    xs = x.astype(np.float64)
    for n in range(n_steps):
        pm.step()
        kick, drift = dynamics.step_factors(0.1, 1.0, n_steps, n, x.shape[1], nf)
        xs = np.mod(xs + drift * v[:, None].astype(np.float64), nf)
    d = pm.x.numpy() - xs
    d -= nf * np.round(d / nf)
    assert np.abs(d).max() < 1e-3


def test_library_tile_transform_timer_runs_on_cpu():
    # the cuFFT comparator of the tile transforms, on CPU tensors: a time
    # that scales with the number of tiles
    t1 = bench.time_library_tile_transforms(64, "cpu", batch=8, reps=1)
    t2 = bench.time_library_tile_transforms(128, "cpu", batch=8, reps=1)
    assert t1 > 0 and t2 > 0 and math.isfinite(t1)


def test_zeldovich_plane_wave_grows_linearly():
    # Einstein-de Sitter: x = q + a Psi(q) is exact until shell crossing.  A
    # box-scale plane wave from a = 0.05 to 0.4 (a A 2 pi / L = 0.5 at the
    # end) must grow by a_final / a_init; a wrong force constant or time
    # factor misses by more than 10%.
    n_p, nf = 32, 64
    ai, af, S = 0.05, 0.4, 16
    A = 0.5 * nf / (2 * np.pi * af)
    g1 = (np.arange(n_p) + 0.5) * (nf / n_p)
    q = np.stack(np.meshgrid(g1, g1, g1, indexing="ij")).reshape(3, -1)
    psi = np.zeros_like(q)
    psi[0] = A * np.sin(2 * np.pi * q[0] / nf)
    x = np.mod(q + ai * psi, nf)
    pm = bench.PlainPM(torch.tensor(x.astype(np.float32)), torch.tensor((ai ** 1.5 * psi).astype(np.float32)),
                       nf, ai, af, S)
    for _ in range(S):
        pm.step()
    disp = pm.x.numpy().astype(np.float64)[0] - q[0]
    disp -= nf * np.round(disp / nf)
    shape = np.sin(2 * np.pi * q[0] / nf)
    amp = disp @ shape / (shape @ shape)
    assert 0.97 < amp / (af * A) < 1.01, amp / (af * A)
    assert np.abs(disp - af * A * shape).max() < 0.03 * af * A


def test_run_plain_pm_continues_the_schedule(monkeypatch):
    # bench's hook on CPU: a stand-in sim at the end of its own schedule;
    # the comparator continues from the current a without running off it
    class FakeSim:
        device = "cpu"

        def fetch_decoded(self):
            rng = np.random.default_rng(1)
            return (rng.integers(0, 16 * 256, size=(3, 512)).astype(np.int32),
                    rng.normal(size=(3, 512)).astype(np.float32))

        def fetch_scalars(self):
            return {"a": 1.0, "step": 10}

    class Cfg:
        nc, n, pos_bytes, a_init, a_final, n_steps = 16, 512, 1, 0.02, 1.0, 10

    class FakeEvent:
        def __init__(self, enable_timing=True):
            self.t = 0.0

        def record(self):
            import time
            self.t = time.perf_counter()

        def synchronize(self):
            pass

        def elapsed_time(self, other):
            return (other.t - self.t) * 1000.0 + 1e-3

    monkeypatch.setattr(torch.cuda, "Event", FakeEvent)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a: None)
    out = bench.run_plain_pm(Cfg(), FakeSim(), 3, 1)
    assert out["value"] > 0 and out["steps"] == 3 and out["bytes_per_particle"] == 24
