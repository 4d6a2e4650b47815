"""Python handle on one PM-PM simulation (a thin wrapper over include/pmpm.h).

PyTorch supplies the device workspace and the stream; every step of the path
runs inside libpmpm.  Host arrays are numpy.
"""

import ctypes
from dataclasses import dataclass

import numpy as np

from . import _lib


@dataclass
class SimConfig:
    """Mirror of pmpm_config (include/pmpm.h)."""
    np: int                 # particles per side of the initial lattice
    nc: int                 # coarse cells per side (fine mesh 4 nc)
    a_init: float = 0.02
    a_final: float = 1.0
    n_steps: int = 20
    tile_max: int = 5       # largest tile edge in coarse cells (4 or 5)
    buffer: int = 6         # tile buffer, fine cells (Sec. IV-A.2)
    pos_bytes: int = 1
    vel_bytes: int = 1
    pk_mesh_max: int = 0
    lowmem: bool = False    # low-memory step: new momenta kept, new codes derived again
    fine_fp16: bool = False # tile spectrum stored as FP16 (PMPM_FLAG_FINE_FP16)
    omega_m: float = 0.0    # background: 0, 0 = Einstein-de Sitter; else LambdaCDM (Sec. IV-A.2)
    omega_l: float = 0.0

    def to_c(self):
        c = _lib.Config()
        c.np, c.nc, c.tile_max, c.buffer = self.np, self.nc, self.tile_max, self.buffer
        c.pos_bytes, c.vel_bytes, c.pk_mesh_max = self.pos_bytes, self.vel_bytes, self.pk_mesh_max
        c.flags = (_lib.FLAG_LOWMEM if self.lowmem else 0) | (_lib.FLAG_FINE_FP16 if self.fine_fp16 else 0)
        c.a_init, c.a_final, c.n_steps = self.a_init, self.a_final, self.n_steps
        c.omega_m, c.omega_l = self.omega_m, self.omega_l
        return c

    @property
    def n(self):
        return self.np ** 3

    @property
    def ncells(self):
        return self.nc ** 3


def split_store(raw, n, pos_bytes):
    """Position and velocity bins of a raw PMPM_STREAMS buffer."""
    raw = np.ascontiguousarray(raw).reshape(-1)
    pb = pos_bytes
    m = raw[:3 * pb * n].view(np.uint8 if pb == 1 else np.uint16).reshape(3, n)
    u = raw[3 * pb * n:].reshape(3, n)
    return m, u


def join_store(m, u):
    """The raw PMPM_STREAMS buffer of position bins m [3, N] and velocity bins u."""
    return np.concatenate([np.ascontiguousarray(m).view(np.uint8).reshape(-1),
                           np.ascontiguousarray(u, np.uint8).reshape(-1)])


def workspace_bytes(cfg):
    lib = _lib.load()
    out = ctypes.c_size_t(0)
    c = cfg.to_c()
    _lib.check(lib.pmpm_workspace_bytes(ctypes.byref(c), ctypes.byref(out)))
    return out.value


def step_factors(cfg, step):
    """(kick, drift, ic_momentum) of one step of cfg's schedule (float64,
    host only; pmpm_step_factors)."""
    lib = _lib.load()
    k, d, p = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    c = cfg.to_c()
    _lib.check(lib.pmpm_step_factors(ctypes.byref(c), step, ctypes.byref(k), ctypes.byref(d),
                                     ctypes.byref(p)))
    return k.value, d.value, p.value


def codec_tables():
    lib = _lib.load()
    T = np.zeros(256, np.float32)
    E = np.zeros(256, np.float32)
    _lib.check(lib.pmpm_codec_tables(T.ctypes.data, E.ctypes.data))
    return T, E


class Simulation:
    """One simulation on one GPU.  The workspace is a torch uint8 tensor."""

    def __init__(self, cfg, device="cuda", stream=None, workspace=None, donor=None):
        import torch
        self.cfg = cfg
        self.lib = _lib.load()
        self.device = torch.device(device)
        nbytes = workspace_bytes(cfg)
        if workspace is None:
            workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        if workspace.numel() < nbytes:
            raise ValueError("workspace too small")
        self.workspace = workspace
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        handle = ctypes.c_void_p()
        c = cfg.to_c()
        with torch.cuda.device(self.device):
            if donor is None:
                rc = self.lib.pmpm_init(ctypes.byref(c), ctypes.c_void_p(workspace.data_ptr()),
                                        nbytes, ctypes.c_void_p(self.stream.cuda_stream),
                                        ctypes.byref(handle))
            else:
                rc = self.lib.pmpm_init_like(ctypes.byref(c), ctypes.c_void_p(workspace.data_ptr()),
                                             nbytes, ctypes.c_void_p(self.stream.cuda_stream),
                                             donor.h, ctypes.byref(handle))
        _lib.check(rc, None)
        self.h = handle

    # -- lifecycle
    def close(self):
        if getattr(self, "h", None):
            self.lib.pmpm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        _lib.check(rc, self.h)

    # -- physics
    def ic_zeldovich(self, seed, slope=-1.5, k_c=np.pi / 2, rms_disp=0.3):
        self._check(self.lib.pmpm_ic_zeldovich(self.h, seed, slope, k_c, rms_disp))

    def graph_mode(self, enable=True):
        self._check(self.lib.pmpm_graph_mode(self.h, int(enable)))

    def step(self, nsteps=1):
        self._check(self.lib.pmpm_step(self.h, nsteps))

    def sync(self):
        self._check(self.lib.pmpm_sync(self.h))

    def power_spectrum(self, nmesh, nbins):
        k = np.zeros(nbins)
        pk = np.zeros(nbins)
        nm = np.zeros(nbins, np.int64)
        self._check(self.lib.pmpm_power_spectrum(self.h, nmesh, nbins, k.ctypes.data,
                                                 pk.ctypes.data, nm.ctypes.data))
        return k, pk, nm

    # -- transfers
    def _fetch(self, what, arr):
        self._check(self.lib.pmpm_fetch(self.h, what, arr.ctypes.data, arr.nbytes))
        return arr

    def fetch_streams(self):
        """The raw store: uint8 [6, N] for 1-byte positions, otherwise the
        (3 pos_bytes + 3) N bytes of include/pmpm.h's PMPM_STREAMS layout."""
        if self.cfg.pos_bytes == 1:
            return self._fetch(_lib.STREAMS, np.empty((6, self.cfg.n), np.uint8))
        return self._fetch(_lib.STREAMS, np.empty((3 * self.cfg.pos_bytes + 3) * self.cfg.n, np.uint8))

    def fetch_store(self):
        """(m [3, N] uint8 or uint16 position bins, u [3, N] uint8 velocity bins)."""
        return split_store(self.fetch_streams(), self.cfg.n, self.cfg.pos_bytes)

    def fetch_counts(self):
        return self._fetch(_lib.COUNTS, np.empty(self.cfg.ncells, np.int32))

    def fetch_vc(self):
        return self._fetch(_lib.VC, np.empty((3, self.cfg.ncells), np.float32))

    def fetch_scalars(self):
        sc = _lib.Scalars()
        self._check(self.lib.pmpm_fetch(self.h, _lib.SCALARS, ctypes.addressof(sc),
                                        ctypes.sizeof(sc)))
        return {"a": sc.a, "sigma": sc.sigma, "step": sc.step, "n": sc.n}

    def fetch_decoded(self):
        Q = self._fetch(_lib.DECODED_Q, np.empty((3, self.cfg.n), np.int32))
        P = self._fetch(_lib.DECODED_P, np.empty((3, self.cfg.n), np.float32))
        return Q, P

    def fetch_force(self):
        return self._fetch(_lib.FORCE, np.empty((3, self.cfg.n), np.float32))

    def fetch_step_qp(self):
        """New codes Q' [3, N] int32 and kicked momenta p' [3, N] float32 of
        the last step, in the storage order that step started from."""
        n = self.cfg.n
        buf = self._fetch(_lib.STEP_QP, np.empty(24 * n, np.uint8))
        return buf[:12 * n].view(np.int32).reshape(3, n), buf[12 * n:].view(np.float32).reshape(3, n)

    def fetch_tile_density(self, tile):
        """(uint32 [32, 32, 32] fine box indexed [z, y, x], origin (3,) in fine
        nodes, tile edge (3,) in fine cells) of one tile after its deposit."""
        box = np.empty((32, 32, 32), np.uint32)
        org = np.zeros(3, np.int32)
        edge = np.zeros(3, np.int32)
        self._check(self.lib.pmpm_fetch_tile_density(self.h, tile, box.ctypes.data, box.nbytes,
                                                     org.ctypes.data, edge.ctypes.data))
        return box, org, edge

    def fetch_coarse_density(self):
        return self._fetch(_lib.COARSE_DENSITY, np.empty(self.cfg.ncells, np.int64))

    def fetch_into(self, host):
        """Fetch streams, counts and v_c into preallocated host arrays (e.g.
        pinned), shaped like fetch_state()'s."""
        self._fetch(_lib.STREAMS, host["streams"])
        self._fetch(_lib.COUNTS, host["counts"])
        self._fetch(_lib.VC, host["vc"])
        return host

    def fetch_state(self):
        return {"streams": self.fetch_streams(), "counts": self.fetch_counts(),
                "vc": self.fetch_vc(), "scalars": self.fetch_scalars()}

    def _load(self, what, arr):
        arr = np.ascontiguousarray(arr)
        self._check(self.lib.pmpm_load(self.h, what, arr.ctypes.data, arr.nbytes))

    def load_scalars(self, a, sigma, step):
        sc = _lib.Scalars(a, sigma, step, self.cfg.n)
        self._check(self.lib.pmpm_load(self.h, _lib.SCALARS, ctypes.addressof(sc),
                                       ctypes.sizeof(sc)))

    def load_state(self, state):
        self._load(_lib.STREAMS, np.ascontiguousarray(state["streams"]).view(np.uint8))
        self._load(_lib.COUNTS, np.asarray(state["counts"], np.int32))
        self._load(_lib.VC, np.asarray(state["vc"], np.float32))
        sc = state["scalars"]
        self.load_scalars(sc["a"], sc["sigma"], sc["step"])

    def load_qp(self, Q, P, a, step=0):
        """Encode codes Q [3, N] int32 and momenta P [3, N] float32 (Sec. III-A)."""
        self.load_scalars(a, 1.0, step)
        buf = np.concatenate([np.ascontiguousarray(Q, np.int32).view(np.uint8).ravel(),
                              np.ascontiguousarray(P, np.float32).view(np.uint8).ravel()])
        self._check(self.lib.pmpm_load(self.h, _lib.QP, buf.ctypes.data, buf.nbytes))

    def stage_times(self, enable=True, reset=False):
        if reset:
            self._check(self.lib.pmpm_stage_times(self.h, int(enable), None, 0, None))
            return None
        t = np.zeros(6)
        nl = ctypes.c_int64(0)
        self._check(self.lib.pmpm_stage_times(self.h, int(enable), t.ctypes.data, 6,
                                              ctypes.byref(nl)))
        return t, nl.value
