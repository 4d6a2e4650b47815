"""ctypes view of libpmpm.so (the C ABI declared in include/pmpm.h).

Argument marshalling only.  Loading fails loudly when the library has not
been built; there is no fallback implementation.
"""

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpmpm.so")

PMPM_OK = 0
PMPM_EINVAL = -1
PMPM_ENOMEM = -2
PMPM_ECUDA = -3
PMPM_EOVERFLOW = -4
PMPM_ECOUNT = -5
PMPM_ESTATE = -6
PMPM_ETIMEOUT = -7

STREAMS = 1
COUNTS = 2
VC = 3
SCALARS = 4
DECODED_Q = 5
DECODED_P = 6
FORCE = 7
COARSE_DENSITY = 8
QP = 9
STEP_QP = 10

FLAG_LOWMEM = 1
FLAG_FINE_FP16 = 2

ERROR_NAMES = {
    PMPM_EINVAL: "PMPM_EINVAL",
    PMPM_ENOMEM: "PMPM_ENOMEM",
    PMPM_ECUDA: "PMPM_ECUDA",
    PMPM_EOVERFLOW: "PMPM_EOVERFLOW",
    PMPM_ECOUNT: "PMPM_ECOUNT",
    PMPM_ESTATE: "PMPM_ESTATE",
    PMPM_ETIMEOUT: "PMPM_ETIMEOUT",
}

# every entry point the header declares, for the export check
EXPORTS = [
    "pmpm_workspace_bytes", "pmpm_step_factors", "pmpm_init", "pmpm_init_like", "pmpm_graph_mode",
    "pmpm_ic_zeldovich", "pmpm_step",
    "pmpm_power_spectrum", "pmpm_fetch", "pmpm_fetch_tile_density", "pmpm_load", "pmpm_sync",
    "pmpm_stage_times",
    "pmpm_destroy", "pmpm_last_error", "pmpm_codec_tables", "pmpm_power_spectrum_noalloc",
    "pmpm_noalloc_last_error",
    "pmpm_arena_create", "pmpm_arena_alloc", "pmpm_arena_free", "pmpm_arena_stats",
    "pmpm_arena_destroy", "pmpm_batch_create", "pmpm_batch_submit", "pmpm_batch_progress",
    "pmpm_batch_run", "pmpm_batch_poll", "pmpm_batch_clock", "pmpm_batch_get_stats",
    "pmpm_batch_destroy", "pmpm_batch_last_error", "pmpm_abi_sizes", "pmpm_probe_fma",
]
NO_RC = ("pmpm_destroy", "pmpm_last_error", "pmpm_noalloc_last_error", "pmpm_arena_destroy",
         "pmpm_batch_destroy", "pmpm_batch_last_error", "pmpm_batch_clock")


class Config(ctypes.Structure):
    _fields_ = [
        ("np", ctypes.c_int32),
        ("nc", ctypes.c_int32),
        ("tile_max", ctypes.c_int32),
        ("buffer", ctypes.c_int32),
        ("pos_bytes", ctypes.c_int32),
        ("vel_bytes", ctypes.c_int32),
        ("pk_mesh_max", ctypes.c_int32),
        ("flags", ctypes.c_int32),
        ("a_init", ctypes.c_double),
        ("a_final", ctypes.c_double),
        ("n_steps", ctypes.c_int32),
        ("reserved2", ctypes.c_int32), ("omega_m", ctypes.c_double), ("omega_l", ctypes.c_double),
    ]


class Scalars(ctypes.Structure):
    _fields_ = [
        ("a", ctypes.c_double),
        ("sigma", ctypes.c_double),
        ("step", ctypes.c_int64),
        ("n", ctypes.c_int64),
    ]


class Request(ctypes.Structure):
    _fields_ = [
        ("np", ctypes.c_int32), ("nc", ctypes.c_int32), ("n_steps", ctypes.c_int32),
        ("pk_nmesh", ctypes.c_int32), ("pk_nbins", ctypes.c_int32), ("flags", ctypes.c_int32),
        ("a_init", ctypes.c_double), ("a_final", ctypes.c_double), ("seed", ctypes.c_uint64),
        ("slope", ctypes.c_double), ("k_c", ctypes.c_double), ("rms_disp", ctypes.c_double),
        ("arrival", ctypes.c_double),
        ("k", ctypes.c_void_p), ("pk", ctypes.c_void_p), ("nmodes", ctypes.c_void_p),
        ("streams", ctypes.c_void_p), ("counts", ctypes.c_void_p),
    ]


class Result(ctypes.Structure):
    _fields_ = [
        ("id", ctypes.c_int64), ("status", ctypes.c_int32), ("reserved", ctypes.c_int32),
        ("t_arrival", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double),
        ("a", ctypes.c_double), ("sigma", ctypes.c_double), ("particle_steps", ctypes.c_int64),
    ]


class BatchConfig(ctypes.Structure):
    _fields_ = [
        ("max_active", ctypes.c_int32), ("share_tables", ctypes.c_int32),
        ("graphs", ctypes.c_int32), ("priorities", ctypes.c_int32),
        ("steps_per_chunk", ctypes.c_int32), ("chunks_in_flight", ctypes.c_int32),
        ("large_np", ctypes.c_int32), ("max_large", ctypes.c_int32),
    ]


class BatchStats(ctypes.Structure):
    _fields_ = [
        ("submitted", ctypes.c_int64), ("admitted", ctypes.c_int64),
        ("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
        ("table_builds", ctypes.c_int64), ("launches", ctypes.c_int64),
        ("particle_steps", ctypes.c_int64), ("active", ctypes.c_int64),
        ("arena_used", ctypes.c_size_t), ("arena_peak", ctypes.c_size_t),
    ]


# binding structs in the order pmpm_abi_sizes reports them
ABI_STRUCTS = [Config, Scalars, Request, Result, BatchConfig, BatchStats]


class PmpmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None


def load():
    """Load libpmpm.so once; raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built; run paper_2003_03931_gb300/build.py "
                          "(or __graft_entry__.build())")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.c_void_p
    lib.pmpm_workspace_bytes.argtypes = [ctypes.POINTER(Config), ctypes.POINTER(ctypes.c_size_t)]
    lib.pmpm_init.argtypes = [ctypes.POINTER(Config), P, ctypes.c_size_t, P, ctypes.POINTER(P)]
    lib.pmpm_init_like.argtypes = [ctypes.POINTER(Config), P, ctypes.c_size_t, P, P,
                                   ctypes.POINTER(P)]
    lib.pmpm_graph_mode.argtypes = [P, ctypes.c_int32]
    lib.pmpm_ic_zeldovich.argtypes = [P, ctypes.c_uint64, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double]
    lib.pmpm_step.argtypes = [P, ctypes.c_int32]
    lib.pmpm_power_spectrum.argtypes = [P, ctypes.c_int32, ctypes.c_int32, P, P, P]
    lib.pmpm_fetch.argtypes = [P, ctypes.c_int32, P, ctypes.c_size_t]
    lib.pmpm_load.argtypes = [P, ctypes.c_int32, P, ctypes.c_size_t]
    lib.pmpm_fetch_tile_density.argtypes = [P, ctypes.c_int32, P, ctypes.c_size_t, P, P]
    D = ctypes.POINTER(ctypes.c_double)
    lib.pmpm_step_factors.argtypes = [ctypes.POINTER(Config), ctypes.c_int32, D, D, D]
    lib.pmpm_sync.argtypes = [P]
    lib.pmpm_stage_times.argtypes = [P, ctypes.c_int32, P, ctypes.c_int32, P]
    lib.pmpm_destroy.argtypes = [P]
    lib.pmpm_destroy.restype = None
    lib.pmpm_last_error.argtypes = [P]
    lib.pmpm_last_error.restype = ctypes.c_char_p
    lib.pmpm_codec_tables.argtypes = [P, P]
    lib.pmpm_power_spectrum_noalloc.argtypes = [ctypes.c_int32, ctypes.c_int64, P, P, P, P,
                                                ctypes.c_int32, ctypes.c_int32, P, P, P, P]
    lib.pmpm_noalloc_last_error.argtypes = []
    lib.pmpm_noalloc_last_error.restype = ctypes.c_char_p
    S = ctypes.c_size_t
    lib.pmpm_arena_create.argtypes = [S, ctypes.POINTER(P)]
    lib.pmpm_arena_alloc.argtypes = [P, S, ctypes.POINTER(S)]
    lib.pmpm_arena_free.argtypes = [P, S]
    lib.pmpm_arena_stats.argtypes = [P, ctypes.POINTER(S), ctypes.POINTER(S),
                                     ctypes.POINTER(ctypes.c_int64)]
    lib.pmpm_arena_destroy.argtypes = [P]
    lib.pmpm_arena_destroy.restype = None
    lib.pmpm_batch_create.argtypes = [ctypes.POINTER(BatchConfig), P, S, ctypes.POINTER(P)]
    lib.pmpm_probe_fma.argtypes = [P, ctypes.c_int64, P, ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(ctypes.c_float)]
    lib.pmpm_batch_submit.argtypes = [P, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_int64)]
    lib.pmpm_batch_progress.argtypes = [P, ctypes.POINTER(ctypes.c_int32)]
    lib.pmpm_batch_run.argtypes = [P, ctypes.c_double]
    lib.pmpm_batch_poll.argtypes = [P, ctypes.POINTER(Result), ctypes.c_int32,
                                    ctypes.POINTER(ctypes.c_int32)]
    lib.pmpm_batch_clock.argtypes = [P]
    lib.pmpm_batch_clock.restype = ctypes.c_double
    lib.pmpm_batch_get_stats.argtypes = [P, ctypes.POINTER(BatchStats)]
    lib.pmpm_batch_destroy.argtypes = [P]
    lib.pmpm_batch_destroy.restype = None
    lib.pmpm_batch_last_error.argtypes = [P]
    lib.pmpm_batch_last_error.restype = ctypes.c_char_p
    lib.pmpm_abi_sizes.argtypes = [ctypes.POINTER(ctypes.c_int64), ctypes.c_int32]
    for name in EXPORTS:
        if name not in NO_RC:
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def check(rc, handle=None):
    if rc != PMPM_OK:
        msg = load().pmpm_last_error(handle)
        raise PmpmError(rc, msg.decode() if msg else "")
