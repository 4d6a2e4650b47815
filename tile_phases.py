"""Per-phase clock breakdown of the tile pass: a measurement tool beside
bench.py (the library itself is not built with it).

Builds a second copy of the library with -DPMPM_PHASE_CLOCKS, in which
thread 0 of every tile CTA stamps clock64() after each block barrier of the
tile pass, runs a box, and prints the mean cycles per phase over the first
4096 tiles of the chosen steps:

    python tile_phases.py [--workload c3_512] [--steps 1 10 20]
"""

import argparse
import ctypes
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
PKG = os.path.join(ROOT, "paper_2003_03931_gb300")
PROF_LIB = os.path.join(PKG, "_build_phases", "libpmpm_phases.so")

# stamp k closes phase k - 1; names follow the kernel's phase order
PHASES = ["prologue (loads, zero)", "halo scan + cell maps", "deposit + long-range gather",
          "forward x (R2C)", "forward y", "forward z",
          "Green x + inverse z", "inverse y (x force)", "inverse x (x force)", "interpolate x",
          "Green y + inverse z", "inverse y (y force)", "inverse x (y force)", "interpolate y",
          "Green z + inverse z", "inverse y (z force)", "inverse x (z force)",
          "interpolate z + kick + drift"]
MARKS = [0, 1, 2, 3, 4, 5, 7, 8, 9, 10, 11, 12, 13, 14, 15, 16, 17, 18, 19]
N_MARKS = 24


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="c3_512")
    ap.add_argument("--steps", type=int, nargs="+", default=[1, 10, 20])
    args = ap.parse_args(argv)
    from paper_2003_03931_gb300 import build
    build.build(defines=("PMPM_PHASE_CLOCKS",), lib=PROF_LIB,
                build_dir=os.path.join(PKG, "_build_phases"))
    from paper_2003_03931_gb300 import _lib
    _lib.LIB_PATH = PROF_LIB
    from paper_2003_03931_gb300 import synth
    from paper_2003_03931_gb300.sim import SimConfig, Simulation
    w = dict(synth.WORKLOADS[args.workload])
    w["n_steps"] = max(w["n_steps"], max(args.steps) + 1)
    sim = Simulation(SimConfig(**w))
    sim.ic_zeldovich(1, **synth.IC_SPECTRUM)
    sim.lib.pmpm_debug_phases.argtypes = [ctypes.c_void_p, ctypes.c_int]
    for step in sorted(args.steps):
        while sim.fetch_scalars()["step"] < step:
            sim.step(1)
        sim.step(1)
        sim.sync()
        buf = np.zeros(4096 * N_MARKS, np.uint64)
        sim.lib.pmpm_debug_phases(buf.ctypes.data, buf.size)
        b = buf.reshape(4096, N_MARKS).astype(np.int64)
        b = b[b[:, 19] > 0]
        d = np.diff(b[:, MARKS], axis=1)
        tot = b[:, 19] - b[:, 0]
        print(f"step {step}: {len(b)} tiles, cycles per tile mean {tot.mean():.0f} max {tot.max():.0f}")
        for i, name in enumerate(PHASES):
            print(f"  {name:32s} {d[:, i].mean():9.0f}  ({100 * d[:, i].mean() / tot.mean():4.1f}%)")
    sim.close()


if __name__ == "__main__":
    sys.exit(main())
