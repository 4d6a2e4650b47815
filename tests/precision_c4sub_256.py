"""Precision of each storage format on the 256^3-particle sub-run (128^3
coarse cells, 512^3 fine cells, Zel'dovich ICs of seed 1, 20 steps a = 0.02
-> 1 equal in log a), each against the FP64 oracle of the same format:

* 1-byte positions (Eq. 2, 6 bytes per particle);
* 2-byte positions (Sec. III-A's 2-byte option, 9 bytes per particle);
* 1-byte positions with the tile spectrum stored as FP16 (the FP16-storage
  option; FP32 arithmetic), when the library offers it.

For each: the force at the initial state (max and rms of |g - g_oracle| /
|g_oracle| over particles with |g_oracle| > 1e-3 max, and the same over all
particles relative to the rms force) and P(k) after the 20 steps on the
512^3 fine mesh (largest |P / P_oracle - 1| below k = 0.5 and over all
shells).  The oracle's two runs (1- and 2-byte initial conditions) go in
parallel processes; the oracle also gives the format's own effect, the 1-byte
P(k) against the 2-byte one.

    python -m tests.precision_c4sub_256 [--steps 20] [--out result.json]

Measurement only (the oracle takes about 45 s per step here); it is not
collected by pytest."""

import argparse
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

NP, NC, A0, A1 = 256, 128, 0.02, 1.0
SEED = 1
NF = 4 * NC


def _oracle_worker(pos_bytes, steps, n_schedule, workdir):
    """Oracle run of one format: ICs (saved for the GPU), force at the ICs,
    `steps` steps, final P(k) on the fine mesh."""
    sys.path.insert(0, ROOT)
    from oracle import dynamics, force, ic, power
    from paper_2003_03931_gb300 import synth
    t0 = time.time()
    st, _, _ = ic.zeldovich(SEED, NP, NC, A0, pos_bytes=pos_bytes, **synth.IC_SPECTRUM)
    np.savez(os.path.join(workdir, f"ic_{pos_bytes}.npz"), counts=st.counts, m=st.m, u=st.u,
             vc=st.vc, sigma=np.float32(st.sigma), a=st.a)
    g0 = force.ForceOperator(NC, pos_bytes).particle_force(st.codes())
    np.save(os.path.join(workdir, f"g0_{pos_bytes}.npy"), g0.astype(np.float64))
    sim = dynamics.Simulation(NC, A0, A1, n_schedule, pos_bytes)
    st = sim.run(st, steps)
    k, pk, nm = power.power_spectrum(st.codes(), NF, NF // 2, NF, pos_bytes)
    np.savez(os.path.join(workdir, f"pk_{pos_bytes}.npz"), k=k, pk=pk, nmodes=nm,
             seconds=time.time() - t0)


def _wait(path, proc):
    while not os.path.exists(path):
        if not proc.is_alive() and not os.path.exists(path):
            raise RuntimeError(f"oracle worker died before writing {path}")
        time.sleep(2)
    time.sleep(1)


def _force_err(g, ref):
    nrm = np.linalg.norm(ref, axis=1)
    sel = nrm > 1e-3 * nrm.max()
    rel = np.linalg.norm(g - ref, axis=1)[sel] / nrm[sel]
    rms = np.sqrt((np.linalg.norm(g - ref, axis=1) ** 2).mean() / (nrm ** 2).mean())
    return {"max_rel": float(rel.max()), "rms_rel": float(np.sqrt((rel ** 2).mean())),
            "rms_over_rms_force": float(rms)}


def _pk_err(k, pk, pk_ref):
    rel = np.abs(pk / pk_ref - 1.0)
    return {"max_rel_k_le_0.5": float(rel[k <= 0.5].max()), "max_rel_all": float(rel.max()),
            "k_of_max": float(k[rel.argmax()])}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--out", default=None)
    ap.add_argument("--workdir", default=None,
                    help="where the oracle processes leave their arrays (default: a temporary "
                         "directory, removed at the end)")
    args = ap.parse_args(argv)
    import shutil
    import tempfile
    own = args.workdir is None
    args.workdir = tempfile.mkdtemp(prefix="pmpm_precision_") if own else args.workdir
    os.makedirs(args.workdir, exist_ok=True)
    n_schedule = 20
    # the oracle processes start before this process touches the GPU
    ctx = mp.get_context("spawn")
    procs = {pb: ctx.Process(target=_oracle_worker, args=(pb, args.steps, n_schedule, args.workdir))
             for pb in (1, 2)}
    for p in procs.values():
        p.start()

    from paper_2003_03931_gb300 import _lib
    from paper_2003_03931_gb300.sim import SimConfig, Simulation, join_store

    formats = [("1-byte positions", 1, False), ("2-byte positions", 2, False)]
    if hasattr(_lib, "FLAG_FINE_FP16"):
        formats.append(("1-byte positions, FP16-stored tile spectrum", 1, True))
    results = {"workload": "256^3 particles, 128^3 coarse, 512^3 fine, seed %d, %d steps a %.2f -> %.0f"
                           % (SEED, args.steps, A0, A1), "formats": {}}
    for name, pb, fp16 in formats:
        _wait(os.path.join(args.workdir, f"g0_{pb}.npy"), procs[pb])
        ic = np.load(os.path.join(args.workdir, f"ic_{pb}.npz"))
        cfg = SimConfig(np=NP, nc=NC, a_init=A0, a_final=A1, n_steps=n_schedule, pos_bytes=pb,
                        fine_fp16=fp16) if fp16 else \
            SimConfig(np=NP, nc=NC, a_init=A0, a_final=A1, n_steps=n_schedule, pos_bytes=pb)
        sim = Simulation(cfg, device="cuda:0")
        m = np.ascontiguousarray(ic["m"].T).astype(np.uint8 if pb == 1 else np.uint16)
        raw = join_store(m, ic["u"].T)
        if pb == 1:
            raw = raw.reshape(6, -1)
        sim.load_state({"streams": raw, "counts": ic["counts"], "vc": ic["vc"].T,
                        "scalars": {"a": float(ic["a"]), "sigma": float(ic["sigma"]), "step": 0}})
        g = sim.fetch_force().T.astype(np.float64)
        g0 = np.load(os.path.join(args.workdir, f"g0_{pb}.npy"))
        t = time.time()
        sim.step(args.steps)
        sim.sync()
        t = time.time() - t
        kg, pg, ng = sim.power_spectrum(NF, NF // 2)
        sim.close()
        _wait(os.path.join(args.workdir, f"pk_{pb}.npz"), procs[pb])
        ref = np.load(os.path.join(args.workdir, f"pk_{pb}.npz"))
        assert (ng == ref["nmodes"]).all()
        results["formats"][name] = {
            "bytes_per_particle": 3 * pb + 3, "force_at_ics": _force_err(g, g0),
            "pk_after_steps": _pk_err(kg, pg, ref["pk"]), "gpu_seconds_for_steps": t,
            "oracle_seconds": float(ref["seconds"])}
    r1 = np.load(os.path.join(args.workdir, "pk_1.npz"))
    r2 = np.load(os.path.join(args.workdir, "pk_2.npz"))
    results["oracle_1_byte_vs_2_byte_pk"] = _pk_err(r1["k"], r1["pk"], r2["pk"])
    for p in procs.values():
        p.join()
    if own:
        shutil.rmtree(args.workdir, ignore_errors=True)
    text = json.dumps(results, indent=1)
    print(text)
    if args.out:
        with open(args.out, "w") as f:
            f.write(text + "\n")


if __name__ == "__main__":
    main()
