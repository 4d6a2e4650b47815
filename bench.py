#!/usr/bin/env python3
"""Benchmark of the PM-PM step (particle-steps/s) on GB300.

Headline workload: 2048^3 particles (51.5 GB at 6 bytes per particle) on
1024^3 coarse cells and a 4096^3 fine mesh in tiles of 16/20 fine cells + a
6-cell buffer, stepped by the low-memory step (one tile pass per step, the
new momenta kept in HBM and the new codes derived again by the re-encode) on
one GPU; Zel'dovich ICs from a seeded power-law spectrum; a = 0.02 -> 1 over
all steps.  Beside it the line carries the same measurement at 512^3
particles (default step, one tile pass), the plain float32 full-mesh PM with
the same total force kernel at 512^3 ("vs plain GPU form"; at 2048^3 its
mesh alone would not fit), the measured FP32 FMA peak that the tile passes'
roofline divides by, the tile transforms done by cuFFT, the FP64 oracle on
the host cores, and the serving measurement (a mixed stream of whole-box
requests through the batched engine against sequential plain stepping).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank evolves its own box (independent replicas, weak
scaling); value is the particle-steps of all ranks over the slowest rank's
time.  --impl reference times the FP64 oracle on the host cores instead.
"""

import os
import re

# separate hardware queues for the serving engine's per-box streams; must be
# set before the CUDA context exists
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

import argparse
import hashlib
import json
import math
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PMPM particle-steps/s"
UNIT = "particle-steps/s"
SM_COUNT = 152
FP32_LANES_PER_SM = 128
TILE_FFT = 32
TILE_FILES = ["paper_2003_03931_gb300/csrc/tile_core.cuh", "paper_2003_03931_gb300/csrc/regfft.cuh",
              "paper_2003_03931_gb300/csrc/tile.cu", "paper_2003_03931_gb300/csrc/common.cuh"]


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="c4_2048")
    ap.add_argument("--side-workload", default="c3_512",
                    help="a second box measured beside the headline (one GPU; empty: none)")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serving", type=int, default=120,
                    help="requests in the serving measurement (0: skip)")
    ap.add_argument("--serving-rates", default="0.5,1.0,1.5",
                    help="Poisson arrival rates for the latency runs, as fractions of the "
                         "sequential capacity (comma list; empty: skip)")
    ap.add_argument("--serving-only", action="store_true")
    ap.add_argument("--no-fma-probe", action="store_true",
                    help="divide by the lanes x clock FP32 peak instead of the measured one")
    ap.add_argument("--no-library-fft", action="store_true")
    ap.add_argument("--plain-pm", type=int, default=3, metavar="STEPS",
                    help="steps of the plain float32 full-mesh PM comparator (0: skip)")
    return ap.parse_args(argv)


# ------------------------------------------------------------------ helpers

def tile_flops_per_launch(nc, tile_max=5):
    """Algorithmic FLOPs of one tile pass: per tile one real 32^3 forward
    transform and three real inverse transforms, 2.5 M log2 M each
    (M = 32^3 points), over all tiles."""
    nt = -(-nc // tile_max)
    m = TILE_FFT ** 3
    return 4 * 2.5 * m * math.log2(m) * nt ** 3


def fp32_peak_tflops(sm_mhz, sms=SM_COUNT):
    """SMs x 128 FP32 lanes x 2 FLOP (FMA) x SM clock."""
    return sms * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12


# Algorithmic HBM bytes of the memory-bound stages: (per particle, per coarse
# cell), the least each stage must move.
HBM_STAGE_BYTES = {
    # position bins in; counts and offsets in, int64 density out
    "coarse_deposit": (3, 20),
    # density in and spectrum out, spectrum in and F_l out (one pass each way)
    "coarse_fft_green": (0, 36),
    # counts and momentum sums in; offsets and v_c out
    "hist_scan_cell_means": (0, 48),
    "scan_cell_means": (0, 48),
    # per cell: counts and momentum sums in (the cell part of the dispersion)
    "dispersion": (0, 28),
    "cell_moments_sigma": (0, 28),
    # new codes and momenta in, store out; v_c and offsets in
    "encode_scatter": (30, 20),
    # low-memory re-encode: old position bins and new momenta in, store out;
    # old offsets, new offsets and v_c in
    "reencode_scatter": (21, 28),
}


def stage_rooflines(stage_ms, n, ncells, hbm_gbs, tile_flops, fp32_tflops):
    """Per-stage achieved rate against its roofline: HBM stages in GB/s of
    algorithmic bytes over the measured copy bandwidth, tile passes in
    TFLOP/s of algorithmic FLOPs over the FP32 FMA peak."""
    out = {}
    for name, ms in stage_ms.items():
        if ms <= 0:
            continue
        if name in HBM_STAGE_BYTES:
            bp, bc = HBM_STAGE_BYTES[name]
            gb = (bp * n + bc * ncells) / 1e9
            rate = gb / (ms / 1e3)
            out[name] = {"bound": "hbm", "ms": ms, "algorithmic_gb": gb, "achieved": rate,
                         "unit": "GB/s", "peak": hbm_gbs, "frac": rate / hbm_gbs if hbm_gbs else None}
        elif name.startswith("tile"):
            rate = tile_flops / (ms / 1e3) / 1e12
            out[name] = {"bound": "alu", "ms": ms, "achieved": rate, "unit": "TFLOP/s",
                         "peak": fp32_tflops, "frac": rate / fp32_tflops}
    return out


def _code_only(text):
    """C/C++ source without comments and blank space: what the compiler sees."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def source_hash(paths):
    """Hash of the kernel sources' code (comment edits do not change it)."""
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), encoding="utf-8") as f:
            h.update(_code_only(f.read()).encode())
    return h.hexdigest()[:16]


def recorded_traffic(workload, lowmem=False):
    """DRAM bytes per tile-pass launch from the committed ncu summary, if it
    was taken on the current kernel source."""
    name = f"tile_pass_lowmem_{workload}.md" if lowmem else f"tile_pass_{workload}.md"
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    vals = {}
    with open(path) as f:
        for line in f:
            if ":" in line and line.startswith("- "):
                k, v = line[2:].split(":", 1)
                vals[k.strip()] = v.strip()
    try:
        if vals.get("source_sha") != source_hash(TILE_FILES):
            return None
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f)
    return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.dev), "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def reduce_max(value, device):
    """Max of a float over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, t_max):
    """Whole-job throughput: the units of all ranks over the slowest rank's time."""
    return world * units_per_rank / t_max


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ------------------------------------------------------------------ oracle timing

def time_oracle_steps(np_side, nc, warmup, steps):
    """Time the FP64 oracle on this host: `steps` steps of an np_side^3 box
    after `warmup` untimed ones.  Returns (particle-steps/s, seconds)."""
    from oracle import dynamics, ic
    st, _, _ = ic.zeldovich(1, np_side, nc, 0.02)
    sim = dynamics.Simulation(nc, 0.02, 1.0, warmup + steps)
    sim.op.Ks_hat()
    sim.op.Kl_hat()
    st = sim.run(st, warmup)
    t0 = time.perf_counter()
    st = sim.run(st, steps)
    dt = time.perf_counter() - t0
    return np_side ** 3 * steps / dt, dt


# The oracle's bounded sample of every workload: steps of a 128^3-particle
# box (64^3 coarse, 256^3 fine), the same per-particle work as the 512^3 and
# 2048^3 boxes (8 particles per coarse cell, 8 fine cells per particle).
ORACLE_SAMPLE = (128, 64)


def oracle_sample_text(steps, seconds):
    return ("FP64 oracle, %d step(s) of a %d^3-particle box (%d^3 coarse, %d^3 fine cells: "
            "the same 8 particles per coarse cell and 8 fine cells per particle as the "
            "timed workload), %.1f s" % (steps, ORACLE_SAMPLE[0], ORACLE_SAMPLE[1],
                                         4 * ORACLE_SAMPLE[1], seconds))


def oracle_cores():
    # numpy.fft (pocketfft) and np.add.at run on one thread; no BLAS is used
    return 1


# ------------------------------------------------------------------ our arm

def pinned_state_bytes(cfg):
    """Pinned host bytes of one rank's end-to-end buffers (store, counts,
    v_c), each rounded up to a power of two as the pinned-memory cache
    allocates them."""
    def p2(x):
        return 1 << (int(x) - 1).bit_length()
    return p2((3 * cfg.pos_bytes + 3) * cfg.n) + p2(4 * cfg.ncells) + p2(12 * cfg.ncells)


def host_memory_available():
    """Bytes of host memory this process may still use: MemAvailable, capped
    by the cgroup's limit where one is set; None if neither can be read."""
    avail = None
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    avail = int(line.split()[1]) * 1024
    except OSError:
        pass
    try:
        with open("/sys/fs/cgroup/memory.max") as f:
            lim = f.read().strip()
        with open("/sys/fs/cgroup/memory.current") as f:
            cur = int(f.read().strip())
        if lim != "max":
            room = int(lim) - cur
            avail = room if avail is None else min(avail, room)
    except (OSError, ValueError):
        pass
    return avail


def measure_box(workload, K, W, E, local, world, rank):
    """One box: ICs, W warm-up steps, K steps timed with CUDA events on the
    library's stream (clocks sampled meanwhile, per-stage times recorded),
    then E end-to-end steps through the C ABI from pinned host buffers (load
    the store, step, fetch the store).  Returns the measurement and the
    still-open sim."""
    import torch

    from paper_2003_03931_gb300 import synth
    from paper_2003_03931_gb300.sim import SimConfig, Simulation

    w = dict(synth.WORKLOADS[workload])
    w["n_steps"] = W + K + E
    cfg = SimConfig(**w)
    sim = Simulation(cfg, device=f"cuda:{local}")
    stream = sim.stream
    t_ic = time.perf_counter()
    sim.ic_zeldovich(1 + rank, **synth.IC_SPECTRUM)
    sim.step(W)
    sim.sync()
    t_ic = time.perf_counter() - t_ic

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    sim.stage_times(enable=True, reset=True)
    sampler = ClockSampler(local)
    barrier()
    sampler.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(K)
    e1.record(stream)
    e1.synchronize()
    barrier()
    clocks = sampler.stop()
    t = e0.elapsed_time(e1) / 1000.0
    stages, launches = sim.stage_times(enable=False)
    sim.sync()
    t = reduce_max(t, f"cuda:{local}")

    e2e = None
    if E:
        # every rank on this node pins a copy of its whole state; skip the
        # end-to-end leg on all ranks if the node's host memory cannot hold them
        need = pinned_state_bytes(cfg)
        local_ranks = int(os.environ.get("LOCAL_WORLD_SIZE", world))
        avail = host_memory_available()
        short = avail is not None and local_ranks * (need + (2 << 30)) > avail
        if reduce_max(1.0 if short else 0.0, f"cuda:{local}") > 0.0:
            e2e = {"value": None, "unit": UNIT,
                   "skipped": "host memory: %d rank(s) x %.1f GB of pinned state exceed the %.1f GB "
                              "available" % (local_ranks, need / 1e9, (avail or 0) / 1e9)}
            E = 0
    if E:
        n, C = cfg.n, cfg.ncells
        pin = lambda shape, dt: torch.empty(shape, dtype=dt, pin_memory=True).numpy()
        pb = cfg.pos_bytes
        shape = (6, n) if pb == 1 else ((3 * pb + 3) * n,)
        host = {"streams": pin(shape, torch.uint8), "counts": pin((C,), torch.int32),
                "vc": pin((3, C), torch.float32)}
        sim.fetch_into(host)
        host["scalars"] = sim.fetch_scalars()
        barrier()
        t0 = time.perf_counter()
        parts = [0.0, 0.0, 0.0]     # load (h2d), step, fetch (d2h), host clock
        for _ in range(E):
            ta = time.perf_counter()
            sim.load_state(host)
            tb = time.perf_counter()
            sim.step(1)
            sim.sync()
            tc = time.perf_counter()
            sim.fetch_into(host)
            host["scalars"] = sim.fetch_scalars()
            td = time.perf_counter()
            parts[0] += tb - ta
            parts[1] += tc - tb
            parts[2] += td - tc
        torch.cuda.synchronize()
        te = reduce_max(time.perf_counter() - t0, f"cuda:{local}")
        per = (3 * pb + 3) * n + 4 * C + 12 * C + 32
        e2e = {"value": job_rate(n * E, world, te), "unit": UNIT, "h2d_bytes_per_step": per,
               "d2h_bytes_per_step": per, "steps": E,
               "seconds_per_step": {"load": parts[0] / E, "step": parts[1] / E, "fetch": parts[2] / E},
               "what": "per step: pmpm_load of the whole state from pinned host memory, "
                       "pmpm_step, pmpm_fetch of the whole state back"}
        del host
    stage_names = ["coarse_deposit", "coarse_fft_green", "tile_pm_kick_drift", "hist_scan_cell_means",
                   "dispersion", "encode_scatter"]
    if cfg.lowmem:
        stage_names = ["coarse_deposit", "coarse_fft_green", "tile_pm_kick_drift", "scan_cell_means",
                       "cell_moments_sigma", "reencode_scatter"]
    return {"cfg": cfg, "sim": sim, "t": t, "K": K, "W": W, "value": job_rate(cfg.n * K, world, t),
            "stages": {k: v / K for k, v in zip(stage_names, stages)}, "launches": launches,
            "clocks": clocks, "e2e": e2e, "setup_s": t_ic, "workspace_gb": sim.workspace.numel() / 1e9}


def box_roofline(m, workload, fp32_peak, peak_basis, hbm):
    """The dominant kernel's roofline (the tile pass) and every stage's."""
    cfg = m["cfg"]
    flops = tile_flops_per_launch(cfg.nc, cfg.tile_max)
    tile_stages = [k for k in m["stages"] if k.startswith("tile")]
    tile_ms = sum(m["stages"][k] for k in tile_stages)
    launches = len(tile_stages)
    avg_ms = tile_ms / launches
    achieved = flops / (avg_ms / 1e3) / 1e12
    kernel = ("k_tile, low-memory form (tile fine PM + kick + drift; new momenta kept, codes not)"
              if cfg.lowmem else "k_tile (tile fine PM + kick + drift)")
    roof = {"bound": "alu", "kernel": kernel, "achieved": achieved, "peak": fp32_peak,
            "unit": "TFLOP/s", "frac": achieved / fp32_peak,
            "traffic": recorded_traffic(workload, lowmem=cfg.lowmem),
            "peak_basis": peak_basis, "flops_per_launch": flops, "avg_launch_ms": avg_ms,
            "launches_per_step": launches}
    stages = stage_rooflines(m["stages"], cfg.n, cfg.ncells, hbm, flops, fp32_peak)
    return roof, stages


def box_config(m, workload, world):
    cfg = m["cfg"]
    n = cfg.n
    return {"workload": workload, "particles": n, "np": cfg.np, "nc": cfg.nc, "nf": 4 * cfg.nc,
            "step": "low-memory (one tile pass, re-encode from the old store)" if cfg.lowmem else "default",
            "workspace_gb": m["workspace_gb"], "tile_fine": "16/20 + 6 buffer in 32^3",
            "schedule": f"a 0.02->1 in {cfg.n_steps} steps, timed steps {m['W'] + 1}..{m['W'] + m['K']}",
            "parallelism": f"replicas x{world}", "bytes_per_particle_store": 3 * cfg.pos_bytes + 3,
            "l2": "inputs larger than L2 (%.0f MB particle store)" % ((3 * cfg.pos_bytes + 3) * n / 1e6)}


def run_ours(args):
    import torch

    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device(f"cuda:{local}")
    K, W = args.steps, args.warmup
    E = 0 if args.no_e2e else args.e2e_steps
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    m = measure_box(args.workload, K, W, E, local, world, rank)
    m["sim"].close()
    del m["sim"]
    torch.cuda.empty_cache()
    if rank != 0:
        return None

    sm_max = m["clocks"].get("sm_max_mhz") or measured_peaks().get("sm_max_mhz") or 2070.0
    derived = fp32_peak_tflops(sm_max, sms)
    peak, basis = derived, "FP32 FMA: %d SMs x 128 lanes x 2 x %d MHz (max SM clock)" % (sms, sm_max)
    if not args.no_fma_probe:
        peak = probe_fp32_tflops(dev)
        basis = "measured: FP32 FMA probe (pmpm_probe_fma), best of 5"
    hbm = measured_peaks().get("hbm_gbs")
    roof, stage_roof = box_roofline(m, args.workload, peak, basis, hbm)
    if not args.no_fma_probe:
        roof["peak_derived"] = derived
    out = {
        "metric": METRIC, "value": m["value"], "unit": UNIT, "n_gpus": world, "steps": K,
        "warmup": W, "ms_per_step": m["t"] / K * 1000.0, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": box_config(m, args.workload, world),
        "e2e": m["e2e"],
        "gpu_launches": m["launches"],
        "roofline": roof,
        "stage_ms_per_step": m["stages"],
        "stage_roofline": stage_roof,
        "hbm_peak_gbs": hbm,
        "clocks": m["clocks"],
        "setup_s": m["setup_s"],
    }
    if world == 1 and not args.no_cpu_baseline:
        v, dt = time_oracle_steps(ORACLE_SAMPLE[0], ORACLE_SAMPLE[1], 0, 2)
        out["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": oracle_cores(), "kind": "oracle",
                               "sample": oracle_sample_text(2, dt)}
    side = None
    if world == 1 and args.side_workload and args.side_workload != args.workload:
        s = measure_box(args.side_workload, K, W, 0 if args.no_e2e else 8, local, world, rank)
        sroof, sstages = box_roofline(s, args.side_workload, peak, basis, hbm)
        side = {"value": s["value"], "unit": UNIT, "ms_per_step": s["t"] / K * 1000.0,
                "config": box_config(s, args.side_workload, world), "e2e": s["e2e"],
                "gpu_launches": s["launches"], "roofline": sroof, "stage_ms_per_step": s["stages"],
                "stage_roofline": sstages, "clocks": s["clocks"]}
        cfg = s["cfg"]
        if not args.no_library_fft:
            nt = -(-cfg.nc // cfg.tile_max)
            s_lib = time_library_tile_transforms(nt ** 3, f"cuda:{local}")
            side["library_fft_tiles"] = {
                "ms_per_step": s_lib * 1000.0, "tiles": nt ** 3,
                "ours_tile_pass_ms_per_step": s["stages"]["tile_pm_kick_drift"],
                "what": "torch.fft (cuFFT) over batched 32^3 boxes in device memory: 1 R2C + 3 "
                        "(complex multiply, C2R) per tile, the transforms alone; the tile pass also "
                        "deposits, interpolates, kicks and drifts"}
            out["library_fft_tiles"] = dict(side["library_fft_tiles"], workload=args.side_workload)
        if args.plain_pm:
            plain = run_plain_pm(cfg, s["sim"], args.plain_pm, 1)
            plain["ours_over_plain"] = s["value"] / plain["value"]
            side["plain_gpu_pm"] = plain
            out["plain_gpu_pm"] = dict(plain, workload=args.side_workload)
        s["sim"].close()
        del s["sim"]
        torch.cuda.empty_cache()
        out[args.side_workload] = side
    if args.workload == "c4_2048":
        out["plain_gpu_pm_at_workload"] = {
            "feasible": False,
            "why": "a float32 4096^3 mesh is 275 GB and its spectrum as much again, more than "
                   "the GPU's 288 GB; the compressed step holds the whole box in %.0f GB"
                   % m["workspace_gb"]}
    if world == 1 and args.serving:
        out["serving"] = run_serving(args, f"cuda:{local}")
    return out


def periodic_kernel_spectra(nf, device, alpha=0.35, reach=16, dtype=None):
    """Spectra of the unit-G periodic pair force (a unit mass, all its images
    and the removed mean density) sampled at the integer separations of an
    nf^3 mesh of unit cells, one per component: the kernel's DFT is i S_d
    (the sampled kernel is real and odd), S_d float32 [nf, nf, nf/2 + 1].
    The force is split as Ewald did: a Gaussian-damped Fourier sum, which is
    exactly an inverse DFT once the damping has made the modes past the
    mesh's Nyquist frequency negligible (exp(-pi^2 / 4 alpha^2) = 2e-9 at
    alpha = 0.35 per cell), plus erfc-screened real-space terms of the
    nearest image within `reach` cells on each axis (below 1e-12 of the
    force beyond).  Built once per mesh in float64 (returned as `dtype`,
    float32 by default)."""
    import torch
    # nearest images only: the reach stays inside half the box (the screened
    # terms are below 1e-12 of the force past 15 cells)
    reach = min(reach, nf // 2 - 1)
    if reach < 15:
        raise ValueError("mesh too small for the real-space part")
    f64 = torch.float64
    two_pi = 2.0 * math.pi
    n = torch.fft.fftfreq(nf, d=1.0 / nf, device=device, dtype=f64)
    nr = torch.fft.rfftfreq(nf, d=1.0 / nf, device=device, dtype=f64)
    kz = (two_pi / nf * n).view(-1, 1, 1)
    ky = (two_pi / nf * n).view(1, -1, 1)
    kx = (two_pi / nf * nr).view(1, 1, -1)
    k2 = kx * kx + ky * ky + kz * kz
    k2[0, 0, 0] = 1.0
    # Fourier part: F~(k) = 4 pi i k / k^2 exp(-k^2 / 4 alpha^2); modes on a
    # Nyquist plane alias with their mirror images and are dropped
    damp = (4.0 * math.pi) * torch.exp(-k2 / (4.0 * alpha * alpha)) / k2
    del k2
    damp[0, 0, 0] = 0.0
    half = nf // 2
    damp[half, :, :] = 0.0
    damp[:, half, :] = 0.0
    damp[:, :, half] = 0.0
    # real-space part: -d/|d|^3 (erfc(alpha r) + 2 alpha r / sqrt(pi) e^(-alpha^2 r^2))
    d = torch.arange(-reach, reach + 1, device=device, dtype=f64)
    dz, dy, dx = torch.meshgrid(d, d, d, indexing="ij")
    r = torch.sqrt(dx * dx + dy * dy + dz * dz)
    r[reach, reach, reach] = 1.0
    fac = (torch.special.erfc(alpha * r) + 2.0 * alpha * r / math.sqrt(math.pi) *
           torch.exp(-(alpha * r) ** 2)) / r ** 3
    fac[reach, reach, reach] = 0.0
    iz = torch.remainder(dz.long(), nf)
    iy = torch.remainder(dy.long(), nf)
    ix = torch.remainder(dx.long(), nf)
    out = []
    for kd, dd in ((kx, dx), (ky, dy), (kz, dz)):
        field = torch.fft.irfftn((1j * kd) * damp, s=(nf, nf, nf))
        field[iz, iy, ix] += -dd * fac
        out.append(torch.fft.rfftn(field).imag.to(dtype or torch.float32))
        del field
    return out


class PlainPM:
    """The plain particle-mesh step that the compressed PM-PM step is measured
    against: one full-resolution mesh with the same total force kernel.
    Float32 positions (fine cells) and momenta, 24 bytes per particle; CIC
    deposit on the whole fine mesh (4 nc per side); one real-to-complex FFT;
    per component the multiply by the spectrum of the periodic pair force
    sampled at the fine-mesh separations (the kernel whose short- and
    long-range parts the two-level method splits between the fine tiles and
    the coarse mesh) and one complex-to-real FFT; CIC gather; the library's
    kick-drift schedule (equal steps in log a, momenta at the geometric
    mid-steps).  torch.fft is cuFFT on the GPU.  The same code runs on CPU
    tensors, so its arithmetic is tested there.  Measurement only: no force
    split, no compression."""

    def __init__(self, x, p, nf, a_init, a_final, n_steps, step=0, spectra=None):
        import torch
        self.torch = torch
        self.x, self.p, self.L, self.N = x, p, nf, x.shape[1]
        self.a = [a_init * (a_final / a_init) ** (i / n_steps) for i in range(n_steps + 1)]
        self.step_i = step
        self.S = spectra if spectra is not None else periodic_kernel_spectra(nf, x.device)

    def _corners(self):
        torch = self.torch
        s = self.x - 0.5
        i0 = torch.floor(s)
        f = s - i0
        i0 = i0.to(torch.int64)
        L = self.L
        for c in range(8):
            d = [(c >> e) & 1 for e in range(3)]
            w = torch.ones_like(f[0])
            idx = torch.zeros_like(i0[0])
            for e in (2, 1, 0):
                w = w * (f[e] if d[e] else 1.0 - f[e])
                idx = idx * L + torch.remainder(i0[e] + d[e], L)
            yield idx, w

    def force(self):
        """g = sum_j K_per(x - x_j) at every particle (CIC both ways), float32 [3, N]."""
        torch, L = self.torch, self.L
        rho = torch.zeros(L * L * L, dtype=torch.float32, device=self.x.device)
        for idx, w in self._corners():
            rho.index_add_(0, idx, w)
        rho_k = torch.fft.rfftn(rho.view(L, L, L))
        del rho
        g = torch.empty_like(self.x)
        for d in range(3):
            gd = torch.fft.irfftn(rho_k * (1j * self.S[d]), s=(L, L, L)).reshape(-1)
            acc = torch.zeros_like(self.x[0])
            for idx, w in self._corners():
                acc += w * gd[idx]
            g[d] = acc
        return g

    def step(self):
        a, n = self.a, self.step_i
        a_lo = a[0] if n == 0 else math.sqrt(a[n - 1] * a[n])
        a_hi = math.sqrt(a[n] * a[n + 1])
        rho_bar = self.N / float(self.L) ** 3
        kick = 3.0 / (8.0 * math.pi * rho_bar) * 2.0 * (math.sqrt(a_hi) - math.sqrt(a_lo))
        drift = 2.0 * (1.0 / math.sqrt(a[n]) - 1.0 / math.sqrt(a[n + 1]))
        self.p += kick * self.force()
        self.x = self.torch.remainder(self.x + drift * self.p, float(self.L))
        self.step_i += 1


def probe_fp32_tflops(device, repeats=5, iters=1 << 15):
    """Best of `repeats` runs of pmpm_probe_fma over 8 blocks of 256 threads
    per SM (full occupancy), TFLOP/s."""
    import ctypes

    import torch

    from paper_2003_03931_gb300 import _lib
    lib = _lib.load()
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    out = torch.empty(sms * 8 * 256, dtype=torch.float32, device=device)
    stream = torch.cuda.current_stream(device)
    best = 0.0
    for _ in range(repeats):
        flops, ms = ctypes.c_double(), ctypes.c_float()
        rc = lib.pmpm_probe_fma(ctypes.c_void_p(out.data_ptr()), out.numel(),
                                ctypes.c_void_p(stream.cuda_stream), iters, ctypes.byref(flops),
                                ctypes.byref(ms))
        if rc != _lib.PMPM_OK:
            raise RuntimeError(f"pmpm_probe_fma failed ({rc})")
        best = max(best, flops.value / (ms.value * 1e-3) / 1e12)
    return best


def time_library_tile_transforms(ntiles, device, batch=2048, reps=3):
    """The tile pass's transforms done by the FFT library instead (torch.fft,
    cuFFT on the GPU): per 32^3 tile box one real-to-complex transform and,
    per force component, one complex multiply by a spectrum and one
    complex-to-real transform, over batches of `batch` boxes in device
    memory.  Returns seconds for `ntiles` tiles (scaled from the best of
    `reps` batches).  No deposit, interpolation or output pruning: the
    transforms alone."""
    import torch
    gen = torch.Generator(device="cpu").manual_seed(7)
    x = torch.randn(batch, 32, 32, 32, generator=gen).to(device)
    spec = torch.randn(3, 32, 32, 17, generator=gen, dtype=torch.complex64).to(device)
    cuda = torch.device(device).type == "cuda"

    def once():
        xk = torch.fft.rfftn(x, dim=(1, 2, 3))
        for d in range(3):
            y = torch.fft.irfftn(xk * spec[d], s=(32, 32, 32), dim=(1, 2, 3))
        return y

    once()
    best = float("inf")
    for _ in range(reps):
        if cuda:
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            once()
            e1.record()
            e1.synchronize()
            t = e0.elapsed_time(e1) / 1000.0
        else:
            t0 = time.perf_counter()
            once()
            t = time.perf_counter() - t0
        best = min(best, t)
    return best * ntiles / batch


def run_plain_pm(cfg, sim, steps, warmup):
    """Time the plain PM comparator on the sim's current particles (decoded
    to float32) for `steps` steps after `warmup`; CUDA events on torch's
    current stream."""
    import torch
    Q, P = sim.fetch_decoded()
    dev = sim.device
    per_fine = (256 if cfg.pos_bytes == 1 else 65536) // 4
    x = (torch.from_numpy(Q).to(dev).to(torch.float64) + 0.5).div_(per_fine).to(torch.float32)
    p = torch.from_numpy(P).to(dev)
    # continue the library's equal-log-a schedule from the current a for
    # as many steps as run here
    a_now = float(sim.fetch_scalars()["a"])
    ratio = (cfg.a_final / cfg.a_init) ** (1.0 / cfg.n_steps)
    pm = PlainPM(x, p, 4 * cfg.nc, a_now, a_now * ratio ** (warmup + steps), warmup + steps)
    for _ in range(warmup):
        pm.step()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        pm.step()
    e1.record()
    e1.synchronize()
    t = e0.elapsed_time(e1) / 1000.0
    return {"value": cfg.n * steps / t, "unit": UNIT, "ms_per_step": t / steps * 1000.0,
            "steps": steps, "warmup": warmup, "bytes_per_particle": 24,
            "method": "float32 x, p; CIC on the whole (4 nc)^3 fine mesh; torch.fft (cuFFT) R2C, "
                      "3 x (multiply by the spectrum of the periodic pair force sampled on the "
                      "fine mesh, C2R); CIC gather; same kick-drift"}


SERVING_ARENA = 48 << 30
SEQUENTIAL = dict(max_active=1, share_tables=False, graphs=False, priorities=False,
                  steps_per_chunk=4, chunks_in_flight=2)
SEQUENTIAL_SHARED = dict(SEQUENTIAL, share_tables=True)
BATCHED = dict(max_active=16, share_tables=True, graphs=True, priorities=1, steps_per_chunk=4,
               chunks_in_flight=2)
# the same engine with at most one 256^3 box resident: the large boxes, which
# make the latency tail, run one after another at nearly the whole GPU while
# the smaller boxes pass them and fill the gaps
BATCHED_LARGE1 = dict(BATCHED, large_np=256, max_large=1)


def alone_rates(device, sizes=(32, 64, 128, 256), steps=10, warmup=2):
    """Stepping throughput of one box of each size alone on the GPU
    (particle-steps/s, CUDA events around `steps` steps)."""
    import torch

    from paper_2003_03931_gb300 import synth
    from paper_2003_03931_gb300.sim import SimConfig, Simulation
    out = {}
    for np_ in sizes:
        sim = Simulation(SimConfig(np=np_, nc=np_ // 2, n_steps=steps + warmup), device=device)
        sim.ic_zeldovich(3, **synth.IC_SPECTRUM)
        sim.step(warmup)
        sim.sync()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(sim.stream)
        sim.step(steps)
        e1.record(sim.stream)
        e1.synchronize()
        out[str(np_)] = np_ ** 3 * steps / (e0.elapsed_time(e1) / 1000.0)
        sim.close()
    return out


def run_serving(args, device):
    """Mixed stream of whole-box requests (32^3..256^3 particles, 10-40 steps,
    weights 0.4/0.3/0.2/0.1): the batched engine against sequential plain
    stepping (one box at a time, each building its own force tables), first
    with every request queued at t=0 (throughput), then on Poisson arrivals
    at fractions of the sequential capacity (latency)."""
    from paper_2003_03931_gb300.serve import (Engine, latency_summary, mixed_requests, run_stream,
                                              with_arrivals)

    def go(kw, reqs):
        eng = Engine(SERVING_ARENA, device=device, **kw)
        res = run_stream(eng, reqs, timeout=1800)
        st = eng.stats()
        eng.close()
        s = latency_summary(res)
        s.update(table_builds=st["table_builds"], gpu_launches=st["launches"],
                 arena_peak_gb=st["arena_peak"] / 2 ** 30)
        return s

    reqs = mixed_requests(args.serving, seed=0)
    go(BATCHED, mixed_requests(8, seed=9, sizes=(32, 64), weights=(1, 1)))    # warm-up
    seq = go(SEQUENTIAL, reqs)
    seq_shared = go(SEQUENTIAL_SHARED, reqs)
    bat = go(BATCHED, reqs)
    bat_large1 = go(BATCHED_LARGE1, reqs)
    # Ceiling of any batching of this mix: even if every particle-step ran at
    # the best rate one box reaches alone (the GPU filled by one box), the
    # stream's steps would take sum(work) / max rate; ICs and P(k) only add.
    rates = alone_rates(device)
    work = sum(r.n * r.n_steps for r in reqs)
    best = max(rates.values())
    ceiling = {"alone_rates": rates, "particle_steps": work,
               "steps_at_best_rate_s": work / best,
               "sequential_makespan_s": seq["makespan_s"],
               "ratio_vs_sequential": seq["makespan_s"] / (work / best),
               "what": "sequential makespan over (all particle-steps / the best one-box rate): "
                       "the most any batching of this stream can gain, ICs and P(k) aside"}
    out = {
        "workload": "%d requests: 32^3/64^3/128^3/256^3 particles (weights .4/.3/.2/.1, nc = np/2), "
                    "10-40 steps a 0.02->1, slopes U[-2,-1], seeds 1000+i; P(k) on an np^3 mesh "
                    "at the end" % len(reqs),
        "unit": UNIT,
        "sequential": dict(seq, config=SEQUENTIAL),
        "sequential_shared_tables": dict(seq_shared, config=SEQUENTIAL_SHARED),
        "batched": dict(bat, config=BATCHED),
        "batched_one_large": dict(bat_large1, config=BATCHED_LARGE1),
        "throughput_ratio_vs_sequential": bat["particle_steps_per_s"] / seq["particle_steps_per_s"],
        "throughput_ratio_one_large_vs_sequential":
            bat_large1["particle_steps_per_s"] / seq["particle_steps_per_s"],
        "ceiling": ceiling,
        "throughput_ratio_vs_sequential_shared_tables":
            bat["particle_steps_per_s"] / seq_shared["particle_steps_per_s"],
        "latency": [],
    }
    cap = seq["requests_per_s"]
    for f in [float(x) for x in args.serving_rates.split(",") if x.strip()]:
        arr = with_arrivals(reqs, rate=f * cap, seed=1)
        out["latency"].append({"rate_fraction_of_sequential_capacity": f,
                               "rate_requests_per_s": f * cap,
                               "sequential": go(SEQUENTIAL, arr), "batched": go(BATCHED, arr),
                               "batched_one_large": go(BATCHED_LARGE1, arr)})
    return out


def run_reference(args):
    world, rank, local = dist_setup(args)
    if rank != 0:
        return None
    K, W = args.steps, args.warmup
    # each step a bounded sample of the workload: one oracle step of the
    # 128^3-particle box (same per-particle work)
    v, dt = time_oracle_steps(ORACLE_SAMPLE[0], ORACLE_SAMPLE[1], W, K)
    sample = oracle_sample_text(K, dt) + " after %d untimed" % W
    return {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": K,
            "warmup": W, "ms_per_step": dt / K * 1000.0, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": args.workload, "timed_box": "%d^3 particles (bounded sample)"
                       % ORACLE_SAMPLE[0], "parallelism": "host cores"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": oracle_cores(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main(argv=None):
    args = parse_args(argv)
    if args.serving_only:
        out = {"metric": "serving", "serving": run_serving(args, "cuda:0")}
    else:
        out = run_reference(args) if args.impl == "reference" else run_ours(args)
    if out is not None:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
