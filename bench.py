#!/usr/bin/env python3
"""Benchmark of the local level-set grain-growth step on GB300.

A "step" is one pass of the whole hot path over every grain box: heat-kernel
predictor, comparison step, taxicab re-initialisation and box update.  The
workload is a 256^3 periodic domain with 5000 Voronoi grains (seed 2), ideal
growth, dt = 1 (kernel variance 2 per axis), FP32 -- the paper-like 3D shape
(about 19 cells per grain diameter).

Output: one JSON line on rank 0.  ``value`` = box cell-updates per second
(box cells advanced by one full step, summed over grains and timed steps,
divided by the device time of the timed steps, max over ranks, summed over
ranks' work).  Multi-GPU runs are independent replicas (the step has no
cross-replica exchange): weak scaling.

--impl reference times the FP64 oracle on the host cores on a bounded sample
of the same workload (a 64^3 periodic sub-domain at the same grain density).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import re
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOADS = {
    "256": {"n": 256, "grains": 5000, "seed": 2, "dt": 1.0},
    # small case for ncu captures: same grain density, state still larger than L2
    "160": {"n": 160, "grains": 1221, "seed": 2, "dt": 1.0},
    # non-ideal growth: Laguerre tessellation with lognormal radii (sigma 0.5) and
    # 1 % of grains with 5x volume, random cubic orientations, Read-Shockley
    # boundary energy (theta_max 15 deg) and mobility 0.1 below 15 deg
    "512rs": {"n": 512, "grains": 40000, "seed": 3, "dt": 1.0, "physics": "read_shockley", "init": "laguerre"},
    # small case of the Read-Shockley workload for profilers (the same grain density)
    "160rs": {"n": 160, "grains": 1221, "seed": 3, "dt": 1.0, "physics": "read_shockley", "init": "laguerre"},
    # magnetically driven growth: random c-axes, field (0, cos 32, sin 32), bulk
    # energy B^2 dchi cos^2 / (2 mu0) in grid units (4.07e-3 at cos^2 = 1)
    "384mag": {"n": 384, "grains": 10000, "seed": 4, "dt": 1.0, "physics": "magnetic", "energy_scale": 4.07e-3},
    # small case of the magnetic workload for profilers (the grain density of the 256^3 workload)
    "160mag": {"n": 160, "grains": 1221, "seed": 4, "dt": 1.0, "physics": "magnetic", "energy_scale": 4.07e-3},
}
WORKLOAD = dict(WORKLOADS["256"])
SAMPLE = {"n": 64, "grains": 78, "seed": 2}     # same density: 64^3 / 78 = 3361 cells per grain
METRIC = "LS box cell-updates/s"
UNIT = "cell-updates/s"


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            return json.load(open(p)), "measured"
        except Exception:
            pass
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# the sources the pass kernels are compiled from: their file and every header
# it includes
PASS_KERNEL_SOURCES = ("paper_1701_06658_gb300/csrc/passes.cu", "paper_1701_06658_gb300/csrc/bulk_copy.cuh",
                       "paper_1701_06658_gb300/csrc/kernels_common.cuh", "paper_1701_06658_gb300/csrc/group.cuh",
                       "paper_1701_06658_gb300/csrc/lsgg_internal.cuh", "include/lsgg.h")


def _code_only(text: str) -> str:
    """C/C++ source without comments and with whitespace collapsed (string
    literals in these sources hold no comment markers)."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def kernel_source_hash():
    """Hash of the pass kernels' code (comments and layout ignored)."""
    h = hashlib.sha256()
    for f in PASS_KERNEL_SOURCES:
        h.update(_code_only(open(os.path.join(ROOT, f), encoding="utf-8").read()).encode())
    return h.hexdigest()[:16]


# Bytes per box cell (per domain cell for the field) the design's five passes
# must move at least: each reads its input field once and writes its output
# once.  The state X is FP32 (4 B) or BF16 (2 B); with physics the z pass also
# reads the previous step's phi and ID-field of each cell.
def pass_bytes(kernel: str, state_bytes: int, physics: bool, keep_field: bool = False):
    """(bytes per box cell of the launch's tier, bytes per domain cell)."""
    name = kernel.split("[")[0]
    if name == "p_conv_xy":
        return state_bytes + 4.0, 0.0                     # X (old layout) in, Z out
    if name == "p_conv_z":
        return 8.0 + ((state_bytes + 4.0) if physics else 0.0), 0.0   # Z in, Y out (+ phi, IDF)
    if name == "p_field":
        # phi_p read once (the top two), phi_c written (and the ID-field with
        # physics); the top-two field is consumed in registers, its 16 B per
        # domain cell stored only on request (lsgg_keep_field)
        return 8.0 + (4.0 if physics else 0.0), 16.0 if keep_field else 0.0
    if name == "p_redist_xy":
        return 8.0, 0.0                                   # phi_c in, x/y-scanned magnitudes out
    if name == "p_redist_z":
        return 4.0 + state_bytes, 0.0                     # magnitudes in, phi (X) out
    raise KeyError(kernel)


def step_roofline(box_cells: float, dom_cells: float, ms_per_step: float, peak_gbs: float, passes: bool,
                  state_bytes: int = 4, physics: bool = False, keep_field: bool = False):
    """The whole step against the bytes the method must move at least (one
    read and write of phi per box cell -- the ID-field's too with physics --
    and 44 B of top-two field per domain cell: 16 cleared, 16 written, 12
    read) and against the bytes of this design's five passes (the sum of
    pass_bytes over the passes), both over the measured step time."""
    idf = 8.0 if physics else 0.0
    minimum = (2.0 * state_bytes + idf) * box_cells + 44.0 * dom_cells
    t = ms_per_step * 1e-3
    out = {"minimum_bytes_per_step": minimum, "minimum_bound_ms": minimum / (peak_gbs * 1e9) * 1e3,
           "achieved_minimum_gbs": minimum / t / 1e9, "frac_minimum": minimum / t / 1e9 / peak_gbs,
           "peak": peak_gbs, "unit": "GB/s"}
    if passes:
        per_box = sum(pass_bytes(k, state_bytes, physics)[0]
                      for k in ("p_conv_xy", "p_conv_z", "p_field", "p_redist_xy", "p_redist_z"))
        design = per_box * box_cells + pass_bytes("p_field", state_bytes, physics, keep_field)[1] * dom_cells
        out.update(design_bytes_per_step=design, design_bytes_per_box_cell=per_box,
                   achieved_design_gbs=design / t / 1e9, frac_design=design / t / 1e9 / peak_gbs)
    return out


def kernel_roofline(pass_ms: dict, tier_cells, box_cells: float, dom_cells: float, n_grains: int, peak_gbs: float,
                    state_bytes: int = 4, physics: bool = False, keep_field: bool = False):
    """Roofline of the pass with the longest time per launch: its algorithmic
    bytes per launch (pass_bytes x the box cells of its tier, or of all boxes
    for the field pass) over its CUDA-event time."""
    dominant = max(pass_ms, key=pass_ms.get)
    if dominant == "k_bin":
        units, alg = float(n_grains), 32.0 * n_grains
    else:
        per_box, per_dom = pass_bytes(dominant, state_bytes, physics, keep_field)
        units = box_cells if dominant == "p_field" else float(tier_cells[int(dominant[-2])])
        alg = per_box * units + per_dom * dom_cells
    achieved = alg / (pass_ms[dominant] * 1e-3) / 1e9
    return {"bound": "hbm", "kernel": dominant, "achieved": achieved, "peak": peak_gbs, "unit": "GB/s",
            "frac": achieved / peak_gbs, "algorithmic_bytes_per_launch": alg, "units_per_launch": units,
            "launch_ms": pass_ms[dominant]}


def profiled_traffic(kernel: str, units_per_launch: float):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, scaled
    to this launch by units processed; None if the kernel changed since."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    try:
        d = json.load(open(p))
        k = d.get(kernel)
        if not k or k.get("source_hash") != kernel_source_hash():
            return None
        return k["dram_bytes_per_launch"] * units_per_launch / k["units_per_launch"]
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None
        self.gpu = gpu_index

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu),
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        try:
            self.fh.close()
        except Exception:
            pass

    def summary(self):
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        except Exception:
            rows = []
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in rows if r[0].strip().replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for k, nm in enumerate(names):
                if len(r) > 4 + k and r[4 + k].strip() == "Active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


# ---------------------------------------------------------------- oracle (CPU)

def oracle_sample_run(steps: int, warmup: int, seed: int = SAMPLE["seed"]):
    """The FP64 oracle on the bounded sample: 64^3 periodic domain, 78 Voronoi
    grains (seed 2 by default), dt = 1; returns (cell-updates/s, seconds,
    cell-updates)."""
    import numpy as np
    from oracle import lsgg_oracle as O
    from paper_1701_06658_gb300 import inputs as I
    n, g = SAMPLE["n"], SAMPLE["grains"]
    ms = O.tessellate((n, n, n), I.voronoi_seeds(seed, g, (n, n, n)))
    for _ in range(warmup):
        ms = O.step(ms, 1.0)
    cells = 0
    t0 = time.perf_counter()
    for _ in range(steps):
        cells += sum(int(np.prod(gr.dims)) for gr in ms.grains if gr.alive)
        ms = O.step(ms, 1.0)
    dt = time.perf_counter() - t0
    return cells / dt, dt, cells


def _oracle_worker(steps, seed, barrier, out):
    """One process of the all-core run: tessellate, wait for the others, then
    time `steps` oracle steps (wall-clock start and end)."""
    import numpy as np
    from oracle import lsgg_oracle as O
    from paper_1701_06658_gb300 import inputs as I
    n, g = SAMPLE["n"], SAMPLE["grains"]
    ms = O.tessellate((n, n, n), I.voronoi_seeds(seed, g, (n, n, n)))
    barrier.wait()
    t0 = time.time()
    cells = 0
    for _ in range(steps):
        cells += sum(int(np.prod(gr.dims)) for gr in ms.grains if gr.alive)
        ms = O.step(ms, 1.0)
    out.put((cells, t0, time.time()))


def cpu_model() -> str:
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def oracle_all_cores(steps: int):
    """The oracle as it stands on every host core: one spawned process per
    core, each with its own 64^3 sample (seeds 2, 3, ...); after all have
    tessellated they start together, and the throughput is all processes'
    cell-updates over the span from the first start to the last finish."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    env_keep = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in env_keep:                      # one thread per process: the cores are the parallelism
        os.environ[k] = "1"
    try:
        ctx = mp.get_context("spawn")
        barrier, out = ctx.Barrier(cores), ctx.Queue()
        procs = [ctx.Process(target=_oracle_worker, args=(steps, SAMPLE["seed"] + k, barrier, out))
                 for k in range(cores)]
        for p in procs:
            p.start()
        res = [out.get(timeout=600) for _ in procs]
        for p in procs:
            p.join(timeout=60)
    finally:
        for k, v in env_keep.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    cells = sum(r[0] for r in res)
    span = max(r[2] for r in res) - min(r[1] for r in res)
    return {"value": cells / span, "cores": cores, "span_s": span, "cell_updates": cells}


def cpu_baseline_block(steps: int = 2):
    """cpu_baseline of the bench line: the oracle on all host cores (value)
    and on one core, with the host's core count and CPU model."""
    one_rate, one_s, _ = oracle_sample_run(steps, 0)
    allc = oracle_all_cores(steps)
    sample = (f"{steps} oracle steps of a {SAMPLE['n']}^3 periodic sub-domain at the workload's grain density "
              f"({SAMPLE['grains']} Voronoi grains) per process, one process per core (seeds "
              f"{SAMPLE['seed']}..{SAMPLE['seed'] + allc['cores'] - 1}), started together after "
              f"tessellating; {allc['span_s']:.1f} s from the first start to the last finish")
    return {"value": allc["value"], "unit": UNIT, "cores": allc["cores"], "kind": "oracle", "sample": sample,
            "nproc": os.cpu_count(), "cpu_model": cpu_model(),
            "single_core": {"value": one_rate, "unit": UNIT, "cores": 1, "seconds": one_s}}


def reference_arm(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    rate, secs, cells = oracle_sample_run(args.steps, args.warmup)
    sample = (f"{SAMPLE['n']}^3 periodic sub-domain at the workload's grain density "
              f"({SAMPLE['grains']} Voronoi grains, seed {SAMPLE['seed']}), {args.steps} steps")
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(),
            "cpu_baseline": {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                             "nproc": os.cpu_count(), "cpu_model": cpu_model()},
            "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def replica_seed(rank: int) -> int:
    """Tessellation seed of a rank's replica: independent replicas, no exchange."""
    return WORKLOAD["seed"] + 1000 * rank


def reduce_over_ranks(dev_ms, cells, e2e_s, e2e_cells, world):
    """Whole-job timing of independent replicas: the slowest rank's times and
    the sum of all ranks' cell-updates (a no-op on one rank)."""
    if world <= 1:
        return dev_ms, float(cells), e2e_s, float(e2e_cells)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([dev_ms, float(cells), e2e_s, float(e2e_cells)], dtype=torch.float64, device=dev)
    mx, sm = t.clone(), t.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return mx[0].item(), sm[1].item(), mx[2].item(), sm[3].item()


def workload_kwargs(L, wl=None):
    """Microstructure keyword arguments of a workload's physics and tessellation."""
    wl = WORKLOAD if wl is None else wl
    kw = {}
    ph = wl.get("physics", "ideal")
    if ph == "read_shockley":
        kw["physics"] = L.PHYSICS_READ_SHOCKLEY
    elif ph == "magnetic":
        kw["physics"] = L.PHYSICS_MAGNETIC
        kw["energy_scale"] = wl["energy_scale"]
    if wl.get("init") == "laguerre":
        kw["init_kind"] = L.INIT_LAGUERRE
    if wl.get("redist") == "godunov":
        kw["redist"] = L.REDIST_GODUNOV
    return kw


def workload_config(wl=None):
    wl = WORKLOAD if wl is None else wl
    ph = {"ideal": "ideal growth", "read_shockley": "Read-Shockley energy and step mobility, random cubic orientations",
          "magnetic": "magnetic driving force, random c-axes"}[wl.get("physics", "ideal")]
    tess = ("Laguerre grains, lognormal radii sigma 0.5, 1 % at 5x volume" if wl.get("init") == "laguerre"
            else "Voronoi grains")
    rd = "" if wl.get("redist", "taxicab") == "taxicab" else ", Godunov re-initialisation"
    return {"workload": f"{wl['n']}^3 periodic, {wl['grains']} {tess} (seed {wl['seed']}), "
                        f"{ph}{rd}, dt={wl['dt']}, box halo 5, eps 7, FP32",
            "domain": [wl["n"]] * 3, "grains": wl["grains"], "dt": wl["dt"],
            "l2": f"inputs larger than L2: box arenas of ~{wl['n'] ** 3 * 8.5 * 4 / 1e9:.1f} GB each and a "
                  f"{16 * wl['n'] ** 3 / 1e6:.0f} MB field vs 129 MB L2"}


def device_block(L, I, torch, wl, device, steps, warmup, storage, prof_steps=3):
    """Device-timed steps of a workload (CUDA events on the library's stream,
    SM clocks sampled meanwhile), then profiled steps for the per-pass times
    and the roofline of the longest pass."""
    n, g, dt = wl["n"], wl["grains"], wl["dt"]
    seeds = I.voronoi_seeds(wl["seed"], g, (n, n, n))
    physics = wl.get("physics", "ideal") != "ideal"
    sb = 2 if storage == L.STORAGE_BF16 else 4
    t0 = time.perf_counter()
    with L.Microstructure(n, n, n, g, seeds=seeds, device=device, storage=storage, **workload_kwargs(L, wl)) as ms:
        create_s = time.perf_counter() - t0
        stream = torch.cuda.ExternalStream(ms.stream)
        ms.step(warmup, dt)
        ms.sync()
        s0 = ms.stats()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        with ClockSampler(device) as clk:
            e0.record(stream)
            ms.step(steps, dt)
            e1.record(stream)
            ms.sync()
            torch.cuda.synchronize()
        dev_ms = e0.elapsed_time(e1)
        s1 = ms.stats()
        L.profile(ms.ctx, True)
        ms.step(prof_steps, dt)
        L.kernel_times(ms.ctx)
        ptimes = L.pass_times(ms.ctx)
        L.profile(ms.ctx, False)
        s2 = ms.stats()
    cells = s1.cell_updates - s0.cell_updates
    box_cells = cells / steps
    pass_ms = {k: v[0] / max(1, v[1]) for k, v in ptimes.items() if v[1] > 0}
    peaks, src = measured_peaks()
    cfg = workload_config(wl)
    cfg["workload"] = cfg["workload"].replace("FP32", "BF16 state storage, FP32 arithmetic" if sb == 2 else "FP32")
    out = {"config": cfg, "value": cells / (dev_ms * 1e-3), "unit": UNIT, "steps": steps, "warmup": warmup,
           "ms_per_step": dev_ms / steps, "box_cells_per_step": box_cells, "superimposition": box_cells / n ** 3,
           "domain_cell_updates_per_s": n ** 3 * steps / (dev_ms * 1e-3), "create_s": create_s,
           "pass_ms_per_step": pass_ms, "pass_cells_per_tier": list(s2.pass_cells), "clocks": clk.summary(),
           "timing": "CUDA events on the library's stream around the timed steps (graph replay)"}
    if pass_ms:
        prof_cells = (s2.cell_updates - s1.cell_updates) / prof_steps
        rl = kernel_roofline(pass_ms, list(s2.pass_cells), prof_cells, float(n) ** 3, g, peaks.get("hbm_gbs"),
                             sb, physics)
        rl["peak_source"] = src
        out["roofline"] = rl
    out["step_roofline"] = step_roofline(box_cells, float(n) ** 3, dev_ms / steps, peaks.get("hbm_gbs"),
                                         bool(pass_ms), sb, physics)
    return out


# ---------------------------------------------------------------- GPU arm

def gpu_arm(args):
    import numpy as np  # noqa: F401
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_1701_06658_gb300 import inputs as I
    from paper_1701_06658_gb300 import lsgg as L
    L.lib()
    n, g, dt = WORKLOAD["n"], WORKLOAD["grains"], WORKLOAD["dt"]
    seed = replica_seed(rank)                      # independent replica per rank
    seeds = I.voronoi_seeds(seed, g, (n, n, n))

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    # ---------------- device-resident timing ----------------
    exec_mode = {"batched": L.EXEC_BATCHED, "streamed": L.EXEC_STREAMED}[args.exec]
    ms = L.Microstructure(n, n, n, g, seeds=seeds, device=local, exec_mode=exec_mode, **workload_kwargs(L))
    stream = torch.cuda.ExternalStream(ms.stream)
    ms.step(args.warmup, dt)
    ms.sync()
    tiles = None
    if not args.no_tune:                          # untimed: real steps under each trial setting
        tiles = {"register_ring": L.autotune(ms.ctx, 2, dt), "pass_path": L.pass_tuning(ms.ctx)}
    ms.sync()
    s0 = ms.stats()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ev0.record(stream)
        ms.step(args.steps, dt)
        ev1.record(stream)
        ms.sync()
        torch.cuda.synchronize()
    barrier()
    dev_ms = ev0.elapsed_time(ev1)
    s1 = ms.stats()
    cells = s1.cell_updates - s0.cell_updates
    box_cells_mean = cells / args.steps

    # ---------------- per-kernel event timing (separate pass) ----------------
    L.profile(ms.ctx, True)
    kprof = min(args.steps, 20)
    ms.step(kprof, dt)
    ktimes, kcount = L.kernel_times(ms.ctx)
    ptimes = L.pass_times(ms.ctx)
    L.profile(ms.ctx, False)
    s2 = ms.stats()
    tier_cells = list(s2.pass_cells)
    cells_prof = s2.cell_updates - s1.cell_updates
    ms.close()

    # ---------------- end to end through the public API ----------------
    torch.cuda.synchronize()
    barrier()
    e2e_s, e2e_cells, d2h = float("nan"), 0, 0
    if not args.no_e2e:
        # the results land in pinned host buffers (allocated once, before the
        # timed region), as a caller moving them every step would keep them
        h_vol = torch.empty(g, dtype=torch.float64).pin_memory()
        h_own = torch.empty((n, n, n), dtype=torch.int32).pin_memory()
        t0 = time.perf_counter()
        e2e = L.Microstructure(n, n, n, g, seeds=seeds, device=local,    # H2D of the seeds, init
                               exec_mode=exec_mode, **workload_kwargs(L))
        for _ in range(args.steps):
            e2e.step(1, dt)
            vol = e2e.grain_volumes(h_vol.numpy())                         # D2H of the step's result
            d2h += vol.nbytes
        own = e2e.voxel_owner(h_own.numpy())
        d2h += own.nbytes
        se = e2e.stats()
        e2e.close()
        e2e_s = time.perf_counter() - t0
        e2e_cells = se.cell_updates

    # ---------------- comparison paths on the same workload ----------------
    # the plain path (one launch per grain per sub-step, the comparator the
    # metric is quoted against) and the box-streaming kernels, a few steps each
    compare = None
    if not args.no_compare and rank == 0:
        compare = {}
        for name, mode, steps in (("plain_gpu", L.EXEC_PLAIN, 3), ("box_streaming_gpu", L.EXEC_STREAMED, 10)):
            with L.Microstructure(n, n, n, g, seeds=seeds, device=local, exec_mode=mode, **workload_kwargs(L)) as cm:
                cm.step(2, dt)
                cm.sync()
                c0 = cm.stats().cell_updates
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                cm.step(steps, dt)
                cm.sync()
                el = time.perf_counter() - t0
                rate = (cm.stats().cell_updates - c0) / el
            compare[name] = {"value": rate, "unit": UNIT, "steps": steps, "ms_per_step": 1e3 * el / steps,
                             "timing": "host wall clock around the steps (synchronised)"}

    # ---------------- BF16 state storage on the same workload ----------------
    # phi stored in BF16 between steps (FP32 arithmetic): device-timed steps and
    # the per-grain volume error against FP32 after the same number of steps
    bf16 = None
    if not args.no_compare and rank == 0:
        steps_b = 10
        vols = {}
        for st in (L.STORAGE_FP32, L.STORAGE_BF16):
            with L.Microstructure(n, n, n, g, seeds=seeds, device=local, exec_mode=exec_mode, storage=st,
                                  **workload_kwargs(L)) as bm:
                bm.step(2, dt)
                bm.sync()
                c0 = bm.stats().cell_updates
                bstream = torch.cuda.ExternalStream(bm.stream)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record(bstream)
                bm.step(steps_b, dt)
                e1.record(bstream)
                bm.sync()
                torch.cuda.synchronize()
                vols[st] = (bm.grain_volumes(), (bm.stats().cell_updates - c0) / (e0.elapsed_time(e1) * 1e-3),
                            e0.elapsed_time(e1) / steps_b)
        v32, v16 = vols[L.STORAGE_FP32][0], vols[L.STORAGE_BF16][0]
        alive = v32 > 50.0
        rel = np.abs(v16[alive] - v32[alive]) / v32[alive]
        bf16 = {"value": vols[L.STORAGE_BF16][1], "unit": UNIT, "ms_per_step": vols[L.STORAGE_BF16][2],
                "fp32_same_run": vols[L.STORAGE_FP32][1], "steps": 2 + steps_b,
                "volume_rel_error_vs_fp32": {"max": float(rel.max()), "mean": float(rel.mean())}}

    # ---------------- grid coarsening (Sec. 4.1) of the same workload ----------------
    # lsgg_coarsen to half the cells per axis after a few steps (host wall clock
    # around the synchronising call), then device-timed steps on the coarse grid
    coarsening = statistics = None
    if not args.no_compare and rank == 0 and WORKLOAD.get("physics", "ideal") == "ideal" and n % 2 == 0:
        with L.Microstructure(n, n, n, g, seeds=seeds, device=local, exec_mode=exec_mode,
                              **workload_kwargs(L)) as km:
            km.step(5, dt)
            km.sync()
            # the size analysis on the device (Sec. 5): statistics and texture shares
            t0 = time.perf_counter()
            gs = km.grain_statistics(20, 3.0)
            t_stats = time.perf_counter() - t0
            t0 = time.perf_counter()
            km.texture_shares(np.arange(g, dtype=np.int32) % 2, 2)
            t_tex = time.perf_counter() - t0
            fine_cells = km.stats().box_cells
            t0 = time.perf_counter()
            km.coarsen(n // 2, n // 2, n // 2)
            el = time.perf_counter() - t0
            coarse_cells = km.stats().box_cells
            km.step(2, dt)
            km.sync()
            c0 = km.stats().cell_updates
            kstream = torch.cuda.ExternalStream(km.stream)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            steps_k = 10
            torch.cuda.synchronize()
            e0.record(kstream)
            km.step(steps_k, dt)
            e1.record(kstream)
            km.sync()
            torch.cuda.synchronize()
            kms = e0.elapsed_time(e1)
            k_rate = (km.stats().cell_updates - c0) / (kms * 1e-3)
        statistics = {"grain_statistics_ms": 1e3 * t_stats, "texture_shares_ms": 1e3 * t_tex,
                      "alive": int(gs["alive"]), "rho": gs["rho"], "var_z": gs["var_z"],
                      "timing": "host wall clock around each synchronising call after 5 steps"}
        coarsening = {"from": [n, n, n], "to": [n // 2] * 3, "ms": 1e3 * el,
                      "timing": "host wall clock around lsgg_coarsen (box copies, relayout, projection, "
                                "re-initialisation, box update; synchronising)",
                      "fine_box_cells": int(fine_cells), "coarse_box_cells": int(coarse_cells),
                      "fine_box_cells_per_s": fine_cells / el,
                      "coarse_steps": {"value": k_rate, "unit": UNIT, "ms_per_step": kms / steps_k,
                                       "steps": steps_k}}

    # ---------------- the non-ideal and magnetic workloads ----------------
    # 512^3 / 40000 lognormal Laguerre grains under Read-Shockley physics (FP32
    # state and BF16 state) and 384^3 / 10000 grains with the magnetic driving
    # force: device-timed steps of each, with their own rooflines
    configs = None
    if not args.no_configs and rank == 0:
        configs = {}
        for name, key, st in (("512rs_fp32", "512rs", L.STORAGE_FP32), ("512rs_bf16", "512rs", L.STORAGE_BF16),
                              ("384mag", "384mag", L.STORAGE_FP32)):
            torch.cuda.synchronize()
            configs[name] = device_block(L, I, torch, WORKLOADS[key], local, args.config_steps, 3, st)

    # ---------------- step groups: many microstructures in one set of launches ----------------
    group = None
    if not args.no_compare and rank == 0:
        group = group_block(L, I, torch, local)

    # ---------------- serving: continuous batching under an HBM budget ----------------
    serving = None
    if args.serve_requests > 0 and rank == 0:
        serving = serving_run(L, I, args.serve_requests, local)

    # ---------------- reduce over ranks ----------------
    dev_ms, cells_all, e2e_s, e2e_cells_all = reduce_over_ranks(dev_ms, cells, e2e_s, e2e_cells, world)
    if rank != 0:
        return 0

    value = cells_all / (dev_ms * 1e-3)
    # roofline of the pass with the longest time per launch (its algorithmic bytes
    # per launch over its CUDA-event time), against the measured copy bandwidth
    peaks, src = measured_peaks()
    dom_cells = n ** 3
    box_cells_prof = cells_prof / kprof
    physics = WORKLOAD.get("physics", "ideal") != "ideal"
    pass_ms = {name: v[0] / max(1, v[1]) for name, v in ptimes.items() if v[1] > 0}
    if pass_ms:
        roof = kernel_roofline(pass_ms, tier_cells, box_cells_prof, float(dom_cells), g, peaks.get("hbm_gbs"), 4,
                               physics)
        dominant, units = roof["kernel"], roof["units_per_launch"]
    else:
        # box-streaming kernels: 8 B per box cell + the 16-byte field per domain cell
        per_launch_ms = {k: ktimes[k] / max(1, kprof) for k in ("k_predict", "k_correct")}
        dominant = max(per_launch_ms, key=per_launch_ms.get)
        units = box_cells_prof
        alg_bytes = 8.0 * box_cells_prof + 16.0 * dom_cells
        achieved = alg_bytes / (per_launch_ms[dominant] * 1e-3) / 1e9
        roof = {"bound": "hbm", "kernel": dominant, "achieved": achieved, "peak": peaks.get("hbm_gbs"),
                "unit": "GB/s", "frac": achieved / peaks.get("hbm_gbs"), "algorithmic_bytes_per_launch": alg_bytes,
                "units_per_launch": units, "launch_ms": per_launch_ms[dominant]}
    roof["peak_source"] = src
    roof["traffic"] = profiled_traffic(dominant, units)
    roof["traffic_source"] = ("dram__bytes_read.sum + dram__bytes_write.sum per launch from the ncu capture in "
                              "profiles/traffic.json, scaled by units processed" if roof["traffic"] is not None
                              else "no capture of the current pass kernels")
    cpu = None if args.no_cpu else cpu_baseline_block(2)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dev_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(),
        "domain_cell_updates_per_s": world * dom_cells * args.steps / (dev_ms * 1e-3),
        "box_cells_per_step": box_cells_mean,
        "superimposition": box_cells_mean / dom_cells,
        "kernel_ms_per_step": {k: v / max(1, kprof) for k, v in ktimes.items()},
        "pass_ms_per_step": pass_ms, "pass_cells_per_tier": tier_cells, "exec": args.exec,
        "tile_variants": tiles,
        "gpu_launches": int(sum(kcount.values()) * args.steps / max(1, kprof)),
        "roofline": roof,
        "step_roofline": step_roofline(box_cells_mean, dom_cells, dev_ms / args.steps, peaks.get("hbm_gbs"),
                                       bool(pass_ms), 4, physics),
        "e2e": None if args.no_e2e else {"value": e2e_cells_all / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": 8 * 3 * g / args.steps, "d2h_bytes_per_step": d2h / args.steps,
                "seconds": e2e_s, "includes": "create_microstructure from host seeds, steps, per-step volumes "
                                               "to host, final owner map to host (pinned host buffers)"},
        "cpu_baseline": cpu,
        "clocks": clk.summary(),
        "serving": serving,
        "configs": configs,
        "compare": compare,
        "step_group": group,
        "bf16_storage": bf16,
        "coarsening": coarsening,
        "size_analysis": statistics,
        "speedup_vs_plain_gpu": None if not compare else value / compare["plain_gpu"]["value"],
    }
    print(json.dumps(line), flush=True)
    return 0


def group_block(L, I, torch, device, steps=20):
    """Microstructures of one size advanced as one step group against the same
    ones on their own streams (all enqueued before waiting), CUDA events
    around each pass (a stream waiting for the others' work): 48 of 48^3 / 33
    grains, 16 of 96^3 / 263, 6 of 160^3 / 1221 (seeds 10 + k)."""
    out = {}
    for n, g, cnt in ((48, 33, 48), (96, 263, 16), (160, 1221, 6)):
        ms = [L.Microstructure(n, n, n, g, seeds=I.voronoi_seeds(10 + k, g, (n, n, n)), device=device)
              for k in range(cnt)]
        try:
            for m in ms:
                m.step(2, 1.0)
            for m in ms:
                m.sync()
            cells = sum(m.stats().box_cells for m in ms)

            def timed(run):
                torch.cuda.synchronize()
                s = torch.cuda.Stream()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(s)
                run()
                for m in ms:                       # s waits for every member's stream
                    e = torch.cuda.Event()
                    e.record(torch.cuda.ExternalStream(m.stream))
                    s.wait_event(e)
                b.record(s)
                b.synchronize()
                return a.elapsed_time(b)

            streams_ms = timed(lambda: [m.step(steps, 1.0) for m in ms])
            with L.Group(ms) as grp:
                grp.step(1, 1.0)
                for m in ms:
                    m.sync()
                group_ms = timed(lambda: grp.step(steps, 1.0))
            out[f"{cnt}x{n}^3"] = {"members": cnt, "box_cells_per_step": cells,
                                   "own_streams_ms_per_step": streams_ms / steps,
                                   "group_ms_per_step": group_ms / steps,
                                   "group_cell_updates_per_s": cells * steps / (group_ms * 1e-3),
                                   "speedup": streams_ms / group_ms}
        finally:
            for m in ms:
                m.close()
    return out


def _pct(sorted_vals, q):
    return sorted_vals[min(len(sorted_vals) - 1, max(0, int(math.ceil(q * len(sorted_vals))) - 1))]


def serve_stream(L, reqs, device, budget, max_active=64, steps_per_round=4, mode=None):
    """Submit requests at their arrival times (seconds from the start) and wait
    for all: per request latency = completion - arrival, the time queued
    before admission and the time from admission to completion."""
    lat, queued, service, cells = [], [], [], 0
    mode = L.SERVE_SHARED if mode is None else mode
    with L.Server(budget, max_active=max_active, steps_per_round=steps_per_round, device=device, mode=mode) as srv:
        start = time.perf_counter()
        tickets = []
        for r in reqs:
            delay = start + r.arrival - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            tickets.append((r, srv.submit(r.n, r.n, r.n, r.n_grains, r.steps, seed=r.seed)))
        for r, t in tickets:
            info = srv.wait(t)
            if info.state != 2:
                raise RuntimeError(f"request {r.index} failed with status {info.state}")
            lat.append(info.t_done - info.t_submit)
            queued.append(info.t_admit - info.t_submit)
            service.append(info.t_done - info.t_admit)
            cells += info.cell_updates
        wall = time.perf_counter() - start
        peak = srv.stats().peak_bytes
    lat, queued, service = sorted(lat), sorted(queued), sorted(service)
    return {"p50_s": _pct(lat, 0.5), "p99_s": _pct(lat, 0.99), "mean_s": sum(lat) / len(lat),
            "queued_p50_s": _pct(queued, 0.5), "queued_p99_s": _pct(queued, 0.99),
            "service_p50_s": _pct(service, 0.5), "service_p99_s": _pct(service, 0.99),
            "cell_updates": cells, "cell_updates_per_s": cells / wall, "wall_s": wall, "peak_admitted_bytes": peak}


def serving_run(L, I, n_requests, device):
    """The serving workload: independent simulations with cubic periodic
    domains N in {32, 48, ..., 256}, grains = N^3 / 3355 clamped to [20,
    5000], 10 to 200 steps, seeds 1000 + k, under an HBM budget of 150 GB.
    The closed-loop capacity (requests per second with all of a 32-request
    sample of the same distribution, seeds 5000 + k, submitted at once) sets
    the rates; the n_requests then arrive as a Poisson stream at 0.8x and at
    1.2x (overload) of that capacity.  Latency = completion - arrival.  The
    server runs with shared launches (one step group over the running
    requests); the same closed loop and the 0.8x stream are repeated with a
    stream per request (per_context) for comparison."""
    budget = 150 << 30
    probe = I.serving_requests(32, 1.0, base_seed=5000)
    for r in probe:
        r.arrival = 0.0
    closed = serve_stream(L, probe, device, budget)
    capacity = len(probe) / closed["wall_s"]
    out = {"requests": n_requests, "budget_bytes": budget, "max_active": 64, "mode": "shared launches",
           "capacity_per_s": capacity,
           "closed_loop": {"requests": len(probe), "cell_updates_per_s": closed["cell_updates_per_s"],
                           "wall_s": closed["wall_s"], "p50_s": closed["p50_s"], "p99_s": closed["p99_s"]},
           "rates": {}}
    for factor in (0.8, 1.2):
        reqs = I.serving_requests(n_requests, factor * capacity, base_seed=1000)
        res = serve_stream(L, reqs, device, budget)
        res["rate_per_s"] = factor * capacity
        out["rates"][f"{factor:.1f}x"] = res
    lo = out["rates"]["0.8x"]
    out.update(p50_s=lo["p50_s"], p99_s=lo["p99_s"], cell_updates_per_s=lo["cell_updates_per_s"],
               peak_admitted_bytes=max(r["peak_admitted_bytes"] for r in out["rates"].values()))
    pc_closed = serve_stream(L, probe, device, budget, mode=L.SERVE_PER_CONTEXT)
    pc = serve_stream(L, I.serving_requests(n_requests, 0.8 * capacity, base_seed=1000), device, budget,
                      mode=L.SERVE_PER_CONTEXT)
    out["per_context"] = {"closed_loop": {"cell_updates_per_s": pc_closed["cell_updates_per_s"],
                                          "wall_s": pc_closed["wall_s"], "capacity_per_s": len(probe) / pc_closed["wall_s"]},
                          "0.8x": {k: pc[k] for k in ("p50_s", "p99_s", "mean_s", "cell_updates_per_s", "wall_s")}}
    # small domains only (N in {32, 48, ..., 128}: the requests the step group
    # takes), 64 submitted at once, in both modes
    small = I.serving_requests(64, 1.0, base_seed=7000, sizes=tuple(range(32, 129, 16)))
    for r in small:
        r.arrival = 0.0
    sm = {m: serve_stream(L, small, device, budget, mode=mv)
          for m, mv in (("shared", L.SERVE_SHARED), ("per_context", L.SERVE_PER_CONTEXT))}
    out["small_domains_closed_loop"] = {"requests": len(small), "sizes": "32^3 to 128^3",
                                        **{m: {k: v[k] for k in ("cell_updates_per_s", "wall_s", "p50_s", "p99_s")}
                                           for m, v in sm.items()}}
    return out


def profile_step(args):
    """The profilers' case: create the workload, run the warm-up steps, print
    the box cells each tier's passes will process in the next step (one JSON
    line), run that one step and stop.  An ncu capture of the kernels of the
    last step (-s = warm-up launches) then has exact units for its bytes."""
    import torch
    from paper_1701_06658_gb300 import inputs as I
    from paper_1701_06658_gb300 import lsgg as L
    L.lib()
    n, g, dt = WORKLOAD["n"], WORKLOAD["grains"], WORKLOAD["dt"]
    seeds = I.voronoi_seeds(WORKLOAD["seed"], g, (n, n, n))
    with L.Microstructure(n, n, n, g, seeds=seeds, **workload_kwargs(L)) as ms:
        ms.step(args.warmup, dt)
        ms.sync()
        st = ms.stats()
        print(json.dumps({"workload": workload_config()["workload"], "warmup_steps": args.warmup,
                          "pass_cells_per_tier": list(st.pass_cells), "box_cells": st.box_cells,
                          "domain_cells": n ** 3}), flush=True)
        ms.step(1, dt)
        ms.sync()
        torch.cuda.synchronize()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end pass")
    ap.add_argument("--no-tune", action="store_true", help="skip the tile autotuner")
    ap.add_argument("--no-compare", action="store_true", help="skip the plain / box-streaming comparison runs")
    ap.add_argument("--exec", default="batched", choices=["batched", "streamed"],
                    help="batched: pass path for boxes of side <= 64; streamed: box-streaming kernels only")
    ap.add_argument("--serve-requests", type=int, default=256,
                    help="requests of the serving measurement at each of its two rates (0: skip)")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the 512^3 Read-Shockley (FP32, BF16) and 384^3 magnetic blocks")
    ap.add_argument("--config-steps", type=int, default=8, help="timed steps of each of those blocks")
    ap.add_argument("--profile-step", action="store_true",
                    help="profilers' case: warm-up steps, the next step's tier cells as JSON, one step")
    ap.add_argument("--redist", default="taxicab", choices=["taxicab", "godunov"],
                    help="re-initialisation metric: the paper's taxicab propagation or the Godunov update")
    ap.add_argument("--workload", default="256", choices=sorted(WORKLOADS),
                    help="256: the benchmark workload; 160, 160mag: small cases for profilers; "
                         "512rs, 384mag: the non-ideal and magnetic workloads")
    args = ap.parse_args()
    WORKLOAD.clear()
    WORKLOAD.update(WORKLOADS[args.workload])
    WORKLOAD["redist"] = args.redist
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return reference_arm(args)
    if args.profile_step:
        return profile_step(args)
    return gpu_arm(args)


if __name__ == "__main__":
    import numpy as np
    sys.exit(main())
