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
    # magnetically driven growth: random c-axes, field (0, cos 32, sin 32), bulk
    # energy B^2 dchi cos^2 / (2 mu0) in grid units (4.07e-3 at cos^2 = 1)
    "384mag": {"n": 384, "grains": 10000, "seed": 4, "dt": 1.0, "physics": "magnetic", "energy_scale": 4.07e-3},
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
                       "paper_1701_06658_gb300/csrc/kernels_common.cuh",
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


def step_roofline(box_cells: float, dom_cells: float, ms_per_step: float, peak_gbs: float, passes: bool):
    """The whole step against the bytes the method must move at least (one
    FP32 read and write of phi per box cell, 44 B of top-two field per domain
    cell: 16 cleared, 16 written, 12 read) and against the bytes of this
    design's five passes (44 B per box cell: 8 each for the x/y and z
    convolution and re-initialisation passes, 12 for the field pass; 16 B of
    field per domain cell), both over the measured step time."""
    minimum = 8.0 * box_cells + 44.0 * dom_cells
    design = (44.0 * box_cells + 16.0 * dom_cells) if passes else None
    t = ms_per_step * 1e-3
    out = {"minimum_bytes_per_step": minimum, "minimum_bound_ms": minimum / (peak_gbs * 1e9) * 1e3,
           "achieved_minimum_gbs": minimum / t / 1e9, "frac_minimum": minimum / t / 1e9 / peak_gbs,
           "peak": peak_gbs, "unit": "GB/s"}
    if design is not None:
        out.update(design_bytes_per_step=design, achieved_design_gbs=design / t / 1e9,
                   frac_design=design / t / 1e9 / peak_gbs)
    return out


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

def oracle_sample_run(steps: int, warmup: int):
    """The FP64 oracle on the bounded sample: 64^3 periodic domain, 78 Voronoi
    grains (seed 2), dt = 1; returns (cell-updates/s, seconds, cell-updates)."""
    from oracle import lsgg_oracle as O
    from paper_1701_06658_gb300 import inputs as I
    n, g = SAMPLE["n"], SAMPLE["grains"]
    ms = O.tessellate((n, n, n), I.voronoi_seeds(SAMPLE["seed"], g, (n, n, n)))
    for _ in range(warmup):
        ms = O.step(ms, 1.0)
    cells = 0
    t0 = time.perf_counter()
    for _ in range(steps):
        cells += sum(int(np.prod(gr.dims)) for gr in ms.grains if gr.alive)
        ms = O.step(ms, 1.0)
    dt = time.perf_counter() - t0
    return cells / dt, dt, cells


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
            "cpu_baseline": {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
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


def workload_kwargs(L):
    """Microstructure keyword arguments of the workload's physics and tessellation."""
    kw = {}
    ph = WORKLOAD.get("physics", "ideal")
    if ph == "read_shockley":
        kw["physics"] = L.PHYSICS_READ_SHOCKLEY
    elif ph == "magnetic":
        kw["physics"] = L.PHYSICS_MAGNETIC
        kw["energy_scale"] = WORKLOAD["energy_scale"]
    if WORKLOAD.get("init") == "laguerre":
        kw["init_kind"] = L.INIT_LAGUERRE
    if WORKLOAD.get("redist") == "godunov":
        kw["redist"] = L.REDIST_GODUNOV
    return kw


def workload_config():
    ph = {"ideal": "ideal growth", "read_shockley": "Read-Shockley energy and step mobility, random cubic orientations",
          "magnetic": "magnetic driving force, random c-axes"}[WORKLOAD.get("physics", "ideal")]
    tess = ("Laguerre grains, lognormal radii sigma 0.5, 1 % at 5x volume" if WORKLOAD.get("init") == "laguerre"
            else "Voronoi grains")
    rd = "" if WORKLOAD.get("redist", "taxicab") == "taxicab" else ", Godunov re-initialisation"
    return {"workload": f"{WORKLOAD['n']}^3 periodic, {WORKLOAD['grains']} {tess} (seed {WORKLOAD['seed']}), "
                        f"{ph}{rd}, dt={WORKLOAD['dt']}, box halo 5, eps 7, FP32",
            "domain": [WORKLOAD["n"]] * 3, "grains": WORKLOAD["grains"], "dt": WORKLOAD["dt"],
            "l2": f"inputs larger than L2: box arenas of ~{WORKLOAD['n'] ** 3 * 8.5 * 4 / 1e9:.1f} GB each and a "
                  f"{16 * WORKLOAD['n'] ** 3 / 1e6:.0f} MB field vs 129 MB L2"}


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
    tiles = L.autotune(ms.ctx, 2, dt) if not args.no_tune else None   # untimed: 6 real steps
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
        t0 = time.perf_counter()
        e2e = L.Microstructure(n, n, n, g, seeds=seeds, device=local,    # H2D of the seeds, init
                               exec_mode=exec_mode, **workload_kwargs(L))
        for _ in range(args.steps):
            e2e.step(1, dt)
            vol = e2e.grain_volumes()                                      # D2H of the step's result
            d2h += vol.nbytes
        own = e2e.voxel_owner()
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

    # ---------------- serving: continuous batching under an HBM budget ----------------
    serving = None
    if args.serve_requests > 0 and rank == 0:
        serving = serving_run(L, I, args.serve_requests, local)

    # ---------------- reduce over ranks ----------------
    dev_ms, cells_all, e2e_s, e2e_cells_all = reduce_over_ranks(dev_ms, cells, e2e_s, e2e_cells, world)
    if rank != 0:
        return 0

    value = cells_all / (dev_ms * 1e-3)
    # roofline of the dominant kernel (algorithmic bytes: 8 B per box cell + 16 B per domain cell)
    peaks, src = measured_peaks()
    dom_cells = n ** 3
    box_cells_prof = cells_prof / kprof
    pass_ms = {name: v[0] / max(1, v[1]) for name, v in ptimes.items() if v[1] > 0}
    if pass_ms:
        # pass path: the per-tier passes move 8 B per box cell of their tier (one
        # FP32 read, one FP32 write); the field pass reads phi_p twice, writes
        # phi_c (12 B per box cell) and stores the 16-byte field per domain cell
        dominant = max(pass_ms, key=pass_ms.get)
        if dominant == "p_field":
            units = box_cells_prof
            alg_bytes = 12.0 * units + 16.0 * dom_cells
        elif dominant == "k_bin":
            units, alg_bytes = float(g), 32.0 * g
        else:
            units = float(tier_cells[int(dominant[-2])])
            alg_bytes = 8.0 * units
        dom_ms = pass_ms[dominant]
    else:
        # box-streaming kernels: 8 B per box cell + the 16-byte field per domain cell
        per_launch_ms = {k: ktimes[k] / max(1, kprof) for k in ("k_predict", "k_correct")}
        dominant = max(per_launch_ms, key=per_launch_ms.get)
        units = box_cells_prof
        alg_bytes = 8.0 * box_cells_prof + 16.0 * dom_cells
        dom_ms = per_launch_ms[dominant]
    achieved = alg_bytes / (dom_ms * 1e-3) / 1e9
    traffic = profiled_traffic(dominant, units)
    cpu_rate, cpu_s, cpu_cells = oracle_sample_run(steps=2, warmup=0) if not args.no_cpu else (None, 0, 0)
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
        "roofline": {"bound": "hbm", "kernel": dominant, "achieved": achieved,
                     "peak": peaks.get("hbm_gbs"), "unit": "GB/s",
                     "frac": achieved / peaks.get("hbm_gbs"), "peak_source": src,
                     "algorithmic_bytes_per_launch": alg_bytes, "traffic": traffic},
        "step_roofline": step_roofline(box_cells_mean, dom_cells, dev_ms / args.steps, peaks.get("hbm_gbs"),
                                       bool(pass_ms)),
        "e2e": None if args.no_e2e else {"value": e2e_cells_all / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": 8 * 3 * g / args.steps, "d2h_bytes_per_step": d2h / args.steps,
                "seconds": e2e_s, "includes": "create_microstructure from host seeds, steps, per-step volumes "
                                               "to host, final owner map to host"},
        "cpu_baseline": None if cpu_rate is None else {
            "value": cpu_rate, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"2 oracle steps of a {SAMPLE['n']}^3 periodic sub-domain at the workload's grain "
                      f"density ({SAMPLE['grains']} grains), {cpu_s:.1f} s"},
        "clocks": clk.summary(),
        "serving": serving,
        "compare": compare,
        "bf16_storage": bf16,
        "coarsening": coarsening,
        "size_analysis": statistics,
        "speedup_vs_plain_gpu": None if not compare else value / compare["plain_gpu"]["value"],
    }
    print(json.dumps(line), flush=True)
    return 0


def serving_run(L, I, n_requests, device):
    """Requests drawn from the serving workload (cubic periodic domains 32..256,
    grains = N^3/3355 clamped to [20, 5000], 10..200 steps), HBM budget 150 GB.
    Closed loop first (all submitted at once) to measure capacity in requests/s,
    then Poisson arrivals at 0.8 x capacity: latency = completion - arrival."""
    budget = 150 << 30
    probe = I.serving_requests(min(16, n_requests), 1.0, base_seed=5000)
    with L.Server(budget, max_active=64, steps_per_round=4, device=device) as srv:
        t0 = time.perf_counter()
        tk = [srv.submit(r.n, r.n, r.n, r.n_grains, r.steps, seed=r.seed) for r in probe]
        infos = [srv.wait(t) for t in tk]
        closed_s = time.perf_counter() - t0
        closed_cells = sum(i.cell_updates for i in infos)
    capacity = len(probe) / closed_s
    reqs = I.serving_requests(n_requests, 0.8 * capacity, base_seed=1000)
    lat, cells = [], 0
    with L.Server(budget, max_active=64, steps_per_round=4, device=device) as srv:
        start = time.perf_counter()
        tickets = []
        for r in reqs:
            delay = start + r.arrival - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            tickets.append((r, srv.submit(r.n, r.n, r.n, r.n_grains, r.steps, seed=r.seed)))
        for r, t in tickets:
            info = srv.wait(t)
            lat.append(info.t_done - info.t_submit)
            cells += info.cell_updates
        wall = time.perf_counter() - start
        peak = srv.stats().peak_bytes
    lat = sorted(lat)
    pct = lambda q: lat[min(len(lat) - 1, int(math.ceil(q * len(lat))) - 1)]
    return {"requests": n_requests, "rate_per_s": 0.8 * capacity, "capacity_per_s": capacity,
            "closed_loop_cell_updates_per_s": closed_cells / closed_s,
            "p50_s": pct(0.50), "p99_s": pct(0.99), "mean_s": sum(lat) / len(lat),
            "cell_updates_per_s": cells / wall, "wall_s": wall, "peak_admitted_bytes": peak,
            "budget_bytes": budget}


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
    ap.add_argument("--serve-requests", type=int, default=24,
                    help="requests of the serving measurement (0: skip; 256: the full serving workload)")
    ap.add_argument("--redist", default="taxicab", choices=["taxicab", "godunov"],
                    help="re-initialisation metric: the paper's taxicab propagation or the Godunov update")
    ap.add_argument("--workload", default="256", choices=sorted(WORKLOADS),
                    help="256: the benchmark workload; 160: a small case of the same density for profilers; "
                         "512rs, 384mag: the non-ideal and magnetic workloads")
    args = ap.parse_args()
    WORKLOAD.clear()
    WORKLOAD.update(WORKLOADS[args.workload])
    WORKLOAD["redist"] = args.redist
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return reference_arm(args)
    return gpu_arm(args)


if __name__ == "__main__":
    import numpy as np
    sys.exit(main())
