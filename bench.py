#!/usr/bin/env python
"""Benchmark of the tight-frame CBCT reconstruction hot path on GB300.

One step = one full reconstruction of the paper-scale workload through the C ABI:
512x512x70 voxels of 0.5x0.5x2.5 mm, 512x384 imager at 0.776 mm, 40 views (or --views 80),
3-level multigrid (128x128x18 -> 256x256x35 -> 512x512x70), 50 A2 iterations split 8/17/25
coarsest first (the paper's 1:2:3 proportions), 3 CGLS updates per iteration, mu = 5e-4,
on a seeded 30-ellipsoid torso phantom with Poisson noise at 5e4 photons per ray.

Metric: ray-voxel updates per second of P and P^T — the non-zeros of P (counted by the
projector itself on every level) times the number of P and P^T applications a
reconstruction performs (4 P and 3 P^T per A2 iteration), divided by the device time.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--views 40|80] [--impl ours|reference]

With --gpus N > 1 (launched by torch.distributed.run, one process per GPU) every rank
reconstructs its own phantom (independent problems, weak scaling); there is no data
exchange, only a host-side barrier and a max over ranks of the timed duration.
--impl reference times the FP64 CPU oracle on a bounded sample (a few views of the same
workload) in the same unit.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

METRIC = "ray-voxel updates/s (P+Pᵀ)"
UNIT = "updates/s"
MU = 5e-4
N_CGLS = 3
LEVELS = 3
TOTAL_ITERS = 50
PHOTONS = 5e4
# FP32 arithmetic operations counted per ray-voxel update in the secondary arithmetic model
# of the roofline: next plane-crossing parameter (FMA), nearest crossing (min), segment
# length (subtract), accumulation (FMA).
OPS_PER_UPDATE = 4
FP32_LANES_PER_SM = 128


def parse_args(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--views", type=int, default=40, choices=(40, 80))
    ap.add_argument("--impl", default="ours", choices=("ours", "reference"))
    ap.add_argument("--storage", default="f32", choices=("f32", "bf16", "f16"),
                    help="storage type of the CGLS residual and projected direction (arithmetic stays FP32)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the extra measurements (frame transforms, 16-bit storage, 80 views)")
    ap.add_argument("--cpu-views", type=int, default=40,
                    help="views in the oracle's bounded sample (CPU baseline); the reference arm uses 16 per step")
    return ap.parse_args(argv)


def workload(views: int):
    geom = synth.config_paper(views)
    iters = synth.default_level_iters(LEVELS, TOTAL_ITERS)
    return geom, iters


def workload_config(geom, iters, extra=None):
    cfg = {
        "workload": (f"paper-scale TF-regularised CBCT reconstruction: {geom.nx}x{geom.ny}x{geom.nz} voxels "
                     f"({geom.dx}x{geom.dy}x{geom.dz} mm), {geom.nu}x{geom.nv} imager at {geom.du} mm, "
                     f"{geom.n_views} views, {LEVELS}-level multigrid, A2 iterations {iters} coarsest first, "
                     f"{N_CGLS} CGLS updates each, mu={MU}"),
        "volume": [geom.nx, geom.ny, geom.nz],
        "views": geom.n_views,
        "imager": [geom.nu, geom.nv],
        "levels": LEVELS,
        "iters_per_level": iters,
        "n_cgls": N_CGLS,
        "l2": "working set per step ~2.5 GB (> 126 MB L2); L2 also flushed (1 GiB write) before every timed step",
    }
    if extra:
        cfg.update(extra)
    return cfg


# ---------------------------------------------------------------------------------------
# Distributed plumbing (host-side only: timing scalars, no data exchange)
# ---------------------------------------------------------------------------------------

def dist_info():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def dist_init(world):
    if world <= 1:
        return None
    import torch.distributed as dist
    if not dist.is_initialized():
        dist.init_process_group("gloo")
    return dist


def aggregate(local_seconds: float, local_units: float, dist=None):
    """Whole-job numbers: max over ranks of the timed duration, sum over ranks of the work."""
    if dist is None:
        return local_seconds, local_units
    import torch
    t = torch.tensor([local_seconds], dtype=torch.float64)
    u = torch.tensor([local_units], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


# ---------------------------------------------------------------------------------------
# Clock sampling during the timed region
# ---------------------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
                power.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm),
                "reasons": sorted(reasons)}


def stored_counters(kernel: str):
    """Per-level ncu counters of `kernel` (one launch per multigrid level, profiles/kernels.json,
    written by paper_1008_2042_gb300.profile_counters), or None when the kernel's sources
    changed since that capture (or there is none)."""
    from paper_1008_2042_gb300.profile_counters import kernel_sources_sha
    try:
        with open(os.path.join(ROOT, "profiles", "kernels.json")) as fh:
            rec = json.load(fh).get(kernel)
    except (OSError, ValueError):
        return None
    if not rec or rec.get("sources_sha256") != kernel_sources_sha(kernel):
        return None
    return rec.get("levels")


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


# ---------------------------------------------------------------------------------------
# Frame transforms against the HBM roofline
# ---------------------------------------------------------------------------------------

def time_frame_transforms(cb, geom, device, reps: int = 10, mu: float = MU):
    """Device time of the public analysis W (cbct_tf_analyze) and shrink + synthesis
    (cbct_tf_synthesize_shrink) on the workload's finest grid, FP32 and BF16 coefficients:
    median of `reps` calls, each bracketed by CUDA events on the launching stream. The
    coefficient array (1.98 GB in FP32, 0.99 GB in BF16) exceeds L2, so every call streams
    it from HBM. Algorithmic bytes per voxel: W reads 4 and writes 27 coefficients, the
    synthesis reads 27 coefficients and writes 4."""
    import torch
    peak = float(measured_peaks().get("hbm_gbs") or 6800.0)
    stream = torch.cuda.current_stream()
    n = geom.nx * geom.ny * geom.nz
    gen = torch.Generator(device=device).manual_seed(5)
    f = torch.rand(geom.vol_shape, device=device, generator=gen) * 0.04
    out = torch.empty_like(f)
    res = {}
    for name, dt, es in (("f32", torch.float32, 4), ("bf16", torch.bfloat16, 2)):
        alpha = torch.empty((27,) + tuple(geom.vol_shape), dtype=dt, device=device)
        for op in ("analyze", "synthesize_shrink"):
            def call():
                if op == "analyze":
                    cb.tf_analyze(f, out=alpha)
                else:
                    cb.tf_synthesize_shrink(alpha, mu, True, out=out)
            call()
            torch.cuda.synchronize()
            ms = []
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                call()
                e1.record(stream)
                e1.synchronize()
                ms.append(e0.elapsed_time(e1))
            t = statistics.median(ms)
            nbytes = n * (4 + 27 * es)
            gbs = nbytes / (t / 1e3) / 1e9
            res[f"{op}_{name}"] = {"ms": round(t, 4), "bytes": nbytes, "gbs": round(gbs, 1),
                                    "frac": round(gbs / peak, 4)}
        del alpha
    res["peak_gbs"] = peak
    res["peak_source"] = "MEASURED_PEAKS.json hbm_gbs (measured copy bandwidth)"
    return res


# ---------------------------------------------------------------------------------------
# CPU baseline: the FP64 oracle on a bounded sample of the workload
# ---------------------------------------------------------------------------------------

def oracle_sample(geom, n_views: int, seed: int):
    """P + P^T of the oracle on the first n_views views; returns (updates, seconds, cores)."""
    import dataclasses
    import oracle
    sub = dataclasses.replace(geom, n_views=n_views, angles=tuple(geom.view_angles()[:n_views]))
    f = synth.voxelize(sub, synth.torso_ellipsoids(sub, 1002))
    y = synth.random_projections(sub, seed)
    nnz = oracle.count_nnz(sub)
    t0 = time.perf_counter()
    oracle.project(sub, f)
    oracle.backproject(sub, y)
    dt = time.perf_counter() - t0
    return 2 * nnz, dt, oracle.num_threads()


def run_reference(args):
    world, rank, _ = dist_info()
    if rank != 0:
        return 0
    geom, iters = workload(args.views)
    import oracle
    oracle.build()
    for _ in range(args.warmup):
        oracle_sample(geom, 1, 7)
    upd, secs, cores = 0.0, 0.0, oracle.num_threads()
    for k in range(args.steps):
        u, s, cores = oracle_sample(geom, min(args.cpu_views, 16), 100 + k)
        upd += u
        secs += s
    value = upd / secs
    sample = (f"P + P^T of {min(args.cpu_views, 16)} of the {geom.n_views} views per step "
              f"(nnz counted by the oracle)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic torso phantom (30 ellipsoids), uniform random projections",
        "config": workload_config(geom, iters, {"sample": sample,
                                                "l2": "not applicable: the FP64 oracle runs on the host cores"}),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------------------
# The CUDA path
# ---------------------------------------------------------------------------------------

def make_problem(cb, geom, dev, rank: int):
    """The benchmark's input on `geom`: the seeded torso phantom (seed 1002), projected by
    the library's P, with Poisson noise at PHOTONS per ray (seed 2002 + rank). The same
    phantom and noise seed, projected by the oracle, are the input of the paper-scale
    reconstruction parity test, which also checks the library's P of this phantom against
    the oracle's over the whole stack."""
    import torch
    g = cb.Geometry(geom)
    f_true = torch.tensor(synth.voxelize(geom, synth.torso_ellipsoids(geom, 1002)), dtype=torch.float32, device=dev)
    p_ideal = cb.project(g, f_true).double().cpu().numpy()
    y_host = torch.tensor(synth.noisy_line_integrals(p_ideal, PHOTONS, 2002 + rank), dtype=torch.float32).pin_memory()
    nnz = [cb.count_nnz(g, lev) for lev in range(LEVELS)]  # level 0 = finest
    return g, y_host, nnz


def launches_per_level(iters):
    """P and P^T launches a reconstruction makes on each level (level 0 = finest):
    n_cgls + 1 P and n_cgls P^T per A2 iteration."""
    return ([iters[LEVELS - 1 - lev] * (N_CGLS + 1) for lev in range(LEVELS)],
            [iters[LEVELS - 1 - lev] * N_CGLS for lev in range(LEVELS)])


def time_reconstructions(cb, g, y, iters, steps, flush, storage="f32", ws=None, out=None):
    """Device seconds per reconstruction: mean of `steps` runs after one warm-up, each
    bracketed by CUDA events on the launching stream, the L2 flushed before each."""
    import torch
    stream = torch.cuda.current_stream()
    cb.reconstruct(g, y, MU, LEVELS, iters, n_cgls=N_CGLS, workspace=ws, out=out, storage=storage)
    torch.cuda.synchronize()
    total = 0.0
    for k in range(steps):
        flush.fill_(float(k))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        cb.reconstruct(g, y, MU, LEVELS, iters, n_cgls=N_CGLS, workspace=ws, out=out, storage=storage)
        e1.record(stream)
        e1.synchronize()
        total += e0.elapsed_time(e1) / 1e3
    return total / steps


def run_ours(args):
    import torch

    world, rank, local = dist_info()
    dist = dist_init(world)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1008_2042_gb300 import build as cuda_build
    cuda_build.build()
    import paper_1008_2042_gb300 as cb

    geom, iters = workload(args.views)
    g, y_host, nnz = make_problem(cb, geom, dev, rank)
    y = y_host.to(dev)
    np_lev, npt_lev = launches_per_level(iters)
    updates_P = sum(np_lev[lev] * nnz[lev] for lev in range(LEVELS))
    updates_PT = sum(npt_lev[lev] * nnz[lev] for lev in range(LEVELS))
    updates = updates_P + updates_PT

    ws = torch.empty(cb.reconstruct_workspace_size(g), dtype=torch.uint8, device=dev)
    out = torch.empty(geom.vol_shape, dtype=torch.float32, device=dev)
    flush = torch.empty(1 << 28, dtype=torch.float32, device=dev)  # 1 GiB
    stream = torch.cuda.current_stream()

    def step(y_in, o):
        cb.reconstruct(g, y_in, MU, LEVELS, iters, n_cgls=N_CGLS, workspace=ws, out=o, storage=args.storage)

    for _ in range(max(args.warmup, 0)):
        step(y, out)
    torch.cuda.synchronize()

    # ---- device-timed region: inputs resident in HBM ----
    gpu_id = "GPU-" + str(torch.cuda.get_device_properties(local).uuid) if hasattr(
        torch.cuda.get_device_properties(local), "uuid") else str(local)
    sampler = ClockSampler(gpu_id)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    cb.profiling_reset()
    # per-launch events on the two dominant kernels only (their launches take milliseconds,
    # so the events cost nothing measurable); the short kernels run untimed
    cb.profiling_select(["project", "backproject"])
    launches0 = cb.launch_count()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for k in range(args.steps):
        flush.fill_(float(k))
        ev[k][0].record(stream)
        step(y, out)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    launches = cb.launch_count() - launches0
    cb.profiling(False)
    ktimes = cb.kernel_times()
    # one more (untimed) step with every launch timed: device time per kernel family
    cb.profiling_reset()
    cb.profiling(True)
    step(y, out)
    torch.cuda.synchronize()
    cb.profiling(False)
    family_ms = {k: v[0] for k, v in cb.kernel_times().items()}
    cb.profiling_reset()
    clocks = sampler.stop()
    if dist is not None:
        dist.barrier()
    local_s = sum(a.elapsed_time(b) for a, b in ev) / 1e3
    secs, total_updates = aggregate(local_s, updates * args.steps, dist)
    value = total_updates / secs

    # ---- end to end through the public API: host buffers, copies inside the timed region;
    # the same L2 flush as above before every step, outside its event pair ----
    out_host = torch.empty(geom.vol_shape, dtype=torch.float32).pin_memory()
    y_dev = torch.empty_like(y)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    ee = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for k in range(args.steps):
        flush.fill_(float(k))
        ee[k][0].record(stream)
        y_dev.copy_(y_host, non_blocking=True)
        step(y_dev, out)
        out_host.copy_(out, non_blocking=True)
        ee[k][1].record(stream)
    torch.cuda.synchronize()
    e2e_s, _ = aggregate(sum(a.elapsed_time(b) for a, b in ee) / 1e3, 0.0, dist)
    e2e_value = total_updates / e2e_s

    # ---- roofline of the dominant kernel (P or P^T), from the live event timings ----
    peaks = measured_peaks()
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    sm_max = float(peaks.get("sm_max_mhz") or clocks.get("sm_max_mhz") or 2070.0)
    alu_peak = sms * FP32_LANES_PER_SM * sm_max * 1e6 / 1e12  # T thread instructions/s (one per lane per clock)
    ms_p, n_p = ktimes["project"]
    ms_pt, n_pt = ktimes["backproject"]
    if ms_p >= ms_pt:
        dom, kname, ms_dom, n_dom, upd_dom, per_lev = ("project (P, Siddon column sweep)", "k_project", ms_p, n_p,
                                                       updates_P * args.steps, np_lev)
    else:
        dom, kname, ms_dom, n_dom, upd_dom, per_lev = ("backproject (exact P^T gather)", "k_backproject", ms_pt,
                                                       n_pt, updates_PT * args.steps, npt_lev)
    avg_s = ms_dom / max(n_dom, 1) / 1e3
    counters = stored_counters(kname)
    roofline = {
        "bound": "alu", "kernel": dom, "unit": "T thread-instructions/s", "peak": alu_peak,
        "peak_source": f"{sms} SMs x {FP32_LANES_PER_SM} lanes x {sm_max:.0f} MHz: one instruction per lane per clock "
                       f"(no pipe, L1 or DRAM saturates: the kernel is issue- and latency-bound)",
        "avg_launch_ms": avg_s * 1e3,
        "kernel_share": {k: round(v / sum(family_ms.values()), 4) for k, v in family_ms.items()}
        if sum(family_ms.values()) else {},
    }
    # secondary arithmetic model: OPS_PER_UPDATE FP32 operations per ray-voxel update
    model = (upd_dom * OPS_PER_UPDATE / max(n_dom, 1)) / avg_s / 1e12
    roofline["model_4ops_per_update"] = {"achieved": model, "frac": model / alu_peak}
    if counters:
        # instructions and DRAM bytes the step's launches execute, from one ncu launch per level
        # weighted by the launches per level, over the live average launch time
        w = [per_lev[lev] * args.steps for lev in range(LEVELS)]
        tot = sum(w)
        inst = sum(w[lev] * counters[str(lev)]["thread_inst"] for lev in range(LEVELS)) / tot
        traffic = sum(w[lev] * (counters[str(lev)]["dram_read_bytes"] + counters[str(lev)]["dram_write_bytes"])
                      for lev in range(LEVELS)) / tot
        roofline.update({
            "achieved": inst / avg_s / 1e12, "frac": inst / avg_s / 1e12 / alu_peak, "traffic": traffic,
            "achieved_basis": "thread instructions per launch (ncu smsp__thread_inst_executed.sum, one launch per "
                              "level, weighted by the step's launches per level) / live average launch duration",
            "issue_active_ncu_pct": {lev: counters[lev]["issue_active_pct"] for lev in counters},
            "l1_throughput_ncu_pct": {lev: counters[lev]["l1_throughput_pct"] for lev in counters},
            "thread_inst_per_update": {str(lev): counters[str(lev)]["thread_inst"] / nnz[lev] for lev in range(LEVELS)},
            "counters": "profiles/kernels.json",
        })
    else:
        roofline.update({"achieved": model, "frac": model / alu_peak, "traffic": None,
                         "achieved_basis": f"{OPS_PER_UPDATE} FP32 operations per ray-voxel update (no ncu counters "
                                           f"for the current kernel sources)"})
    # compulsory DRAM bytes of P at the finest level: read the volume, write the stack
    n0 = geom.nx * geom.ny * geom.nz
    m0 = geom.n_views * geom.nv * geom.nu
    roofline["hbm_compulsory_gbs"] = 4.0 * (n0 + m0) / avg_s / 1e9

    extra = {}
    if rank == 0 and world == 1 and not args.no_extra:
        # the public frame transforms against HBM; the reconstruction with 16-bit CGLS vectors
        # and at 80 views (the second view count of the workload)
        extra["frame_transforms_hbm"] = time_frame_transforms(cb, geom, dev)
        for st in ("bf16", "f16"):
            if st != args.storage:
                extra[f"recon_seconds_{st}_storage"] = time_reconstructions(cb, g, y, iters, 3, flush, st, ws, out)
        if args.views == 40:
            del ws
            g80, y80_host, nnz80 = make_problem(cb, synth.config_paper(80), dev, rank)
            ws80 = torch.empty(cb.reconstruct_workspace_size(g80), dtype=torch.uint8, device=dev)
            t80 = time_reconstructions(cb, g80, y80_host.to(dev), iters, 3, flush, args.storage, ws80, out)
            np80, npt80 = launches_per_level(iters)
            u80 = sum((np80[lev] + npt80[lev]) * nnz80[lev] for lev in range(LEVELS))
            extra["recon_80_views"] = {"seconds": t80, "updates_per_s": u80 / t80, "nnz_per_P": nnz80,
                                       "storage": args.storage}
            g80.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            u, s_, cores = oracle_sample(geom, args.cpu_views, 3003)
            cpu = {"value": u / s_, "unit": UNIT, "cores": cores, "kind": "oracle",
                   "sample": f"P + P^T of {args.cpu_views} of the {geom.n_views} views of the same workload "
                             f"({s_:.1f} s)"}
        except Exception as exc:  # the oracle is a reported baseline only
            cpu = {"value": None, "unit": UNIT, "cores": None, "kind": "oracle", "sample": f"failed: {exc}"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic: seeded 30-ellipsoid torso phantom, Poisson noise 5e4 photons/ray (per-rank seeds)",
            "config": workload_config(geom, iters, {"nnz_per_P": nnz,
                                                    "updates_per_step": updates,
                                                    "recon_seconds": secs / args.steps,
                                                    "cgls_vector_storage": args.storage,
                                                    "parallelism": f"replicas x{world}"}),
            "e2e": {"value": e2e_value, "unit": UNIT,
                    "h2d_bytes_per_step": int(y_host.numel() * 4),
                    "d2h_bytes_per_step": int(out_host.numel() * 4),
                    "ms_per_step": 1e3 * e2e_s / args.steps},
            "gpu_launches": int(launches),
            "roofline": roofline,
            "kernel_ms_timed_steps": {k: ktimes[k][0] for k in ("project", "backproject")},
            "kernel_launches_timed_steps": {k: ktimes[k][1] for k in ("project", "backproject")},
            "family_ms_one_profiled_step": family_ms,
            "clocks": clocks,
        }
        line.update(extra)
        if cpu is not None:
            line["cpu_baseline"] = cpu
        print(json.dumps(line), flush=True)
    g.close()
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
