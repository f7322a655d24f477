"""Throughput of the SOC hot path on GB300: photon-cell steps per second.

One step = one pass of the whole path over the 128^3 lognormal cloud
(sigma_lnrho 1.5, P(k) ~ k^-3.5), 64 log-spaced frequencies 3e11-3e15 Hz,
1e6 background packages per frequency (HG g = 0.5, kappa ~ nu^2 with a smooth
albedo, 3-blackbody background): counter reset, the persistent tracer over
all 64 frequencies in one launch, the FP64 absorbed-power integral and the
temperature update.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line.  --impl reference times the CPU oracle (the reference
arm of this project) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import tempfile
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

BYTES_PER_STEP = 12          # 4 B cell word read + 8 B int64 counter update per photon-cell step
N_PACKAGES = 1_000_000
WORKLOAD = "lognormal 128^3, 64 nu (3e11-3e15 Hz), 1e6 background packages/nu, HG g=0.5, FP64 T update"


# DRAM bytes (read + write) per photon-cell step of trace_kernel from one ncu
# capture (small case of the same workload, scaled by steps), valid only for
# the kernel source it was taken on.
TRACE_DRAM = {"source_sha1": "0195c78cace870d5542a5cb2f8fcc31015d7c503", "bytes_per_step": 2.2797,
              "warp_instructions_per_step": 7.758, "l2_bytes_per_step": 73.00,
              "profile": "profiles/trace_kernel_lognormal128_8nu_1e6pkg_full.md"}
# issue-rate peak: 4 warp-instructions per cycle per SM (4 schedulers)
ISSUE_PER_SM_CYCLE = 4
# FP32 operations one photon-cell step of the method needs (no scattering),
# counted from the FP32 contract: exit distances 3 x (sub, mul) + 3 compares;
# scattering depth (rho ksca) h, x s and 2 compares; absorption depth
# ((rho kabs) h) sp and 1 compare; 1 - e^-tau ~20 (reduction + degree-7
# polynomial, or the short series); deposit float(W) x q and its rounding 3;
# tau_f update 1; the move 3 x (mul, add, min, max)
FP32_OPS_PER_STEP = 54
FP32_LANES_PER_SM = 128


def _trace_source_sha1():
    import hashlib
    h = hashlib.sha1()
    for f in ("soc_trace.cu", "soc_fp32.cuh", "soc_internal.h"):
        with open(os.path.join(ROOT, "paper_1812_06632_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def _traffic_per_launch(steps):
    if TRACE_DRAM["source_sha1"] and TRACE_DRAM["source_sha1"] == _trace_source_sha1():
        return TRACE_DRAM["bytes_per_step"] * steps
    return None


def _issue_roofline(steps, ms, sms, clock_mhz):
    """Instruction-issue roofline of the tracer: warp instructions per step
    (ncu, same kernel source) x steps / time, against 4 per cycle per SM."""
    if not (TRACE_DRAM["source_sha1"] == _trace_source_sha1() and clock_mhz):
        return None
    achieved = TRACE_DRAM["warp_instructions_per_step"] * steps / (ms / 1e3)
    peak = ISSUE_PER_SM_CYCLE * sms * clock_mhz * 1e6
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "warp-instructions/s",
            "frac": achieved / peak, "instructions_per_unit": TRACE_DRAM["warp_instructions_per_step"],
            "peak_source": f"4 issue slots/cycle/SM x {sms} SMs x {clock_mhz:.0f} MHz (median SM clock in the run)"}


def l2_bandwidth(ctx, mib: int = 32, reps: int = 64):
    """Read bandwidth (GB/s) through L2 of this GPU: the library's read probe
    (16-byte loads that bypass L1, four in flight per thread) over a `mib`
    MiB buffer, `reps` passes in one launch, timed with CUDA events on the
    launching stream; best of 5 launches.  A buffer well inside L2 gives the
    L2 read bandwidth; one far larger than L2 gives HBM's."""
    import torch
    buf = torch.ones(mib << 18, dtype=torch.float32, device="cuda")
    s = torch.cuda.current_stream()
    for _ in range(2):
        ctx.probe_read(buf, reps, stream=s)
    best = float("inf")
    for _ in range(5):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        ctx.probe_read(buf, reps, stream=s)
        b.record(s)
        torch.cuda.synchronize()
        best = min(best, a.elapsed_time(b))
    return buf.numel() * 4 * reps / (best / 1e3) / 1e9


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# ---------------------------------------------------------------------------
# CPU oracle on a bounded sample (worker processes are spawned)
# ---------------------------------------------------------------------------
def _oracle_worker(args):
    """The oracle (FP32 contract, then FP64 on an eighth of the packages) on
    background packages pid_lo .. pid_lo + n - 1 of the given frequencies."""
    sys.path.insert(0, ROOT)
    freqs, pid_lo, n = args
    from paper_1812_06632_gb300 import inputs as I
    import oracle
    w = _workload_cache(I)
    cl = w.clouds[0]
    G = oracle.Grid(cl.nx, cl.ny, cl.nz, cl.level_start, cl.rho, cl.child, cl.parent)

    def kappa(f):        # FP32 opacity per root-cell length, as the library derives it
        return (np.float32(np.float64(w.dust.kabs[f]) * np.float64(cl.ell)),
                np.float32(np.float64(w.dust.ksca[f]) * np.float64(cl.ell)))

    steps = 0
    t0 = time.perf_counter()
    for f in freqs:
        ka, ks = kappa(f)
        _, st, _ = oracle.trace(G, source=0, kabs=ka, ksca=ks, g=np.float32(w.dust.g[f]), seed=w.seed, freq=f,
                                pid_lo=pid_lo, n_packages=n)
        steps += st["steps"]
    t_fp32 = time.perf_counter() - t0
    steps64 = 0
    t0 = time.perf_counter()
    for f in freqs:
        ka, ks = kappa(f)
        _, st, _ = oracle.trace64(G, source=0, kabs=ka, ksca=ks, g=np.float32(w.dust.g[f]), seed=w.seed,
                                  freq=f, pid_lo=pid_lo, n_packages=max(n // 8, 1))
        steps64 += st["steps"]
    return steps, t_fp32, steps64, time.perf_counter() - t0


_W = None


def _workload_cache(I):
    global _W
    if _W is None:
        _W = I.config_c2()
    return _W


def cpu_baseline(per_freq: int = 300, cores: int | None = None):
    """Oracle steps/s on all 64 frequencies x per_freq packages each, split
    over `cores` spawned processes (package ranges)."""
    import oracle
    oracle.build()
    cores = max(1, min(cores or os.cpu_count() or 1, per_freq))     # at least one package per process
    freqs = list(range(64))
    # package ranges of (nearly) equal length covering all per_freq packages
    base, extra = divmod(per_freq, cores)
    chunks = [(freqs, k * base + min(k, extra), base + (1 if k < extra else 0)) for k in range(cores)]
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(cores) as pool:
        # warm the workers (cloud generation) outside the timed part
        pool.map(_warm, range(cores))
        t0 = time.perf_counter()
        res = pool.map(_oracle_worker, chunks)
    # the FP32 oracle's wall time: the slowest process's loop (each process
    # then times the FP64 oracle on its own)
    wall = max(r[1] for r in res)
    steps = sum(r[0] for r in res)
    # one core's rate: each process timed its own single-threaded loop (all
    # of them running at once)
    per_core = statistics.mean(r[0] / r[1] for r in res if r[1] > 0)
    fp64 = sum(r[2] for r in res) / max(r[3] for r in res)
    return dict(value=steps / wall, unit="photon-cell steps/s", cores=cores, kind="oracle", wall_s=wall,
                per_core_value=per_core, fp64_oracle_value=fp64,
                sample=f"64 frequencies x {per_freq} background packages of the same 128^3 workload "
                       f"({steps} steps, {wall:.1f} s wall on {cores} processes); per_core_value: one "
                       f"process's own rate; fp64_oracle_value: the FP64 oracle on an eighth of the "
                       f"same packages, all processes")


def _warm(_):
    sys.path.insert(0, ROOT)
    from paper_1812_06632_gb300 import inputs as I
    _workload_cache(I)
    import oracle
    oracle.lib()
    oracle.lib64()
    return 0


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    def __init__(self, index: int):
        self.index = index
        self.proc = None
        # raw samples go to the system's temporary directory (or SOC_CLOCKS_DIR)
        d = os.environ.get("SOC_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(d, f"clocks_bench_{os.getpid()}.csv")

    def __enter__(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}",
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if not self.proc:
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 8:
                continue
            try:
                sm.append(float(p[0]))
                mx.append(float(p[1]))
            except ValueError:
                continue
            for n, v in zip(names, p[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_gpu(args):
    global N_PACKAGES, WORKLOAD
    if args.packages != N_PACKAGES:
        N_PACKAGES = args.packages
        WORKLOAD = WORKLOAD.replace("1e6 background", f"{N_PACKAGES:.0e} background")
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)

    cpu_base = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu_base = cpu_baseline(args.cpu_sample)          # before the first GPU call

    from paper_1812_06632_gb300 import build as B
    B.build()
    from paper_1812_06632_gb300 import inputs as I
    from paper_1812_06632_gb300 import soc

    w = I.config_c2(n_packages=N_PACKAGES)
    cl = w.clouds[0]
    nf = len(w.dust.nu)
    ctx = soc.Context(local, w.seed)
    ctx.dust_upload(w.dust.nu, w.dust.kabs, w.dust.ksca, w.dust.g)
    cid = ctx.grid_upload(cl)
    ctx.sources_upload(cid, w.bg_I[0])
    # rank r traces package ids [r N, (r+1) N) of every frequency (weak scaling)
    from paper_1812_06632_gb300 import shard
    specs = shard.shard_items([dict(source=0, freq=f, n_packages=N_PACKAGES, tally_offset=f * cl.n_cells)
                               for f in range(0, nf, args.freq_stride)], rank, world)
    stream = torch.cuda.Stream()
    tally = torch.zeros(nf * cl.n_cells, dtype=torch.int64, device="cuda")
    stats = torch.zeros((len(specs), 4), dtype=torch.int64, device="cuda")
    e_host = ctx.package_energy(cid, 0, N_PACKAGES * world)
    e_unit = torch.from_numpy(e_host).cuda()
    A = torch.zeros(cl.n_cells, dtype=torch.float64, device="cuda")
    T = torch.full((cl.n_cells,), 2.7, dtype=torch.float32, device="cuda")
    dT = torch.zeros(1, dtype=torch.float64, device="cuda")
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    # the tracer pass as one prepared batch in a CUDA graph (counter reset +
    # persistent launch), the FP64 integral and temperature in a second graph
    batch = ctx.batch_create(ctx.items(specs))
    torch.cuda.synchronize()
    ctx.capture_begin(stream)
    ctx.batch_launch(batch, tally, stats, stream=stream)
    g_trace = ctx.capture_end(stream)
    ctx.capture_begin(stream)
    ctx.absorbed_power(cid, tally, cl.n_cells, e_unit, A, stream=stream)
    ctx.update_temperature(cid, A, T, dT, stream=stream)
    g_temp = ctx.capture_end(stream)

    def step(ev=None):
        with torch.cuda.stream(stream):
            if ev:
                ev[0].record(stream)
            ctx.graph_launch(g_trace, stream=stream)
            if ev:
                ev[1].record(stream)
            if world > 1:
                shard.allreduce_counters(tally)
            ctx.graph_launch(g_temp, stream=stream)
            if ev:
                ev[2].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    step_steps = []
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(float(k))                      # L2 flush between steps, outside the events
            step(evs[k])
            with torch.cuda.stream(stream):              # ordered after this pass's tracer
                step_steps.append(stats[:, 2].sum())
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t_step = [evs[k][0].elapsed_time(evs[k][2]) for k in range(args.steps)]      # ms
    t_trace = [evs[k][0].elapsed_time(evs[k][1]) for k in range(args.steps)]
    steps_per_step = float(torch.stack(step_steps).double().mean().item())
    ms = sum(t_step) / args.steps
    ms_trace = sum(t_trace) / args.steps
    if world > 1:
        t = torch.tensor([ms, steps_per_step], dtype=torch.float64, device="cuda")
        mx = t.clone()
        dist.all_reduce(mx, op=dist.ReduceOp.MAX)
        sm = t.clone()
        dist.all_reduce(sm, op=dist.ReduceOp.SUM)
        ms_all, total_steps = mx[0].item(), sm[1].item()
    else:
        ms_all, total_steps = ms, steps_per_step
    value = total_steps / (ms_all / 1e3)

    # end to end through the public API with host buffers: upload the grid and
    # sources from host memory, run iteration 0 (tracer + absorbed power + T),
    # read T back into pinned host memory
    e2e = None
    if world == 1 and args.e2e_steps > 0:
        T_host = torch.empty(cl.n_cells, dtype=torch.float32).pin_memory()
        rho = np.ascontiguousarray(cl.rho, np.float32)
        child = np.ascontiguousarray(cl.child, np.int32)
        h2d = rho.nbytes + child.nbytes + cl.cells_per_level().nbytes + w.bg_I[0].nbytes
        times = []
        for k in range(args.e2e_steps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            c2 = ctx.grid_upload(cl)
            ctx.sources_upload(c2, w.bg_I[0])
            T2 = torch.empty(cl.n_cells, dtype=torch.float32, device="cuda")
            r = ctx.iterate(c2, T2, n_background=N_PACKAGES, max_iter=0, stream=stream)
            with torch.cuda.stream(stream):
                T_host.copy_(T2, non_blocking=True)
            stream.synchronize()
            dt = time.perf_counter() - t0
            ctx.grid_free(c2)
            if k > 0:
                times.append((dt, r["steps"]))
        tot = sum(t for t, _ in times)
        e2e = {"value": sum(s for _, s in times) / tot, "unit": "photon-cell steps/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(T_host.numel() * 4),
               "ms_per_step": 1e3 * tot / len(times)}

    peaks, peak_kind = _peaks()
    bytes_trace = steps_per_step * BYTES_PER_STEP
    achieved = bytes_trace / (ms_trace / 1e3) / 1e9
    traffic = _traffic_per_launch(steps_per_step)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
                "kernel": "trace_kernel", "peak_source": f"{peak_kind} hbm_gbs (copy)",
                "bytes_per_unit": BYTES_PER_STEP, "units_per_launch": steps_per_step,
                "ms_per_launch": ms_trace, "launch_includes": "counter reset (1.07 GB memset) + tracer"}
    # the same algorithmic bytes against this GPU's L2 read bandwidth, and the
    # L2 sector traffic ncu counted for this kernel (32-byte sectors, so a
    # 4-byte cell-word miss or an 8-byte counter update moves a whole sector)
    l2 = l2_bandwidth(ctx)
    lts = TRACE_DRAM["l2_bytes_per_step"] if TRACE_DRAM["source_sha1"] == _trace_source_sha1() else None
    roofline["l2"] = {"achieved": achieved, "peak": l2, "unit": "GB/s", "frac": achieved / l2,
                      "lts_achieved": None if lts is None else lts * steps_per_step / (ms_trace / 1e3) / 1e9,
                      "lts_frac": None if lts is None else lts * steps_per_step / (ms_trace / 1e3) / 1e9 / l2,
                      "peak_source": "bench.l2_bandwidth: soc_probe_read over a 32 MiB L2-resident buffer, 64 passes in one launch, best of 5",
                      "lts_bytes_per_unit": lts}
    out = {
        "metric": "photon-cell steps/s", "value": value, "unit": "photon-cell steps/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_all,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "cells": int(cl.n_cells), "frequencies": nf,
                   "packages_per_frequency": N_PACKAGES * world, "steps_per_pass": total_steps,
                   "l2": "512 MiB buffer written between steps, outside the step events",
                   "parallelism": f"package shards x{world}" if world > 1 else "single GPU"},
        "roofline": roofline, "gpu_launches": 3 * args.steps, "e2e": e2e,
        "trace_source_sha1": _trace_source_sha1(),
        "cpu_baseline": cpu_base,
    }
    if rank == 0:
        out["clocks"] = clk.summary()
        sms = torch.cuda.get_device_properties(local).multi_processor_count
        mhz = (out["clocks"] or {}).get("sm_mhz")
        out["roofline_alu"] = _issue_roofline(steps_per_step, ms_trace, sms, mhz)
        if mhz:
            fp32 = FP32_OPS_PER_STEP * steps_per_step / (ms_trace / 1e3)
            peak32 = FP32_LANES_PER_SM * sms * mhz * 1e6
            out["roofline"]["fp32"] = {"achieved": fp32, "peak": peak32, "unit": "FP32 op/s", "frac": fp32 / peak32,
                                       "ops_per_unit": FP32_OPS_PER_STEP,
                                       "peak_source": f"128 FP32 lanes/SM x {sms} SMs x {mhz:.0f} MHz"}
    ctx.graph_destroy(g_trace)
    ctx.graph_destroy(g_temp)
    ctx.batch_destroy(batch)
    ctx.close()
    del tally, stats, flush
    torch.cuda.empty_cache()
    if rank == 0:
        if world == 1 and not args.no_workloads:
            # the octree pass, the uneven 64-cloud batch and the learned-seeded
            # time to convergence, each timed on its own (CUDA events for the
            # launches, host wall clock for the iterations), with its clocks
            out["workloads"] = {
                "c3_octree": extra_workload("c3", steps=3, warmup=2),
                "c5_batch": extra_workload("c5", steps=3, warmup=2),
                "learned": learned_record(),
            }
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


def extra_workload(workload, steps, warmup, packages=N_PACKAGES, freq_stride=1, autotune=False,
                   convergence=True):
    """Secondary workloads (a record each):
    c3: octree cloud (64^3 root + 3 levels, 4.4e6 cells), background + 3 point
        sources, 64 nu x 1e6 packages each, one graph-replayed launch per
        pass; plus plain and ALI time to converged T (max |dT| < 0.1 K);
    c5: 64 clouds of side 32-128, 32 nu, background + point sources,
        1e5-1e6 packages per cloud, all in one persistent launch.
    Launches timed with CUDA events on the launching stream, clocks sampled
    during the timed launches."""
    import torch
    from paper_1812_06632_gb300 import build as B
    B.build()
    from paper_1812_06632_gb300 import inputs as I
    from paper_1812_06632_gb300 import soc
    t_gen = time.perf_counter()
    if workload == "c3":
        w = I.config_c3()
    else:
        w = I.config_c5()
    if packages != N_PACKAGES:                  # smaller launches for profiling captures
        w.n_bg = [min(n, packages) for n in w.n_bg]
        w.n_ps = [min(n, packages) for n in w.n_ps]
    t_gen = time.perf_counter() - t_gen
    nf = len(w.dust.nu)
    ctx = soc.Context(0, w.seed)
    ctx.dust_upload(w.dust.nu, w.dust.kabs, w.dust.ksca, w.dust.g)
    ids, offs, specs, off = [], [], [], 0
    for ci, cl in enumerate(w.clouds):
        cid = ctx.grid_upload(cl)
        ctx.sources_upload(cid, w.bg_I[ci], w.ps_pos[ci], w.ps_L[ci])
        ids.append(cid)
    for ci, cl in enumerate(w.clouds):
        for src, npk in ((0, w.n_bg[ci]), (1, w.n_ps[ci])):
            for f in range(0, nf, freq_stride):
                specs.append(dict(cloud=ids[ci], source=src, freq=f, n_packages=npk, tally_offset=off))
                off += cl.n_cells
    stream = torch.cuda.Stream()
    tuned = None
    if autotune:
        # the project's autotuner on this very batch (every candidate must
        # give the same counters), then the launch below uses its choice
        from paper_1812_06632_gb300 import autotune as A
        space = dict(threads_per_block=(128, 256), blocks_per_sm=(4,), chunk=(4, 16), refill=(4, 8),
                     scatter=(4, 8))
        best, res = A.tune(ctx, specs, off, w.clouds, space=space, reps=1, use_cache=False)
        tuned = {"best": best, "candidates": len(res), "ms_default": next(
            (m for c, m in res if c == dict(threads_per_block=256, blocks_per_sm=4, chunk=16, refill=8, scatter=8)),
            None), "ms_best": min(m for _, m in res)}
        torch.cuda.empty_cache()
    tally = torch.zeros(off, dtype=torch.int64, device="cuda")
    stats = torch.zeros((len(specs), 4), dtype=torch.int64, device="cuda")
    batch = ctx.batch_create(ctx.items(specs))
    torch.cuda.synchronize()
    ctx.capture_begin(stream)
    ctx.batch_launch(batch, tally, stats, stream=stream)
    g = ctx.capture_end(stream)
    for _ in range(warmup):
        ctx.graph_launch(g, stream=stream)
    stream.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    with Clocks(torch.cuda.current_device()) as clk:
        for k in range(steps):
            ev[k][0].record(stream)
            ctx.graph_launch(g, stream=stream)
            ev[k][1].record(stream)
        stream.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev) / steps
    st = stats.cpu().numpy()
    n_steps = float(st[:, 2].sum())
    assert np.all(st[:, 1] == 0)
    t_ok = int(tally.sum().item()) + int(st[:, 0].sum()) == int(st[:, 3].sum())
    peaks, peak_kind = _peaks()
    gbs = n_steps * BYTES_PER_STEP / (ms / 1e3) / 1e9
    out = {"metric": "photon-cell steps/s", "value": n_steps / (ms / 1e3), "unit": "photon-cell steps/s",
           "workload": workload, "ms_per_launch": ms, "launches_timed": steps, "steps_per_launch": n_steps,
           "items": len(specs), "clouds": len(w.clouds), "cells": int(sum(c.n_cells for c in w.clouds)),
           "frequencies": len(range(0, nf, freq_stride)),
           "packages": int(sum(s["n_packages"] for s in specs)), "energy_conserved": bool(t_ok),
           "roofline": {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                        "frac": gbs / peaks["hbm_gbs"], "bytes_per_unit": BYTES_PER_STEP,
                        "peak_source": f"{peak_kind} hbm_gbs (copy)",
                        "note": "12 B per photon-cell step; the +4 B per octree level moved are not counted"},
           "clocks": clk.summary(), "input_generation_s": t_gen, "autotune": tuned}
    if workload == "c3" and convergence:
        cl = w.clouds[0]
        out["convergence"] = {}
        Ts = {}
        for mode in ("plain", "ali"):
            T = torch.empty(cl.n_cells, dtype=torch.float32, device="cuda")
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = ctx.iterate(ids[0], T, n_background=w.n_bg[0], n_point=w.n_ps[0], n_per_cell=1, max_iter=40,
                            dT_tol=0.1, ali=(mode == "ali"))
            torch.cuda.synchronize()
            Ts[mode] = T
            out["convergence"][mode] = {"wall_s": time.perf_counter() - t0, "dust_iterations": r["iterations"],
                                        "converged": r["converged"],
                                        "max_dT_history_K": [round(x, 4) for x in r["history"]],
                                        "photon_cell_steps": r["steps"], "T_max_K": float(T.max().item())}
        leaf = torch.from_numpy(cl.leaves().astype(np.int64)).cuda()
        out["convergence"]["max_abs_T_difference_K"] = float(
            (Ts["plain"].index_select(0, leaf) - Ts["ali"].index_select(0, leaf)).abs().max().item())
    ctx.graph_destroy(g)
    ctx.batch_destroy(batch)
    ctx.close()
    del tally, stats
    torch.cuda.empty_cache()
    return out


def run_extra(args):
    import torch
    torch.cuda.set_device(0)
    out = extra_workload(args.workload, args.steps, args.warmup, args.packages, args.freq_stride, args.autotune,
                         not args.no_convergence)
    print(json.dumps(out), flush=True)


# the U-Net's convolutions: (C_in, C_out, level) in forward order (level l has side S / 2^l)
UNET_LAYERS = [(16, 16, 0), (16, 16, 0), (16, 32, 1), (32, 32, 1), (32, 64, 2), (64, 64, 2), (64, 128, 3),
               (128, 128, 3), (192, 64, 2), (64, 64, 2), (96, 32, 1), (32, 32, 1), (48, 16, 0), (16, 16, 0),
               (16, 16, 0)]


def learned_record():
    """The second half of the headline metric: wall time to converged T
    (max|dT| < 0.1 K, frozen dust random numbers) of the 20 held-out hot-core
    clouds, learned-seeded against plain, each as one batched run (one
    tracer launch per iteration for every unconverged cloud) after a shared
    iteration 0, with the committed trained weights.  Host wall clock around
    synchronised runs; clocks sampled throughout."""
    import torch
    from paper_1812_06632_gb300 import learned as L
    if not os.path.exists(L.WEIGHTS):
        return {"unavailable": f"no trained weights ({os.path.relpath(L.WEIGHTS, ROOT)}); "
                               "train with python -m paper_1812_06632_gb300.learned"}
    params, norm, meta, digest = L.load_weights()
    with Clocks(torch.cuda.current_device()) as clk:
        c = L.compare(params, norm, L.TEST, log=lambda *a, **k: None)
    n = c["n_clouds"]
    return {"metric": "wall time to converged T (max|dT|<0.1K), learned-seeded", "value": c["learned_s"],
            "unit": f"s for the batch of {n} clouds", "higher_is_better": False, "plain_value": c["plain_s"],
            "learned_over_plain": c["learned_s"] / c["plain_s"],
            "constant_sources_s": c["constant_s"], "plain_dust_s": c["plain_dust_s"],
            "learned_dust_s": c["learned_dust_s"],
            "plain_dust_iterations": c["plain_iterations"], "learned_dust_iterations": c["learned_iterations"],
            "plain_iterations_total": int(sum(c["plain_iterations"])),
            "learned_iterations_total": int(sum(c["learned_iterations"])),
            "plain_steps": c["plain_steps"], "learned_steps": c["learned_steps"],
            "clouds_converged": {"plain": c["plain_converged"], "learned": c["learned_converged"]},
            "unconverged_final_max_dT_K": c["unconverged_final_dT_K"],
            "max_abs_T_difference_K_converged": c["max_abs_T_difference_K"],
            "seed_max_err_K_mean": float(np.mean(c["seed_max_err_K"])),
            "start_max_err_K_mean": float(np.mean(c["start_max_err_K"])), "seed_after": c["seed_after"],
            "weights_sha256": digest, "trained": {k: meta.get(k) for k in ("best_epoch", "epochs_run", "train", "val")},
            "clocks": clk.summary(),
            "config": {"workload": f"{n} held-out hot-core clouds of {c['side']}^3 (seeds {L.TEST[0]}-{L.TEST[-1]}), "
                                   "64 nu, 2e5 background + 2e5 point packages per nu, 1 dust package per cell "
                                   f"per nu, tolerance {c['tol_K']} K"}}


def run_learned(args):
    """--workload learned: the learned-vs-plain record alone (--retrain: first
    regenerate the data and train, writing the weights file)."""
    import torch
    from paper_1812_06632_gb300 import build as B
    B.build()
    torch.cuda.set_device(0)
    if args.retrain:
        from paper_1812_06632_gb300 import learned as L
        L.run(log=lambda *a, **k: None)
    print(json.dumps({"workload": "learned", **learned_record()}), flush=True)


def _map_segments(n, d, e1, e2, center, npx, npy, pix):
    """Leaf segments of every pixel's ray through a regular n^3 grid (root
    units): 1 + the cell planes crossed per axis between entry and exit."""
    px = ((np.arange(npx) + 0.5) - 0.5 * npx) * pix
    py = ((np.arange(npy) + 0.5) - 0.5 * npy) * pix
    X, Y = np.meshgrid(px, py)
    o = center[None, None, :] + X[..., None] * e1[None, None, :] + Y[..., None] * e2[None, None, :]
    t0 = np.full(X.shape, -np.inf); t1 = np.full(X.shape, np.inf)
    for a in range(3):
        if d[a] == 0.0:
            continue
        ta, tb = (0.0 - o[..., a]) / d[a], (n - o[..., a]) / d[a]
        t0 = np.maximum(t0, np.minimum(ta, tb)); t1 = np.minimum(t1, np.maximum(ta, tb))
    hit = t0 < t1
    segs = np.ones(X.shape)
    for a in range(3):
        xa0 = np.clip(o[..., a] + t0 * d[a], 0, n - 1e-9)
        xa1 = np.clip(o[..., a] + t1 * d[a], 0, n - 1e-9)
        segs += np.abs(np.floor(xa1) - np.floor(xa0))
    return float(segs[hit].sum()), int(hit.sum())


def run_map(args):
    """Surface-brightness maps (the mapping kernel): 2048^2 pixels of the
    128^3 bench cloud along an oblique direction at 4 frequencies, timed with
    CUDA events; leaf segments counted from the grid geometry."""
    import torch
    from paper_1812_06632_gb300 import build as B
    B.build()
    from paper_1812_06632_gb300 import inputs as I
    from paper_1812_06632_gb300 import soc
    torch.cuda.set_device(0)
    w = I.config_c2(n_packages=0)
    cl = w.clouds[0]
    n = cl.nx
    ctx = soc.Context(0, w.seed)
    ctx.dust_upload(w.dust.nu, w.dust.kabs, w.dust.ksca, w.dust.g)
    cid = ctx.grid_upload(cl)
    rho = torch.from_numpy(cl.rho).cuda()
    T = (12.0 + 8.0 * torch.log1p(rho)).float()          # a smooth synthetic temperature field
    d = np.array([1.0, 0.7, 0.4]); d /= np.linalg.norm(d)
    up = np.array([0.0, 0.0, 1.0])
    e1 = np.cross(up, d); e1 /= np.linalg.norm(e1)
    e2 = np.cross(d, e1)
    npx = npy = 2048
    pix = 1.8 * n / npx
    center = np.array([n / 2.0] * 3)
    segs, rays = _map_segments(n, d, e1, e2, center, npx, npy, pix)
    out = torch.empty((npy, npx), dtype=torch.float32, device="cuda")
    freqs = (10, 30, 45, 60)
    for f in freqs:
        ctx.map(cid, T, f, d, up, npx, npy, pix, center, out)
    torch.cuda.synchronize()
    ts = []
    for _ in range(max(args.steps, 1)):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for f in freqs:
            ctx.map(cid, T, f, d, up, npx, npy, pix, center, out)
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b) / len(freqs))
    ms = statistics.mean(ts)
    peaks, kind = _peaks()
    gbs = 8 * segs / (ms / 1e3) / 1e9
    out_line = {"metric": "map leaf segments/s", "value": segs / (ms / 1e3), "unit": "segments/s",
                "workload": "map", "ms_per_map": ms, "segments_per_map": segs, "rays_per_map": rays,
                "pixels_per_s": npx * npy / (ms / 1e3),
                "roofline": {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                             "frac": gbs / peaks["hbm_gbs"], "bytes_per_unit": 8,
                             "peak_source": f"{kind} hbm_gbs (copy)"},
                "config": {"workload": f"128^3 lognormal cloud, {npx}x{npy} pixels, direction (1, 0.7, 0.4), "
                                       f"frequencies {list(freqs)}"}}
    ctx.close()
    print(json.dumps(out_line), flush=True)


def run_unet(args):
    """Learned-seed network (batch 4, 64^3): forward and training step
    (forward, input and weight gradients, Adam) timed with CUDA events;
    convolution FLOPs (2 x voxels x 27 x C_in x C_out per layer) against the
    measured BF16 tensor peak."""
    import torch
    from paper_1812_06632_gb300 import build as B
    B.build()
    from paper_1812_06632_gb300 import soc
    torch.cuda.set_device(0)
    batch, side = 4, 64
    fwd_flops = sum(2.0 * batch * (side >> lv) ** 3 * 27 * ci * co for ci, co, lv in UNET_LAYERS)
    # backward: input gradients of every layer but the first, weight gradients of all
    ci0, co0, lv0 = UNET_LAYERS[0]
    train_flops = 3 * fwd_flops - 2.0 * batch * (side >> lv0) ** 3 * 27 * ci0 * co0
    net = soc.UNet(batch, side)
    rng = np.random.default_rng(0)
    net.set_params((rng.standard_normal(net.n_params) * 0.05).astype(np.float32))
    x = torch.randn(batch, side, side, side, 2, device="cuda")
    t = torch.randn(batch, side, side, side, device="cuda")
    pred = torch.empty(batch, side, side, side, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(args.steps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / args.steps

    ms_f = timed(lambda: net.forward(x, pred))
    ms_t = timed(lambda: (net.backward(x, t, pred, loss), net.adam(1e-4)))
    peak = _peaks()[0]
    tf_f = fwd_flops / (ms_f / 1e3) / 1e12
    out = {"metric": "U-Net convolution TFLOP/s", "workload": "unet", "value": tf_f, "unit": "TFLOP/s",
           "config": {"batch": batch, "side": side, "layers": len(UNET_LAYERS), "params": net.n_params},
           "forward_ms": ms_f, "forward_tflop": fwd_flops / 1e12,
           "train_step_ms": ms_t, "train_step_tflop": train_flops / 1e12,
           "train_step_tflops": train_flops / (ms_t / 1e3) / 1e12,
           "roofline": {"bound": "tensor", "achieved": tf_f, "peak": peak["bf16_tflops"], "unit": "TFLOP/s",
                        "frac": tf_f / peak["bf16_tflops"], "traffic": None,
                        "peak_source": "measured bf16_tflops (cuBLAS burst)"},
           "tensor_error_flag": soc.nn_error_flag()}
    net.close()
    print(json.dumps(out), flush=True)


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    per_step = []
    cb = None
    for k in range(args.warmup + args.steps):
        cb = cpu_baseline(args.cpu_sample)
        if k >= args.warmup:
            per_step.append(cb)
    v = statistics.mean(c["value"] for c in per_step)
    steps_per_pass = None
    ms = 1e3 * statistics.mean(c["wall_s"] for c in per_step)       # wall time of one sample
    # the oracle runs on the host cores of rank 0 alone, whatever the launch's world size
    out = {"impl": "reference", "metric": "photon-cell steps/s", "value": v, "unit": "photon-cell steps/s",
           "n_gpus": int(os.environ.get("WORLD_SIZE", args.gpus)), "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic", "config": {"workload": WORKLOAD, "steps_per_pass": steps_per_pass},
           "cpu_baseline": {"kind": "oracle", "cores": cb["cores"], "sample": cb["sample"], "value": v,
                            "unit": "photon-cell steps/s"},
           "e2e": {"value": v, "unit": "photon-cell steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--cpu-sample", type=int, default=32768,
                    help="oracle packages per frequency (about 20 s of CPU work over all host cores)")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="c2", choices=["c2", "c3", "c5", "unet", "learned", "map"],
                    help="c2 (default, the headline 128^3 x 64 nu pass), c3 octree, c5 uneven 64-cloud batch, "
                         "unet (the learned seed's network), learned (time to convergence, learned vs plain)")
    ap.add_argument("--freq-stride", type=int, default=1,
                    help="trace every k-th frequency only (profiling captures of a smaller case)")
    ap.add_argument("--packages", type=int, default=N_PACKAGES,
                    help="packages per frequency (smaller only for profiling captures)")
    ap.add_argument("--no-convergence", action="store_true",
                    help="c3: skip the time-to-convergence runs (profiling captures)")
    ap.add_argument("--autotune", action="store_true",
                    help="c3/c5: run the launch autotuner on the batch first (16 candidates)")
    ap.add_argument("--no-workloads", action="store_true",
                    help="c2: leave out the octree, batch and learned sub-records")
    ap.add_argument("--retrain", action="store_true",
                    help="learned: regenerate the training clouds and train before the comparison")
    args = ap.parse_args()
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        # one process per GPU: relaunch this command under torchrun
        import socket
        with socket.socket() as sk:
            sk.bind(("127.0.0.1", 0))
            port = sk.getsockname()[1]
        cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={args.gpus}",
               "--master-addr=127.0.0.1", f"--master-port={port}", os.path.abspath(__file__), *sys.argv[1:]]
        sys.exit(subprocess.call(cmd))
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "unet":
        run_unet(args)
    elif args.workload == "learned":
        run_learned(args)
    elif args.workload == "map":
        run_map(args)
    elif args.workload != "c2":
        run_extra(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
