"""Benchmark of the GEM-PIC hot path on GB300 (one JSON line on stdout).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Workload: 3-D LWFA 128 x 128 x 1024, 2 ppc, FP32 push/deposit on cell-relative positions,
a0 = 2.5 (the configuration the particle-pushes/s metric is quoted on).  A step is one
s-step of the whole hot path: front injection, gather + push + deposit of every streaming
particle across every slice, the per-slice transverse FFTs and slice solve, the stored
(trapped) particle s-push, back removal and the FP64 diagnostics.  Multi-GPU runs are
independent replicas (the method does not shard without a per-slice exchange).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# Algorithmic work per unit, counted from the kernels:
FLOP_PER_PUSH = 330.0            # gather 52 + two-pass Boris 156 + advance 22 + Esirkepov/CIC 100
FLOP_PER_MODE = 150.0            # corrector + App. B closed form + fields, complex arithmetic
BYTES_PER_CELL = {32: 48.0, 64: 96.0}   # spectral state read + written once per s-step


def fft_flops(n: int) -> float:
    return 5.0 * n * math.log2(n) if n > 1 else 0.0


def algorithmic_flops(w) -> float:
    """FLOP per s-step: pushes, transverse FFTs (3 forward + 6 inverse real 2-D transforms,
    done as paired complex row transforms and complex column transforms) and the solve."""
    nxh = w.nx // 2
    per_slice_fft = (2 * w.ny + 3 * w.ny) * fft_flops(w.nx) + (3 + 6) * nxh * fft_flops(w.ny)
    return (w.pushes_per_step * FLOP_PER_PUSH
            + w.nzeta * (per_slice_fft + nxh * w.ny * FLOP_PER_MODE))


def algorithmic_bytes(w) -> float:
    return w.nx * w.ny * w.nzeta * BYTES_PER_CELL[w.precision]


def fp32_peak_tflops(sm_mhz: float) -> float:
    """Plain FP32 ALU peak: 152 SMs x 128 FP32 lanes x 2 FLOP (FMA) x clock."""
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0, "fallback": True}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while the timed region runs."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx = max(mx, float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def replica_workload(w, rank: int):
    """Replicas: rank r simulates its own plasma (seed offset r) on its own GPU; there is no
    data-path collective, so per-rank work is fixed as ranks are added (weak scaling)."""
    return w.with_(seed=w.seed + rank)


def max_over_ranks(x: float, device) -> float:
    """The slowest rank sets the job's time: max of a per-rank float over the process group
    (identity without one)."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return world * units_per_rank / seconds


def oracle_window(w):
    """The bounded sample of the workload the oracle is timed on: the same transverse grid and
    particles per cell over a 64-slice window (the laser centred in it; a bunch's head in it,
    with 2^14 macroparticles); pushes/s per slice."""
    s = w.with_(nzeta=64, precision=64)
    if w.laser is not None:
        s = s.with_(laser=w.laser.__class__(**{**w.laser.__dict__, "zeta_center": 32 * w.h}))
    if w.beam is not None:
        s = s.with_(beam=w.beam.__class__(**{**w.beam.__dict__, "zeta_center": 64 * w.h - 0.8,
                                            "n_macro": 1 << 14}))
    return s


def _oracle_worker(job):
    """One oracle process: s-steps of the window until `seconds` or `max_steps`; returns the
    wall-clock start and end of the timed loop and the pushes done."""
    sample, seconds, max_steps = job
    from oracle import RefSim
    sim = RefSim(sample)
    t0 = time.time()
    steps = 0
    while steps < max_steps:
        sim.step()
        steps += 1
        if time.time() - t0 > seconds:
            break
    return t0, time.time(), sample.pushes_per_step * steps, steps


def oracle_sample(w, seconds: float, max_steps: int, procs: int = 0):
    """Time the FP64 oracle, as it stands, on the host cores: `procs` independent processes
    (0 = one per core; spawned, so safe after CUDA is initialised) each march their own seeded
    copy of the window; the rate is all pushes over the wall time from the first start to the
    last end.  procs = 1 runs in this process (single thread)."""
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ.setdefault(v, "1")
    sample = oracle_window(w)
    n = procs if procs > 0 else (os.cpu_count() or 1)
    if n == 1:
        res = [_oracle_worker((sample, seconds, max_steps))]
    else:
        import multiprocessing as mp
        jobs = [(sample.with_(seed=sample.seed + i), seconds, max_steps) for i in range(n)]
        with mp.get_context("spawn").Pool(n) as pool:
            res = pool.map(_oracle_worker, jobs)
    t0 = min(r[0] for r in res)
    t1 = max(r[1] for r in res)
    pushes = sum(r[2] for r in res)
    steps = sum(r[3] for r in res)
    dt = t1 - t0
    return {"value": pushes / dt, "unit": "pushes/s", "cores": n, "kind": "oracle",
            "sample": f"{steps} s-step(s) in {n} process(es) of a {sample.nx}x{sample.ny}x"
                      f"{sample.nzeta} window of the workload ({sample.pushes_per_step} "
                      f"pushes/step), FP64 numpy, one thread per process, {dt:.1f} s wall",
            "ms_per_step": dt / max(1, steps // n) * 1e3}


def run_reference(args, w):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from oracle import RefSim  # noqa: F401
    # warm-up steps and timed steps on the bounded sample, one process per host core
    base = oracle_sample(w, seconds=1e9, max_steps=max(1, args.warmup), procs=1)
    cb = oracle_sample(w, seconds=1e9, max_steps=max(1, args.steps))
    line = {"impl": "reference", "metric": "particle-pushes/s", "value": cb["value"],
            "unit": "pushes/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": cb["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(w),
            "cpu_baseline": {"value": cb["value"], "unit": "pushes/s", "cores": cb["cores"],
                             "kind": "oracle", "sample": cb["sample"]},
            "e2e": {"value": cb["value"], "unit": "pushes/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    del base
    print(json.dumps(line), flush=True)
    return 0


def config_dict(w, shape=None):
    d = {"workload": w.name, "grid": [w.nx, w.ny, w.nzeta], "h": w.h, "hx": w.hx,
         "delta": w.delta, "ppc": sum(s.ppc for s in w.species), "precision": w.precision,
         "laser_a0": w.laser.a0 if w.laser else None,
         "pushes_per_step": w.pushes_per_step,
         "l2": f"spectral state (24 B/cell, {w.nx * w.ny * w.nzeta * 24 / 1e6:.0f} MB) read and "
               "rewritten every s-step: inputs larger than L2"}
    if shape:
        d["launch"] = shape
    return d


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    # 49 = 7 x 7: every cluster of the 7-deep wavefront marches the same number of s-steps
    ap.add_argument("--steps", type=int, default=49)
    ap.add_argument("--warmup", type=int, default=8)
    ap.add_argument("--impl", default="gempic", choices=["gempic", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=49, help="0 skips the end-to-end leg")
    ap.add_argument("--nzeta", type=int, default=0,
                    help="profiling only: shorter window of the same workload")
    ap.add_argument("--pipeline", type=int, default=0, help="s-steps marched concurrently (0 = auto)")
    ap.add_argument("--bucket-capacity", type=int, default=0)
    ap.add_argument("--workload", default="lwfa3d", choices=["lwfa3d", "scan", "pwfa"],
                    help="lwfa3d: the 3-D LWFA (default); scan: the batched 2-D parameter scan; "
                         "pwfa: the beam-driven 3-D case (128 x 128 x 768, 2 e + 2 p per cell, "
                         "a 2^20-particle drive bunch)")
    ap.add_argument("--instances", type=int, default=64, help="scan: number of instances")
    ap.add_argument("--fp64-steps", type=int, default=40,
                    help="s-steps of the FP64-plain comparison on the 2-D workload (0 skips it)")
    ap.add_argument("--denoise-pairs", type=int, default=96,
                    help="denoiser leg: paired s-steps of the 1- and 16-ppc runs (0 skips it)")
    ap.add_argument("--denoise-iters", type=int, default=10000, help="denoiser leg: Adam steps")
    args = ap.parse_args()
    if args.workload == "scan" and args.impl == "gempic":
        return run_scan(args)

    from paper_2509_16793_gb300 import workloads as W
    w = W.pwfa_3d_128x128x768() if args.workload == "pwfa" else W.lwfa_3d_128x128x1024()
    if args.workload == "pwfa":
        args.e2e_steps = 0
        args.fp64_steps = 0
        args.denoise_pairs = 0
    if args.nzeta:
        w = w.with_(nzeta=args.nzeta, name=f"{w.name}_nzeta{args.nzeta}",
                    laser=W.Laser(**{**w.laser.__dict__,
                                     "zeta_center": args.nzeta * w.h - 2.0 * w.laser.duration}))
    if args.impl == "reference":
        return run_reference(args, w)

    import numpy as np
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2509_16793_gb300 import build, gempic
    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        torch.distributed.barrier()
    stream = torch.cuda.current_stream()
    # replicas: each rank simulates its own plasma (seed offset), no data-path collective
    wr = replica_workload(w, rank)
    # the measured FP32 denominator of the ALU roofline: an FMA probe (its own clocks sampled)
    with ClockSampler(local) as pclk:
        probe_tf, probe_ms = gempic.gempic_probe_fp32_fma(400000, stream.cuda_stream)
    sim = gempic.Sim(wr, stream=stream.cuda_stream, pipeline_depth=args.pipeline,
                     bucket_capacity=args.bucket_capacity)
    shape = sim.launch_shape()
    sim.step(args.warmup)
    launches0 = sim.launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        sim.step_async(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
    sim.sync()
    launches = sim.launch_count() - launches0
    ms = max_over_ranks(e0.elapsed_time(e1), "cuda")
    ms_step = ms / args.steps
    value = job_rate(w.pushes_per_step * args.steps, world, ms / 1e3)
    diag = sim.diagnostics()

    # end to end through the C-ABI with host buffers: every s-step's input state comes in from
    # pinned host memory and its result and diagnostics go back out, streamed by groups of
    # slices while the marches run (gempic_step_streamed)
    nb = sim.state_bytes()
    diag_bytes = 9 * shape["cluster_ctas"] * 8          # per-CTA FP64 partials of one s-step
    e2e_s = float("nan")
    e2e_error = None
    if args.e2e_steps > 0:
        host = torch.empty(nb, dtype=torch.uint8, pin_memory=True).numpy()
        sim.gempic_get_state(host)                          # the raw bytes of the state
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        try:
            sim.step_streamed(args.e2e_steps, host)
            e2e_s = (time.perf_counter() - t0) / args.e2e_steps
        except gempic.GempicError as ex:
            # the streamed call needs its copies to run beside the marches (a profiler that
            # serialises the device makes its bounded waits give up)
            e2e_error = str(ex)
    e2e_s = max_over_ranks(e2e_s, "cuda")
    e2e_value = job_rate(w.pushes_per_step, world, e2e_s)

    if rank != 0:
        sim.close()
        if world > 1:
            torch.distributed.barrier()
            torch.distributed.destroy_process_group()
        return 0

    clocks = clk.summary()
    peaks = measured_peaks()
    sm_mhz = clocks.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    peak_alu = probe_tf
    flops = algorithmic_flops(w) * args.steps
    achieved = flops / (ms / 1e3) / 1e12
    hbm = algorithmic_bytes(w) * args.steps / (ms / 1e3) / 1e9
    traffic = measured_traffic(w) * args.steps if measured_traffic(w) else None
    roof = {"bound": "alu", "achieved": achieved, "peak": peak_alu, "unit": "TFLOP/s",
            "frac": achieved / peak_alu, "traffic": traffic,
            "traffic_source": ("profiles/march_kernel_lwfa3d_128x128x1024.md (ncu DRAM bytes per "
                               "s-step, used while its kernel hash matches the source)"
                               if traffic else None),
            "peak_source": f"measured: FP32 FMA probe (gempic_probe_fp32_fma, {probe_ms:.0f} ms, "
                           f"SM clock median {pclk.summary().get('sm_mhz')} MHz); spec figure "
                           f"152 SM x 128 lanes x 2 x {peaks.get('sm_max_mhz', 2070.0):.0f} MHz = "
                           f"{fp32_peak_tflops(peaks.get('sm_max_mhz', 2070.0)):.1f}",
            "kernel": "march_kernel<float>",
            "launches": launches, "launch_ms_avg": ms / max(1, launches),
            "hbm": {"achieved": hbm, "peak": peaks.get("hbm_gbs"), "unit": "GB/s",
                    "frac": hbm / peaks.get("hbm_gbs", 6800.0), "of": "measured"}}
    # the metric's FP32-vs-FP64-plain comparison: the 2-D FP64 workload (128 x 256, 4 ppc, Delta
    # at the stability limit) in FP64 and, on the same grid, in FP32
    fp64 = None
    if args.fp64_steps > 0:
        from paper_2509_16793_gb300 import workloads as W
        w2 = W.lwfa_2d_128x256(precision=64)
        v64, ms64 = time_plain(w2, args.fp64_steps, 3, stream)
        v32, ms32 = time_plain(w2.with_(precision=32), args.fp64_steps, 3, stream)
        fp64 = {"workload": w2.name, "steps": args.fp64_steps,
                "fp64": {"value": v64, "ms_per_step": ms64},
                "fp32": {"value": v32, "ms_per_step": ms32},
                "unit": "pushes/s", "fp32_over_fp64": v32 / v64}
    # the metric's "denoised" form: the learned current denoiser trained on 1- vs 16-ppc runs
    # of the 128 x 128 x 512 LWFA, compared with the 16-ppc plain run
    denoise = None
    if args.denoise_pairs > 0:
        try:
            from paper_2509_16793_gb300 import denoise_train
            denoise = denoise_train.experiment(args.denoise_pairs, args.denoise_iters,
                                               stream=stream.cuda_stream)
        except Exception as ex:  # reported, never the headline
            denoise = {"error": str(ex)}
    cpu = None
    if not args.no_cpu_baseline:
        try:
            cpu = oracle_sample(w, seconds=15.0, max_steps=20)
            cpu.pop("ms_per_step", None)
            one = oracle_sample(w, seconds=10.0, max_steps=20, procs=1)
            cpu["single_core"] = {"value": one["value"], "sample": one["sample"]}
        except Exception as ex:  # the baseline is reported, never the target
            cpu = {"error": str(ex)}
    line = {"metric": "particle-pushes/s", "value": value, "unit": "pushes/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": config_dict(w, shape), "roofline": roof, "cpu_baseline": cpu,
            "e2e": {"value": e2e_value if math.isfinite(e2e_value) else None,
                    "unit": "pushes/s", "h2d_bytes_per_step": nb,
                    "d2h_bytes_per_step": nb + diag_bytes,
                    "steps": args.e2e_steps, "call": "gempic_step_streamed",
                    **({"error": e2e_error} if e2e_error else {})},
            "gpu_launches": launches, "clocks": clocks, "fp64_plain": fp64, "denoiser": denoise,
            "diag": {k: diag[k] for k in ("field_energy", "kinetic_energy", "n_stored", "pushes")}}
    print(json.dumps(line), flush=True)
    sim.close()
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    return 0


def time_plain(w, steps: int, warmup: int, stream):
    """Device time of `steps` s-steps of workload w in one call (CUDA events on the stream the
    library launches on): (pushes/s, ms per step)."""
    import torch
    from paper_2509_16793_gb300 import gempic
    with gempic.Sim(w, stream=stream.cuda_stream) as sim:
        sim.step(warmup)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        sim.step_async(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        sim.sync()
        ms = e0.elapsed_time(e1)
    return w.pushes_per_step * steps / (ms / 1e3), ms / steps


def measured_traffic(w):
    """DRAM bytes per s-step of the march kernel from the committed ncu summary, if it was
    taken on this kernel source and this workload's grid (else None)."""
    import re
    f = os.path.join(ROOT, "profiles", "march_kernel_lwfa3d_128x128x1024.md")
    if not os.path.exists(f) or (w.nx, w.ny, w.nzeta) != (128, 128, 1024) or w.precision != 32:
        return None
    m = re.search(r"traffic_bytes_per_step: (\d+) kernel_hash: (\w+)", open(f).read())
    if not m or m.group(2) != kernel_hash():
        return None
    return int(m.group(1))


def run_scan(args):
    """Batched parameter scan: independent 2-D instances of uneven size stepped side by side,
    one persistent launch per instance per call, each on its own stream.  Timed with CUDA
    events recorded on every instance's stream: latest end minus earliest start."""
    import torch
    from paper_2509_16793_gb300 import build, gempic, workloads as W

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()
    ws = W.scan_2d(n=args.instances, seed=W.SEED + 1000 * rank)
    pushes = sum(w.pushes_per_step for w in ws)
    with gempic.Batch(ws) as b:
        b.step(args.warmup)
        launches0 = sum(v.launch_count() for v in b.sims)
        streams = [torch.cuda.ExternalStream(b.stream(i)) for i in range(len(ws))]
        ref = torch.cuda.Event(enable_timing=True)
        starts = [torch.cuda.Event(enable_timing=True) for _ in ws]
        ends = [torch.cuda.Event(enable_timing=True) for _ in ws]
        torch.cuda.synchronize()
        ref.record(streams[0])
        with ClockSampler(local) as clk:
            for e, st in zip(starts, streams):
                e.record(st)
            b.step_async(args.steps)
            for e, st in zip(ends, streams):
                e.record(st)
            b.sync()
            torch.cuda.synchronize()
        t0 = min(ref.elapsed_time(e) for e in starts)
        t1 = max(ref.elapsed_time(e) for e in ends)
        ms = t1 - t0
        tuned = [b.tuning(i) for i in range(len(ws))]
        # every instance counts the batch's persistent launch once: one launch per call
        launches = (sum(v.launch_count() for v in b.sims) - launches0) // len(ws)
    ms = max_over_ranks(ms, "cuda")
    value = job_rate(pushes * args.steps, world, ms / 1e3)
    if rank == 0:
        peaks = measured_peaks()
        peak_alu, _ = gempic.gempic_probe_fp32_fma(400000)
        flops = sum(algorithmic_flops(w) for w in ws) * args.steps
        achieved = flops / (ms / 1e3) / 1e12
        sizes = sorted({(w.nx, w.nzeta) for w in ws})
        line = {"metric": "particle-pushes/s", "value": value, "unit": "pushes/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": f"scan_2d_{len(ws)}", "instances": len(ws),
                           "sizes_nx_nzeta": sizes, "ppc": 4, "pushes_per_step": pushes,
                           "launch": "one persistent launch per call (work queue of "
                                     "(instance, s-step) items, CUDA graph), "
                                     f"{tuned[0][0]} threads per CTA (autotuned)",
                           "class_ms_per_step": {"min": min(t[1] for t in tuned),
                                                 "max": max(t[1] for t in tuned),
                                                 "sum": sum(t[1] for t in tuned)},
                           "l2": "every instance's state and particles are resident; no L2 flush"},
                "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_alu,
                             "unit": "TFLOP/s", "frac": achieved / peak_alu, "traffic": None,
                             "peak_source": "measured: FP32 FMA probe",
                             "kernel": "batch_kernel<float> (persistent, all instances)"},
                "cpu_baseline": None, "e2e": None, "gpu_launches": launches,
                "clocks": clk.summary()}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    return 0


def kernel_hash() -> str:
    import hashlib
    h = hashlib.sha1()
    for f in ("gempic_kernels.cu", "gempic_internal.h"):
        h.update(open(os.path.join(ROOT, "paper_2509_16793_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:12]


if __name__ == "__main__":
    sys.exit(main())
