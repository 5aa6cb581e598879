"""Training and evaluating the learned current denoiser on pairs of runs of this method.

Pairs: the same workload at few (1) and many (16) particles per cell, each s-step's plain
current kept on the device (GEMPIC_FLAG_CURRENT); the sparse run's current is the input and
the dense run's the target.  Training: Adam on slabs of consecutive half-slices (full
transverse planes) drawn at random from the pairs.  Evaluation: fresh runs, the sparse one with
denoised s-steps, against the dense plain run (on-axis E_z, field energy), the plain deposit
of the sparse run beside it.  Everything runs in the library's kernels; this module only
drives them (argument marshalling, choice of slabs, timing with CUDA events).
"""
from __future__ import annotations

import time
from typing import Dict, List, Tuple

import numpy as np

from . import gempic


def generate_pairs(w_sparse, w_dense, steps: int, stream=None) -> Tuple[list, list, dict]:
    """Run both workloads for `steps` s-steps, one s-step per call, keeping every s-step's plain
    current (device tensors [nz, 3, ny, nx], FP32).  Returns (inputs, targets, timing)."""
    import torch
    xs, ts = [], []
    timing = {}
    for w, out in ((w_sparse, xs), (w_dense, ts)):
        w = w.with_(capture_current=True)
        with gempic.Sim(w, stream=stream, pipeline_depth=1) as sim:
            t0 = time.perf_counter()
            for _ in range(steps):
                sim.step(1)
                out.append(sim.current(torch.empty((w.nzeta, 3, w.ny, w.nx), dtype=torch.float32,
                                                   device="cuda")))
            torch.cuda.synchronize()
            timing[w.name] = (time.perf_counter() - t0) / steps
    return xs, ts, timing


def train(den: "gempic.Denoiser", xs: list, ts: list, iters: int, slab: int = 32,
          lr: float = 1e-3, seed: int = 0, z_margin: int = 3, average_tail: float = 0.2,
          average_every: int = 10) -> List[float]:
    """Adam steps on random slabs of `slab` consecutive half-slices of random pairs; the rate
    drops tenfold for the last fifth.  average_tail > 0: the parameters are averaged over that
    last fraction of the steps (every `average_every` steps; stochastic weight averaging) and
    the average is what the denoiser keeps."""
    rng = np.random.default_rng(seed)
    nz = xs[0].shape[0]
    losses = []
    first_avg = int(iters * (1.0 - average_tail)) if average_tail > 0 else iters
    acc, nacc = None, 0
    for it in range(iters):
        k = int(rng.integers(len(xs)))
        z0 = int(rng.integers(0, nz - slab + 1))
        x = xs[k][z0:z0 + slab].contiguous()
        t = ts[k][z0:z0 + slab].contiguous()
        rate = lr * (0.1 if it > 0.8 * iters else 1.0)
        losses.append(den.train_step(x, t, rate, z_margin=z_margin))
        if it >= first_avg and (iters - 1 - it) % average_every == 0:
            p = den.params().astype(np.float64)
            acc = p if acc is None else acc + p
            nacc += 1
    if nacc:
        den.set_params((acc / nacc).astype(np.float32))
    return losses


def rel_err(a, b, sel=None) -> float:
    """max |a - b| / max |b| (over sel)."""
    a, b = np.asarray(a), np.asarray(b)
    if sel is not None:
        a, b = a[sel], b[sel]
    return float(np.abs(a - b).max() / np.abs(b).max())


def rms_err(a, b, sel=None) -> float:
    """||a - b||_2 / ||b||_2 (over sel)."""
    a, b = np.asarray(a), np.asarray(b)
    if sel is not None:
        a, b = a[sel], b[sel]
    return float(np.sqrt(((a - b) ** 2).sum() / (b ** 2).sum()))


def _timed_steps(sim, n: int) -> float:
    """Device time per s-step of one call of n s-steps (CUDA events on the stream)."""
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    st = torch.cuda.current_stream()
    torch.cuda.synchronize()
    e0.record(st)
    sim.step(n)
    e1.record(st)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / n


def evaluate(w_sparse, w_dense, den: "gempic.Denoiser", steps: int, stream=None,
          chain_depths=(2, 3, 4, 5, 6, 7)) -> Dict:
    """Fresh runs of `steps` s-steps: dense plain, sparse plain, sparse denoised.  On-axis E_z
    and field energy of the sparse runs against the dense run after the last s-step, over the
    window and in front of the region where the dense run traps particles (its front-most
    stored particle plus 64 slices).  Time per s-step: CUDA events on the stream around one call
    of the first steps - 1 s-steps (7 = one full wave of the dense run's 7-deep wavefront); the
    plain runs march as their wavefront, the denoised run as its chain of first and second
    passes with the net between them, at the library's default depth and, on extra runs, at each
    depth of `chain_depths` (the marches in flight: more take SMs from the net)."""
    res = {}
    out = {}
    # a second dense run with other particles: the dense run's own noise, the floor of any
    # comparison against it
    runs = (("dense", w_dense, None), ("dense_other_seed", w_dense.with_(seed=w_dense.seed + 7), None),
            ("sparse", w_sparse, None), ("sparse_denoised", w_sparse, den))
    pipeline = None
    for label, w, d in runs:
        with gempic.Sim(w, stream=stream) as sim:
            if d is not None:
                sim.set_denoiser(d)
            sim.step(0)                          # the level-0 set-up, not timed
            ms = _timed_steps(sim, steps - 1)
            sim.step(1)
            out[label] = {"ms_per_step": ms, "ez": sim.onaxis_ez(), "diag": sim.diagnostics()}
            if label == "dense":
                p = sim.particles(0)
                out[label]["zeta_trap"] = float(p["zeta"].max()) if p["zeta"].size else 0.0
                pipeline = sim.launch_shape()["pipeline"]
    depth_ms = {}
    for depth in chain_depths:
        with gempic.Sim(w_sparse, stream=stream, pipeline_depth=depth) as sim:
            sim.set_denoiser(den)
            sim.step(0)
            depth_ms[str(depth)] = _timed_steps(sim, steps - 1)
    dense_wave_ms = out["dense"]["ms_per_step"]
    ref = out["dense"]["ez"]
    zc = np.arange(w_dense.nzeta) * w_dense.h
    front = zc > out["dense"]["zeta_trap"] + 64 * w_dense.h
    fe = out["dense"]["diag"]["field_energy"]
    for label in ("dense_other_seed", "sparse", "sparse_denoised"):
        res[label] = {"ez_rel_err": rel_err(out[label]["ez"], ref),
                      "ez_rel_err_front": rel_err(out[label]["ez"], ref, front),
                      "ez_rms_err": rms_err(out[label]["ez"], ref),
                      "ez_rms_err_front": rms_err(out[label]["ez"], ref, front),
                      "field_energy_rel_err": abs(out[label]["diag"]["field_energy"] - fe) / fe,
                      "ms_per_step": out[label]["ms_per_step"]}
    res["dense"] = {"ms_per_step_wavefront": dense_wave_ms, "wavefront_depth": pipeline,
                    "front_slices": int(front.sum())}
    res["sparse_denoised"]["ms_per_step_by_chain_depth"] = depth_ms
    res["speedup_vs_dense_wavefront"] = dense_wave_ms / out["sparse_denoised"]["ms_per_step"]
    best = min(depth_ms.values()) if depth_ms else out["sparse_denoised"]["ms_per_step"]
    res["speedup_vs_dense_wavefront_best_depth"] = dense_wave_ms / best
    return res


def time_apply(den: "gempic.Denoiser", w, stream=None, reps: int = 5) -> float:
    """Device time of one application of the denoiser to a current of w's grid (ms)."""
    import torch
    j = torch.randn((w.nzeta, 3, w.ny, w.nx), dtype=torch.float32, device="cuda") * den.scale
    out = torch.empty_like(j)
    den.apply(j, out, stream)
    st = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(st)
    for _ in range(reps):
        den.apply(j, out, stream)
    e1.record(st)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def experiment(pairs: int = 96, iters: int = 10000, eval_steps: int = 8, stream=None,
               average_tail: float = 0.2) -> Dict:
    """The whole experiment on the 128 x 128 x 512 LWFA: pairs of 1- and 16-ppc runs, training,
    evaluation.  Returns a summary dict."""
    from . import workloads as W
    ws, wd = W.lwfa_3d_128x128x512(ppc=1), W.lwfa_3d_128x128x512(ppc=16)
    scale = abs(ws.species[0].charge * ws.species[0].density)
    t0 = time.perf_counter()
    xs, ts, gen = generate_pairs(ws, wd, pairs, stream)
    t1 = time.perf_counter()
    with gempic.Denoiser(None, scale) as den:
        # a small random start for the hidden layers, zero last layer (starts as the identity)
        rng = np.random.default_rng(1)
        p = np.zeros(den.n, np.float32)
        n1 = 27 * 3 * 16
        p[:n1] = rng.standard_normal(n1) * np.sqrt(2.0 / 81)
        o2 = n1 + 16
        n2 = 27 * 16 * 16
        p[o2:o2 + n2] = rng.standard_normal(n2) * np.sqrt(2.0 / 432)
        den.set_params(p)
        losses = train(den, xs, ts, iters, average_tail=average_tail)
        t2 = time.perf_counter()
        del xs, ts
        res = evaluate(ws, wd, den, eval_steps, stream)
        res["apply_ms"] = time_apply(den, ws, stream)
    res["training"] = {"pairs": pairs, "iters": iters, "average_tail": average_tail,
                       "loss_first": float(np.mean(losses[:20])),
                       "loss_last": float(np.mean(losses[-20:])), "generate_s": t1 - t0,
                       "train_s": t2 - t1, "s_per_step_generate": gen}
    res["workload"] = {"sparse": ws.name, "dense": wd.name}
    return res


if __name__ == "__main__":
    # python -m paper_2509_16793_gb300.denoise_train [--apply NZ]: the whole experiment (one
    # JSON document), or only NZ-slice denoiser applications on the 128 x 128 grid (profiling)
    import argparse
    import json
    import torch
    from . import build, workloads as W
    ap = argparse.ArgumentParser()
    ap.add_argument("--apply", type=int, default=0)
    ap.add_argument("--pairs", type=int, default=96)
    ap.add_argument("--iters", type=int, default=10000)
    ap.add_argument("--average-tail", type=float, default=0.2,
                    help="fraction of the last steps whose parameters are averaged (0: none)")
    a = ap.parse_args()
    build.build()
    if a.apply:
        w = W.lwfa_3d_128x128x512(ppc=1).with_(nzeta=a.apply)
        with gempic.Denoiser(None, 0.002) as den:
            rng = np.random.default_rng(1)
            den.set_params(rng.standard_normal(den.n).astype(np.float32) * 0.05)
            print(json.dumps({"apply_ms": time_apply(den, w, reps=3), "nzeta": a.apply}))
    else:
        print(json.dumps(experiment(a.pairs, a.iters, average_tail=a.average_tail), indent=1))
