"""Per-phase cycle profile of the march (a profiling build of the library).

    python -m paper_2509_16793_gb300.phase_timers [nzeta]
    python -m paper_2509_16793_gb300.phase_timers --streamed [steps]

Builds libgempic with GEMPIC_PHASE_TIMERS into the package's build folder (the product library
is untouched), runs the 3-D LWFA 128 x 128 window (nzeta slices, one march in flight, 2 warm-up
and 2 timed s-steps) and prints, per slice and CTA, the clock64 cycles of each phase of the
march, the mean arrival of each CTA at the first cluster barrier, and how long after the mean
the slowest CTA of a slice arrives.  Thread 0 of each CTA accumulates the cycles in global
memory, so the figures are one thread's view of its CTA.

--streamed: the full 128 x 128 x 1024 window at the default number of s-steps in flight,
`steps` s-steps of the device-resident wavefront (gempic_step) against `steps` s-steps streamed
through pinned host memory (gempic_step_streamed), alternately twice on one simulation: the
per-phase cycles of each call (waits for a predecessor or for the host's release of an input
group land in the phase they interrupt) and its time per s-step.
"""
from __future__ import annotations

import ctypes
import json
import os
import sys

import numpy as np

from . import build, gempic
from . import workloads as W

# timer words of the profiling build and the phase each one covers
PHASES = {0: "rejoining particles, diagnostic flush", 1: "outbox, halo send, barrier B1",
          2: "beam current", 3: "forward row transforms + send", 4: "barrier B2",
          5: "column transforms, forward", 6: "per-mode solve", 7: "column transforms, inverse",
          8: "scatter to row owners", 9: "barrier B3", 10: "inverse row transforms",
          11: "barrier B4", 12: "stored particles", 48: "wait for own CTA",
          49: "push, main loop", 50: "own-row fold", 51: "migration inbox"}


def profile(nzeta: int = 1024, steps: int = 2) -> dict:
    out = os.path.join(build.BUILD, "libgempic_timers.so")
    os.makedirs(build.BUILD, exist_ok=True)
    build.build(defines=["GEMPIC_PHASE_TIMERS"], out=out)
    lib = gempic.load(out)
    lib.gempic_phase_timers.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32]
    w = W.lwfa_3d_128x128x1024()
    if nzeta != w.nzeta:
        las = {**w.laser.__dict__, "zeta_center": nzeta * w.h - 2.0 * w.laser.duration}
        w = w.with_(nzeta=nzeta, laser=W.Laser(**las))
    sim = gempic.Sim(w, pipeline_depth=1)
    C = sim.launch_shape()["cluster_ctas"]
    buf = np.zeros(256 + 2 * nzeta * C, np.uint64)
    sim.step(2)
    lib.gempic_phase_timers(sim.h, buf.ctypes.data, buf.size)     # read and reset
    sim.step(steps)
    lib.gempic_phase_timers(sim.h, buf.ctypes.data, buf.size)
    sim.close()
    norm = steps * nzeta * C
    phases = {name: float(buf[k]) / norm for k, name in PHASES.items()}
    arrival = (buf[64:64 + C].astype(np.float64) / (steps * nzeta)).tolist()
    rel = buf[256:256 + 2 * nzeta * C].reshape(nzeta, C, 2).astype(np.float64)
    late = float((rel[:, :, 0].max(1) - rel[:, :, 0].mean(1)).mean())
    return {"nzeta": nzeta, "cluster_ctas": C, "phases": phases,
            "total": float(sum(phases.values())), "arrival_b1": arrival,
            "slowest_after_mean": late}


def compare_streamed(steps: int = 28) -> dict:
    import time

    import torch

    out = os.path.join(build.BUILD, "libgempic_timers.so")
    os.makedirs(build.BUILD, exist_ok=True)
    build.build(defines=["GEMPIC_PHASE_TIMERS"], out=out)
    lib = gempic.load(out)
    lib.gempic_phase_timers.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32]
    w = W.lwfa_3d_128x128x1024()
    stream = torch.cuda.current_stream()
    sim = gempic.Sim(w, stream=stream.cuda_stream)
    C = sim.launch_shape()["cluster_ctas"]
    buf = np.zeros(256 + 2 * w.nzeta * C, np.uint64)
    sim.step(8)
    host = torch.empty(sim.state_bytes(), dtype=torch.uint8, pin_memory=True).numpy()
    sim.gempic_get_state(host)
    res = {}
    for call in ("device", "streamed", "device 2", "streamed 2"):
        torch.cuda.synchronize()
        lib.gempic_phase_timers(sim.h, buf.ctypes.data, buf.size)     # reset
        t0 = time.perf_counter()
        if call.startswith("device"):
            sim.step(steps)
        else:
            sim.step_streamed(steps, host)
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t0) * 1e3 / steps
        lib.gempic_phase_timers(sim.h, buf.ctypes.data, buf.size)
        norm = steps * w.nzeta * C
        res[call] = {"ms_per_step": ms,
                     "phases": {name: float(buf[k]) / norm for k, name in PHASES.items()}}
    sim.close()
    return {"steps": steps, "cluster_ctas": C, "calls": res}


def main(argv=None) -> int:
    argv = sys.argv[1:] if argv is None else argv
    if argv and argv[0] == "--streamed":
        r = compare_streamed(int(argv[1]) if len(argv) > 1 else 28)
        calls = r["calls"]
        print(f"{'phase':40s}" + "".join(f"{c:>12s}" for c in calls))
        for name in PHASES.values():
            print(f"{name:40s}" + "".join(f"{calls[c]['phases'][name]:12.0f}" for c in calls))
        print(f"{'total':40s}" + "".join(f"{sum(calls[c]['phases'].values()):12.0f}" for c in calls))
        print(f"{'ms per s-step (host clock)':40s}" + "".join(f"{calls[c]['ms_per_step']:12.2f}" for c in calls))
        print(json.dumps(r))
        return 0
    r = profile(int(argv[0]) if argv else 1024)
    for name, v in r["phases"].items():
        print(f"{name:40s} {v:9.0f}")
    print(f"{'total':40s} {r['total']:9.0f}")
    print("arrival at B1 per CTA:", " ".join(f"{a:.0f}" for a in r["arrival_b1"]))
    print(f"slowest CTA of a slice arrives {r['slowest_after_mean']:.0f} cycles after the mean "
          "(first march of the launch)")
    print(json.dumps(r))
    return 0


if __name__ == "__main__":
    sys.exit(main())
