"""Writes the oracle fixtures of tests/golden/ (run from the repository root:
python tests/golden/make_golden.py [tiny] [bench]).  Calls only oracle/ and the input recipes.
The tiny fixtures guard the oracle against unintended changes (test_golden.py); the bench
fixture holds the oracle's FP64 result on the full-size bench workload, which the GPU path
is compared with (the oracle needs minutes and gigabytes for it, too much for a test)."""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import RefSim                                   # noqa: E402
from paper_2509_16793_gb300 import workloads as W          # noqa: E402

CASES = {
    "oracle_tiny_2d": dict(kind="2d", nx=8, nzeta=48, ppc=1, a0=2.0, delta=1.5, steps=3),
    "oracle_tiny_3d": dict(kind="3d", nx=8, ny=8, nzeta=12, ppc=1, a0=1.5, steps=2),
}


def workload(c):
    if c["kind"] == "2d":
        return W.small_2d(nx=c["nx"], nzeta=c["nzeta"], ppc=c["ppc"], a0=c["a0"],
                          delta=c["delta"], precision=64)
    return W.small_3d(nx=c["nx"], ny=c["ny"], nzeta=c["nzeta"], ppc=c["ppc"], a0=c["a0"],
                      precision=64)


def run(c):
    o = RefSim(workload(c))
    out = []
    for _ in range(c["steps"]):
        d = o.step()
        out.append({k: (float(d[k]) if "energy" in k or k == "charge_flux" else int(d[k]))
                    for k in ("field_energy", "kinetic_energy", "charge_flux", "n_trapped",
                              "n_stored", "n_rejoined")})
        out[-1]["onaxis_ez"] = [float(v) for v in d["onaxis_ez"]]
    st = o.state()
    norms = {name: float(abs(st[i]).sum()) for i, name in
             enumerate(("Rx", "Ry", "Ez", "Bz", "jx", "jy"))}
    return {"case": c, "steps": out, "state_l1": norms}


# The bench workload (3-D LWFA 128 x 128 x 1024, 2 ppc, a0 = 2.5) after two s-steps, in FP64:
# the diagnostics of both s-steps, the on-axis E_z and a sample of the spectral state (every
# 64th slice and the last one; the 8 x 16 lowest transverse modes: kx index 0..7, ky index
# 0..7 and ny-8..ny-1).  Too large for the oracle inside a test: written here once.
BENCH_FIXTURE = "oracle_lwfa3d_128x128x1024_2steps.npz"
BENCH_SLICES = list(range(0, 1024, 64)) + [1023]


def bench_sample_index(ny):
    ky = list(range(8)) + list(range(ny - 8, ny))
    return np.array(BENCH_SLICES), np.array(ky), np.arange(8)


def bench_fixture(path):
    w = W.lwfa_3d_128x128x1024(precision=64)
    o = RefSim(w)
    rec = {}
    for k in range(2):
        d = o.step()
        for key in ("field_energy", "kinetic_energy", "stored_kinetic_energy", "charge_flux",
                    "n_trapped", "n_stored", "n_rejoined"):
            rec[f"{key}_{k}"] = np.array(d[key])
        rec[f"onaxis_ez_{k}"] = np.asarray(d["onaxis_ez"], dtype=np.float64)
        # the front-most stored (trapped) particle: behind it the wake breaks
        rec[f"stored_zeta_max_{k}"] = np.array(o.stored.zeta.max() if o.stored.n else 0.0)
    sl, ky, kx = bench_sample_index(w.ny)
    st = o.state()
    rec["state_sample"] = st[:, sl][:, :, ky][:, :, :, kx]
    rec["state_absmax"] = np.abs(st).reshape(6, -1).max(axis=1)
    np.savez_compressed(path, **rec)


if __name__ == "__main__":
    here = os.path.dirname(os.path.abspath(__file__))
    which = sys.argv[1:] or ["tiny"]
    if "tiny" in which:
        for name, c in CASES.items():
            with open(os.path.join(here, name + ".json"), "w") as f:
                json.dump(run(c), f, indent=1)
            print("wrote", name)
    if "bench" in which:
        bench_fixture(os.path.join(here, BENCH_FIXTURE))
        print("wrote", BENCH_FIXTURE)
