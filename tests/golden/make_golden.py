"""Writes the oracle regression fixtures of tests/golden/ (run from the repository root:
python tests/golden/make_golden.py).  Calls only oracle/ and the input recipes; the values
guard the oracle against unintended changes (test_golden.py), they do not pin it."""
import json
import os
import sys

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


if __name__ == "__main__":
    here = os.path.dirname(os.path.abspath(__file__))
    for name, c in CASES.items():
        with open(os.path.join(here, name + ".json"), "w") as f:
            json.dump(run(c), f, indent=1)
        print("wrote", name)
