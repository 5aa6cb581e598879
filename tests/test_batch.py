"""Batched parameter scan: independent instances stepped side by side.

CPU: the scan's input recipe.  GPU: every instance of a batch equals the same simulation run
alone (identical kernels and inputs; FP64 current deposits are floating-point shared-memory
reductions whose order varies between runs, so equal to rounding), and an instance matches
the oracle.
"""
import numpy as np
import pytest

from paper_2509_16793_gb300 import workloads as W


def test_scan_inputs_follow_the_recipe():
    ws = W.scan_2d(n=64)
    assert len(ws) == 64
    for w in ws:
        assert w.ny == 1 and w.nx in (128, 256, 512) and w.nzeta in (256, 512, 1024, 2048)
        assert 0.5 <= w.laser.a0 <= 3.0
        n0 = w.species[0].density
        assert 1e-3 <= n0 <= 1e-2 and w.species[0].ppc == 4
        assert abs(w.delta * w.h * n0 - 4.0) < 1e-12          # at the stability limit
    assert len({w.seed for w in ws}) == 64
    again = W.scan_2d(n=64)
    assert [(w.nx, w.nzeta, w.laser.a0, w.species[0].density) for w in ws] == \
           [(w.nx, w.nzeta, w.laser.a0, w.species[0].density) for w in again]


def _small_instances():
    base = [W.small_2d(nx=32, nzeta=48, ppc=3, precision=64),
            W.small_2d(nx=16, nzeta=64, ppc=2, precision=64, a0=1.5),
            W.small_2d(nx=64, nzeta=32, ppc=2, precision=64, a0=0.7, n0=0.02),
            W.small_2d(nx=32, nzeta=40, ppc=4, precision=64, a0=2.0)]
    return [w.with_(seed=w.seed + i) for i, w in enumerate(base)]


@pytest.mark.gpu
def test_batch_instances_equal_single_runs():
    from paper_2509_16793_gb300 import build, gempic
    build.build()
    ws = _small_instances()
    with gempic.Batch(ws) as b:
        assert len(b) == len(ws)
        b.step(1)
        b.step(2)
        for w, v in zip(ws, b.sims):
            with gempic.Sim(w, pipeline_depth=1) as g:
                g.step(1)
                g.step(2)
                a, r = v.state(), g.state()
                fs = max(np.abs(r[c]).max() for c in range(4))       # fields
                js = max(np.abs(r[c]).max() for c in (4, 5))         # currents
                for c in range(6):
                    scale = fs if c < 4 else js
                    assert np.abs(a[c] - r[c]).max() <= 1e-12 * scale, (w.name, c)
                da, dr = v.diagnostics(), g.diagnostics()
                for k in ("step", "n_trapped", "n_stored", "n_rejoined", "pushes"):
                    assert da[k] == dr[k], (w.name, k)
                for k in ("field_energy", "kinetic_energy"):
                    assert abs(da[k] - dr[k]) <= 1e-12 * abs(dr[k]), (w.name, k)
                ez, rz = v.onaxis_ez(), g.onaxis_ez()
                assert np.abs(ez - rz).max() <= 1e-12 * max(np.abs(rz).max(), 1e-300), w.name


@pytest.mark.gpu
def test_batch_instance_matches_oracle():
    from oracle import RefSim
    from paper_2509_16793_gb300 import build, gempic
    build.build()
    ws = _small_instances()
    o = RefSim(ws[2])
    with gempic.Batch(ws) as b:
        for _ in range(2):
            od = o.step()
            b.step(1)
        g = b.sims[2]
        st, ref = g.state(), o.state()
        fs = max(np.abs(ref[c]).max() for c in range(4))
        js = max(np.abs(ref[c]).max() for c in (4, 5))
        for c in range(6):
            scale = fs if c < 4 else js
            assert np.abs(st[c] - ref[c]).max() <= 1e-10 * scale, c
        for k in ("field_energy", "kinetic_energy"):
            assert abs(g.diagnostics()[k] - od[k]) <= 1e-10 * abs(od[k])


@pytest.mark.gpu
def test_batch_rejects_an_invalid_member():
    from paper_2509_16793_gb300 import build, gempic
    build.build()
    ws = _small_instances()
    ws[1] = ws[1].with_(nx=24)                                 # not a power of two
    with pytest.raises(gempic.GempicError):
        gempic.Batch(ws)
