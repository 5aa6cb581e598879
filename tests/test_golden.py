"""Fixtures under tests/golden/.

paper_sec6_parameters.json holds the values Sec. 6 prints for the paper's run; the workload
defaults that restate them are checked against it, and so is the stability bound at the
paper's own steps.  oracle_tiny_*.json are regression fixtures written by
tests/golden/make_golden.py, which calls only the oracle: the oracle must keep reproducing
them (a change to its arithmetic rewrites them in a commit that names the passage behind it),
and the GPU path must match them in FP64.
"""
import json
import math
import os

import numpy as np
import pytest

from paper_2509_16793_gb300 import workloads as W

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _load(name):
    with open(os.path.join(HERE, name)) as f:
        return json.load(f)


def _golden_module():
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(HERE, "make_golden.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_channel_defaults_are_the_papers():
    p = _load("paper_sec6_parameters.json")
    ch = W.Channel()
    assert ch.n1_over_n0 == pytest.approx(p["channel_n1_cm3"] / p["plasma_n0_cm3"])
    # radius in units of c/omega_L: R_ch / lambda * 2 pi
    assert ch.radius == pytest.approx(p["channel_radius_um"] / p["laser_wavelength_um"] * W.LAMBDA_L)


def test_papers_run_is_inside_the_stability_bound():
    """Delta h omega_p^2 <= 4 (Sec. 4.2) at the paper's steps: n0/n_cr with n_cr(0.8 um) =
    1.115e21 / lambda_um^2 cm^-3, lengths in c/omega_L = lambda / 2 pi."""
    p = _load("paper_sec6_parameters.json")
    lam = p["laser_wavelength_um"]
    ncr = 1.115e21 / lam ** 2
    wp2 = p["plasma_n0_cm3"] / ncr
    to_norm = 2.0 * math.pi / lam                           # um -> c/omega_L
    h = max(p["zeta_step_back_nm"], p["zeta_step_front_nm"]) * 1e-3 * to_norm
    for delta in p["delta_um"]:
        assert delta * to_norm * h * wp2 < 4.0
    # the refined profile helper reproduces the paper's two steps (its tanh joint reaches the
    # end values to within 1 % at the window's ends)
    hz = W.refined_h(3000, p["zeta_step_front_nm"], p["zeta_step_front_nm"] / p["zeta_step_back_nm"])
    assert hz.min() == pytest.approx(p["zeta_step_back_nm"], rel=1e-2)
    assert hz.max() == pytest.approx(p["zeta_step_front_nm"], rel=1e-2)


@pytest.mark.parametrize("name", ["oracle_tiny_2d", "oracle_tiny_3d"])
def test_oracle_reproduces_its_fixtures(name):
    g = _load(name + ".json")
    m = _golden_module()
    now = m.run(g["case"])
    for a, b in zip(now["steps"], g["steps"]):
        for k in ("n_trapped", "n_stored", "n_rejoined"):
            assert a[k] == b[k], k
        for k in ("field_energy", "kinetic_energy", "charge_flux"):
            assert a[k] == pytest.approx(b[k], rel=1e-12, abs=1e-300), k
        ez, gz = np.array(a["onaxis_ez"]), np.array(b["onaxis_ez"])
        assert np.abs(ez - gz).max() <= 1e-12 * np.abs(gz).max()
    for k, v in g["state_l1"].items():
        assert now["state_l1"][k] == pytest.approx(v, rel=1e-12, abs=1e-300), k


@pytest.mark.gpu
@pytest.mark.parametrize("name", ["oracle_tiny_2d", "oracle_tiny_3d"])
def test_gpu_matches_the_fixtures(name):
    from paper_2509_16793_gb300 import build, gempic
    build.build()
    g = _load(name + ".json")
    w = _golden_module().workload(g["case"])
    with gempic.Sim(w) as sim:
        for b in g["steps"]:
            sim.step()
            d = sim.diagnostics()
            for k in ("n_trapped", "n_stored", "n_rejoined"):
                assert d[k] == b[k], k
            for k in ("field_energy", "kinetic_energy", "charge_flux"):
                assert abs(d[k] - b[k]) <= 1e-10 * abs(b[k]), k
            ez, gz = sim.onaxis_ez(), np.array(b["onaxis_ez"])
            assert np.abs(ez - gz).max() <= 1e-10 * np.abs(gz).max()


def test_bench_fixture_is_complete_and_consistent():
    """The oracle's full-size bench fixture: both s-steps' diagnostics, the on-axis E_z over
    the window and the state sample; its charge flux is q n0 times the window's volume less the
    few particles trapped on the way (Sec. 5.1: every plane carries rho - j_z = q n0)."""
    m = _golden_module()
    f = np.load(os.path.join(HERE, m.BENCH_FIXTURE))
    w = W.lwfa_3d_128x128x1024()
    for k in range(2):
        assert f[f"onaxis_ez_{k}"].shape == (w.nzeta,) and np.isfinite(f[f"onaxis_ez_{k}"]).all()
        vol = w.nx * w.hx * w.ny * w.hy * w.nzeta * w.h
        qn = w.species[0].charge * w.species[0].density
        assert abs(float(f[f"charge_flux_{k}"]) / (qn * vol) - 1.0) < 2e-3
        assert f[f"field_energy_{k}"] > 0 and f[f"kinetic_energy_{k}"] > 0
    sl, ky, kx = m.bench_sample_index(w.ny)
    assert f["state_sample"].shape == (6, sl.size, ky.size, kx.size)
