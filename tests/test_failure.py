"""Failure detection without a GPU fault: every failure here is made on the host or by a
bounded device wait that is told to give up, and the kernels always run to completion.

* A bounded wait forced to run out (gempic_set_wait_limit with 0 polls, two s-steps marched
  concurrently): the launch completes, the step returns GEMPIC_ETIMEOUT, and the simulation
  is sticky-failed (GEMPIC_ESTATE) afterwards; the CUDA context stays usable.
* A NaN planted in a host-built spectral state (gempic_set_state) reaches the FP64 field and
  kinetic energy sums, whose watchdog returns GEMPIC_ENONFINITE.
* A stored-particle bucket of capacity 1 with trapping returns GEMPIC_EOVERFLOW.
"""
import numpy as np
import pytest

from paper_2509_16793_gb300 import workloads as W

pytestmark = pytest.mark.gpu

ETIMEOUT, ESTATE, EOVERFLOW, ENONFINITE = -5, -6, -7, -8


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2509_16793_gb300 import build
    build.build()


def _status(f, *a):
    from paper_2509_16793_gb300 import gempic
    try:
        f(*a)
        return 0
    except gempic.GempicError as e:
        return e.status


def test_wait_that_runs_out_gives_etimeout_then_estate():
    from paper_2509_16793_gb300 import gempic
    w = W.small_3d(nx=16, ny=16, nzeta=48, ppc=1, precision=64)
    with gempic.Sim(w, cluster_ctas=2, pipeline_depth=2) as g:
        assert g.launch_shape()["pipeline"] == 2
        g.step(1)                                    # initialised, one s-step, no waits
        g.set_wait_limit(0)
        assert _status(g.step, 2) == ETIMEOUT        # the second march gives up at once
        assert _status(g.step, 1) == ESTATE
        assert _status(g.diagnostics) == ESTATE
        assert _status(g.set_wait_limit, 100) == ESTATE
    # the context is intact: a new simulation runs and matches a fresh reference run
    with gempic.Sim(w, cluster_ctas=2, pipeline_depth=2) as a, \
            gempic.Sim(w, cluster_ctas=2, pipeline_depth=1) as b:
        a.step(3)
        b.step(3)
        assert np.abs(a.state() - b.state()).max() <= 1e-12 * np.abs(b.state()).max()
    with gempic.Sim(w, cluster_ctas=2) as g:
        assert _status(g.set_wait_limit, -1) == -1


def test_nan_in_a_host_state_trips_the_watchdog():
    from paper_2509_16793_gb300 import gempic
    w = W.small_3d(nx=16, ny=16, nzeta=48, ppc=1, precision=64)
    with gempic.Sim(w, cluster_ctas=2) as g:
        s = g.state()
        s[0, 30, 3, 2] = np.nan                      # R_x of one mode of slice 30
        g.set_state(s)
        assert _status(g.step, 1) == ENONFINITE
        assert _status(g.step, 1) == ESTATE
    # the same state without the NaN steps normally
    with gempic.Sim(w, cluster_ctas=2) as g:
        s = g.state()
        g.set_state(s)
        g.step(1)
        d = g.diagnostics()
        assert np.isfinite(d["field_energy"]) and np.isfinite(d["kinetic_energy"])


def test_infinity_in_fp32_trips_the_watchdog():
    from paper_2509_16793_gb300 import gempic
    w = W.small_2d(nx=32, nzeta=64, ppc=2, precision=32)
    with gempic.Sim(w) as g:
        s = g.state()
        s[2, 40, 0, 1] = np.inf                      # E_z of one mode
        g.set_state(s)
        assert _status(g.step, 1) == ENONFINITE


def test_bucket_capacity_one_with_trapping_overflows():
    from paper_2509_16793_gb300 import gempic
    w = W.small_2d(nx=16, nzeta=96, ppc=2, precision=64, a0=2.0, delta=1.5)
    with gempic.Sim(w, bucket_capacity=1) as g:
        st = 0
        for _ in range(3):
            st = _status(g.step, 1)
            if st != 0:
                break
        assert st == EOVERFLOW
        assert _status(g.step, 1) == ESTATE
