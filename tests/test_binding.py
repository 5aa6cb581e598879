"""Argument marshalling of the ctypes binding (no GPU): what config_from_workload hands the
C-ABI for the options beyond the basic run, and the input recipes behind them."""
import math

import numpy as np
import pytest

from paper_2509_16793_gb300 import gempic as G
from paper_2509_16793_gb300 import workloads as W


def test_plain_workload_sets_no_options():
    w = W.small_2d(nx=16, nzeta=24, ppc=2)
    cfg, keep = G.config_from_workload(w)
    assert not cfg.channel and not cfg.hz            # NULL pointers
    assert bool(cfg.laser) and cfg.laser.contents.a0 == w.laser.a0
    assert cfg.flags & G.GEMPIC_FLAG_DIAG and not cfg.flags & G.GEMPIC_FLAG_GT1
    assert cfg.grid.nx == 16 and cfg.grid.nzeta == 24 and cfg.delta == w.delta
    assert cfg.species[0].ppc == 2 and cfg.species[0].density == w.species[0].density


def test_gt1_channel_and_table_reach_the_config():
    w = W.small_2d(nx=16, nzeta=24, ppc=2)
    hz = W.refined_h(w.nzeta, w.h, 2.0)
    w = w.with_(particle_law="GT1", channel=W.Channel(0.25, 7.0), hz=hz)
    cfg, keep = G.config_from_workload(w)
    assert cfg.flags & G.GEMPIC_FLAG_GT1
    assert cfg.channel.contents.n1_over_n0 == 0.25 and cfg.channel.contents.radius == 7.0
    assert [cfg.hz[i] for i in range(w.nzeta)] == list(hz)


@pytest.mark.parametrize("bad", [dict(particle_law="GT3"), dict(hz=np.ones(5))])
def test_bad_options_are_refused_before_the_library(bad):
    w = W.small_2d(nx=16, nzeta=24, ppc=2).with_(**bad)
    with pytest.raises(ValueError):
        G.config_from_workload(w)


def test_refined_profile():
    """Fine over the back third, coarse in front, monotone, joined smoothly (neighbouring
    slabs differ by a small fraction of a slab)."""
    hz = W.refined_h(900, 1.0, 4.0)
    assert hz[0] == pytest.approx(0.25, rel=2e-2) and hz[-1] == pytest.approx(1.0, rel=2e-2)
    assert np.all(np.diff(hz) >= 0)
    assert np.max(np.abs(np.diff(hz))) < 0.02
    mid = np.searchsorted(hz, 0.625)
    assert abs(mid / 900 - 1.0 / 3.0) < 0.02


def test_channel_defaults_convert_the_papers_units():
    ch = W.Channel()
    assert ch.radius == pytest.approx(76.4 / 0.8 * 2 * math.pi)
