"""s-steps with the state streamed through host memory (gempic_step_streamed).

The marches read every s-step's old level from a device buffer that the library refills from
the host, group of slices by group of slices, and write the new level to a second buffer that
it copies out; so the result is only right if every group went out and back in before the
next s-step read it.  It must equal the regular path's (same kernels, same arithmetic: the
state, each s-step's diagnostics), leave the simulation's own state at the last result, and
work with several s-steps in flight.
"""
import numpy as np
import pytest

from paper_2509_16793_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _pinned(nbytes):
    import torch
    return torch.empty(nbytes, dtype=torch.uint8, pin_memory=True).numpy()


def _run(w, n, pipeline, **kw):
    from paper_2509_16793_gb300 import build, gempic
    build.build()
    with gempic.Sim(w, pipeline_depth=pipeline, **kw) as ref:
        ref.step(1)                          # initialised, one s-step done
        s0 = ref.gempic_get_state()
        diags, states = [], []
        for _ in range(n):
            ref.step(1)
            diags.append(ref.diagnostics())
        states.append(ref.gempic_get_state())
        ref.step(1)
        after = ref.gempic_get_state()
    with gempic.Sim(w, pipeline_depth=pipeline, **kw) as g:
        g.step(1)
        s0g = g.gempic_get_state()
        # FP64 deposits add in floating-point shared-memory atomics: two runs agree to
        # round-off, not bit for bit
        assert _close(s0g, s0, 1e-12)
        host = _pinned(g.state_bytes())
        host.view(s0.dtype)[:] = s0g.reshape(-1)
        got = g.step_streamed(n, host)
        out = host.view(s0.dtype).reshape(s0.shape)
        dev = g.gempic_get_state()
        g.step(1)
        after_g = g.gempic_get_state()
    return diags, states[-1], after, got, out, dev, after_g


def _close(a, b, tol):
    scale = max(np.abs(b).max(), 1e-300)
    return np.abs(a - b).max() / scale <= tol


@pytest.mark.parametrize("pipeline", [1, 3])
def test_streamed_matches_regular_fp64(pipeline):
    w = W.small_3d(nx=16, ny=16, nzeta=40, ppc=2, precision=64, a0=2.0)
    n = 5
    diags, ref, after, got, out, dev, after_g = _run(w, n, pipeline, cluster_ctas=2)
    assert _close(out, ref, 1e-12)
    assert np.array_equal(dev, out)                  # the device state is the last result
    assert _close(after_g, after, 1e-12)             # and the simulation continues from it
    for i in range(n):
        assert got[i]["step"] == diags[i]["step"]
        for key in ("field_energy", "kinetic_energy", "charge_flux"):
            assert abs(got[i][key] - diags[i][key]) <= 1e-12 * abs(diags[i][key]) + 1e-300, (i, key)
        for key in ("pushes", "n_trapped", "n_stored", "n_rejoined"):
            assert got[i][key] == diags[i][key], (i, key)


def test_streamed_bench_shape_fp32():
    """The bench's launch shape (128 x 128, 16-CTA clusters, 7 s-steps in flight) on a
    shorter window, 9 s-steps: more s-steps than marches in flight."""
    w = W.lwfa_3d_128x128x1024()
    w = w.with_(nzeta=256, laser=W.Laser(**{**w.laser.__dict__,
                                            "zeta_center": 256 * w.h - 2.0 * w.laser.duration}))
    n = 9
    diags, ref, after, got, out, dev, after_g = _run(w, n, 7)
    assert _close(out, ref, 1e-6)
    assert np.array_equal(dev, out)
    assert _close(after_g, after, 1e-6)
    for i in range(n):
        for key in ("field_energy", "kinetic_energy"):
            assert abs(got[i][key] - diags[i][key]) <= 1e-6 * abs(diags[i][key]), (i, key)
        assert got[i]["pushes"] == diags[i]["pushes"]


def test_streamed_rejects_bad_arguments():
    from paper_2509_16793_gb300 import build, gempic
    build.build()
    w = W.small_3d(nx=16, ny=16, nzeta=16, ppc=1, precision=64, a0=0.5)
    with gempic.Sim(w) as g:
        small = np.zeros(g.state_bytes() - 8, np.uint8)
        with pytest.raises(ValueError):
            g.step_streamed(1, small)
        assert g.lib.gempic_step_streamed(g.h, -1, small.ctypes.data, small.nbytes, None) != 0
        assert g.lib.gempic_step_streamed(g.h, 1, None, g.state_bytes(), None) != 0
        assert g.lib.gempic_step_streamed(g.h, 1, small.ctypes.data, small.nbytes, None) != 0
