"""The allocation-free s-step (gempic_step_noalloc) against the regular entry point.

Callers that cannot allocate device memory use gempic_step_noalloc on a state they own; its
working memory is a fixed array inside the library.  Two calls in a row from the same initial
state must reproduce two regular gempic_step calls within the FP64 parity tolerance, and
oversized grids must be rejected before any work.
"""
import numpy as np
import pytest

from paper_2509_16793_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("channel", [False, True])
def test_noalloc_matches_gempic_step_twice(channel):
    import torch
    from paper_2509_16793_gb300 import build, gempic
    build.build()
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream().cuda_stream
    # a laser weak enough that no particle is trapped (the allocation-free step keeps no
    # stored particles)
    w = W.small_3d(nx=16, ny=16, nzeta=40, ppc=2, precision=64, a0=0.8)
    if channel:                            # density channel (Eq. n_plasma) through the config
        w = w.with_(channel=W.Channel(0.25, 3.0 * w.hx))
    with gempic.Sim(w, cluster_ctas=2, stream=stream) as ref:
        shape = ref.state_shape()
        s0 = torch.empty(shape, dtype=torch.complex128, device="cuda")
        ref.gempic_get_state(s0)
        outs = []
        diags = []
        for k in range(2):
            ref.step(1)
            outs.append(ref.gempic_get_state())
            diags.append(ref.diagnostics())
    state = s0.clone()
    for k in range(2):
        st, d, ez = gempic.gempic_step_noalloc(w, k, state, onaxis=True, stream=stream,
                                               cluster_ctas=2)
        torch.cuda.synchronize()
        assert st == 0, gempic.load().gempic_strerror(st).decode()
        got = state.cpu().numpy()
        exp = outs[k]
        for c in range(6):
            scale = np.abs(exp[c]).max()
            err = np.abs(got[c] - exp[c]).max()
            assert err <= 1e-10 * max(scale, 1e-300), (k, c, err, scale)
        for key in ("field_energy", "kinetic_energy", "charge_flux"):
            assert abs(d[key] - diags[k][key]) <= 1e-10 * abs(diags[k][key]), key
        assert d["pushes"] == w.pushes_per_step and d["n_trapped"] == 0
        assert np.isfinite(ez).all()


def test_noalloc_rejects_sizes_beyond_its_limits():
    import torch
    from paper_2509_16793_gb300 import gempic
    torch.cuda.set_device(0)
    small = torch.zeros(16, dtype=torch.complex128, device="cuda")
    w = W.small_3d(nx=16, ny=16, nzeta=5000, ppc=1, precision=64)
    st, _, _ = gempic.gempic_step_noalloc(w, 0, small)
    assert st == -1                        # nzeta above 4096
    w = W.small_3d(nx=16, ny=16, nzeta=40, ppc=1, precision=64)
    st, _, _ = gempic.gempic_step_noalloc(w, 0, small)
    assert st == -1                        # state buffer too small
