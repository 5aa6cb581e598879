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


@pytest.mark.parametrize("nx,cluster", [(16, 2), (128, 16)])
def test_noalloc_fp32_matches_gempic_step(nx, cluster):
    """FP32, within the FP32 parity tolerance (1e-4): a 16 x 16 grid and the bench grid
    128 x 128 with 16 CTAs (8 rows per CTA: the kernel compiled for that grid's transforms)."""
    import torch
    from paper_2509_16793_gb300 import build, gempic
    build.build()
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream().cuda_stream
    w = W.small_3d(nx=nx, ny=nx, nzeta=40, ppc=2, precision=32, a0=0.8)
    with gempic.Sim(w, cluster_ctas=cluster, stream=stream) as ref:
        s0 = torch.empty(ref.state_shape(), dtype=torch.complex64, device="cuda")
        ref.gempic_get_state(s0)
        outs, diags = [], []
        for k in range(2):
            ref.step(1)
            outs.append(ref.gempic_get_state())
            diags.append(ref.diagnostics())
    state = s0.clone()
    for k in range(2):
        st, d, ez = gempic.gempic_step_noalloc(w, k, state, onaxis=True, stream=stream,
                                               cluster_ctas=cluster)
        torch.cuda.synchronize()
        assert st == 0, gempic.load().gempic_strerror(st).decode()
        got = state.cpu().numpy()
        for c in range(6):
            scale = np.abs(outs[k][c]).max()
            assert np.abs(got[c] - outs[k][c]).max() <= 1e-4 * max(scale, 1e-30), (k, c)
        for key in ("field_energy", "kinetic_energy"):
            assert abs(d[key] - diags[k][key]) <= 1e-4 * abs(diags[k][key]), key


def test_noalloc_trapping_returns_eoverflow_and_advances():
    """There is no stored-particle store: a step that traps particles still advances the
    state (finite), drops the trapped particles and returns GEMPIC_EOVERFLOW."""
    import torch
    from paper_2509_16793_gb300 import build, gempic
    build.build()
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream().cuda_stream
    w = W.small_2d(nx=16, nzeta=96, ppc=2, precision=64, a0=2.0, delta=1.5)
    with gempic.Sim(w, stream=stream) as ref:
        s0 = torch.empty(ref.state_shape(), dtype=torch.complex128, device="cuda")
        ref.gempic_get_state(s0)
    state = s0.clone()
    st, d, ez = gempic.gempic_step_noalloc(w, 0, state, onaxis=True, stream=stream)
    torch.cuda.synchronize()
    assert st == -7
    assert d["n_trapped"] > 0
    assert torch.isfinite(torch.view_as_real(state)).all()
    assert not torch.equal(state, s0)
    assert np.isfinite(ez).all()


def test_noalloc_allocates_no_device_memory():
    """After the set-up call, further calls leave the free device memory and torch's
    allocator untouched."""
    import torch
    from paper_2509_16793_gb300 import build, gempic
    build.build()
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream().cuda_stream
    w = W.small_3d(nx=16, ny=16, nzeta=40, ppc=2, precision=64, a0=0.8)
    with gempic.Sim(w, cluster_ctas=2, stream=stream) as ref:
        state = torch.empty(ref.state_shape(), dtype=torch.complex128, device="cuda")
        ref.gempic_get_state(state)
    st, _, _ = gempic.gempic_step_noalloc(w, 0, state, stream=stream, cluster_ctas=2)
    assert st == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for k in range(1, 3):
        st, _, _ = gempic.gempic_step_noalloc(w, k, state, stream=stream, cluster_ctas=2)
        assert st == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0 and torch.cuda.memory_allocated() == alloc0


def test_noalloc_rejects_what_it_has_no_buffers_for():
    import torch
    from paper_2509_16793_gb300 import gempic
    torch.cuda.set_device(0)
    w = W.small_3d(nx=16, ny=16, nzeta=40, ppc=1, precision=64)
    state = torch.zeros((6, 40, 16, 8), dtype=torch.complex128, device="cuda")
    for kw in (dict(residual=True), dict(snapshot=True),
               dict(beam=W.Beam(n_macro=10, sigma_r=1.0, sigma_z=1.0, zeta_center=5.0))):
        st, _, _ = gempic.gempic_step_noalloc(w.with_(**kw), 0, state)
        assert st == -1, kw


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
