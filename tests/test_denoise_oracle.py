"""Pins of the denoiser oracle (oracle/denoise_ref.py), no GPU: the convolution's taps against
identities and brute force, the backward pass against finite differences and the adjoint
identity, Adam's first step against its closed form, BF16 rounding against torch."""
import itertools

import numpy as np
import pytest

from oracle import denoise_ref as D


def _rand(shape, seed):
    return np.random.default_rng(seed).standard_normal(shape)


def test_delta_kernel_is_the_identity():
    X = _rand((5, 4, 6, 3), 1)
    W = np.zeros((3, 3, 3, 3, 3))
    W[1, 1, 1] = np.eye(3)
    b = np.array([0.5, -1.0, 2.0])
    assert np.array_equal(D.conv3d(X, W, b), X + b)


@pytest.mark.parametrize("axis,tap", [(2, (1, 1, 2)), (1, (1, 2, 1)), (0, (2, 1, 1)), (0, (0, 1, 1))])
def test_tap_orientation_and_boundaries(axis, tap):
    """A single tap (dz, dy, dx) reads X[z+dz][y+dy][x+dx]: across it wraps (periodic), along
    zeta it reads zero outside the window."""
    X = _rand((5, 4, 6, 2), 2)
    W = np.zeros((3, 3, 3, 2, 2))
    W[tap] = np.eye(2)
    Y = D.conv3d(X, W)
    d = tap[axis] - 1
    if axis > 0:
        assert np.array_equal(Y, np.roll(X, -d, axis=axis))
    else:
        Z = np.zeros_like(X)
        if d > 0:
            Z[:-1] = X[1:]
        else:
            Z[1:] = X[:-1]
        assert np.array_equal(Y, Z)


def test_conv_against_brute_force():
    nz, ny, nx, ci, co = 4, 3, 5, 3, 4
    X = _rand((nz, ny, nx, ci), 3)
    W = _rand((3, 3, 3, ci, co), 4)
    b = _rand((co,), 5)
    Y = D.conv3d(X, W, b)
    for z, y, x in itertools.product(range(nz), range(ny), range(nx)):
        acc = b.copy()
        for kz, ky, kx in itertools.product(range(3), repeat=3):
            zz = z + kz - 1
            if zz < 0 or zz >= nz:
                continue
            acc += X[zz, (y + ky - 1) % ny, (x + kx - 1) % nx] @ W[kz, ky, kx]
        assert np.allclose(Y[z, y, x], acc, rtol=0, atol=1e-12)


def test_backward_is_the_adjoint_and_matches_finite_differences():
    X = _rand((4, 3, 5, 3), 6)
    W = _rand((3, 3, 3, 3, 2), 7)
    b = _rand((2,), 8)
    G = _rand((4, 3, 5, 2), 9)
    dX, dW, db = D.conv3d_backward(X, W, G)
    # adjoint: <conv(X), G> = <X, dX> (linear in X, no bias)
    assert abs((D.conv3d(X, W) * G).sum() - (X * dX).sum()) < 1e-10
    f = lambda X_, W_, b_: (D.conv3d(X_, W_, b_) * G).sum()
    eps = 1e-6
    rng = np.random.default_rng(10)
    for _ in range(8):
        i = tuple(rng.integers(0, s) for s in X.shape)
        Xp, Xm = X.copy(), X.copy()
        Xp[i] += eps
        Xm[i] -= eps
        assert abs((f(Xp, W, b) - f(Xm, W, b)) / (2 * eps) - dX[i]) < 1e-6
        j = tuple(rng.integers(0, s) for s in W.shape)
        Wp, Wm = W.copy(), W.copy()
        Wp[j] += eps
        Wm[j] -= eps
        assert abs((f(X, Wp, b) - f(X, Wm, b)) / (2 * eps) - dW[j]) < 1e-6
    assert np.allclose(db, G.sum(axis=(0, 1, 2)))


def test_net_gradient_matches_finite_differences():
    P = D.init_params(seed=3, hidden=4, cin=3, scale3=1.0)
    x0 = _rand((4, 3, 4, 3), 11)
    t = _rand((4, 3, 4, 3), 12)
    loss, g = D.loss_and_grad(P, x0, t)
    eps = 1e-6
    rng = np.random.default_rng(13)
    for name in ("W1", "b1", "W2", "b2", "W3", "b3"):
        for _ in range(3):
            i = tuple(rng.integers(0, s) for s in P[name].shape)
            Pp = {k: v.copy() for k, v in P.items()}
            Pm = {k: v.copy() for k, v in P.items()}
            Pp[name][i] += eps
            Pm[name][i] -= eps
            fd = (D.loss_and_grad(Pp, x0, t)[0] - D.loss_and_grad(Pm, x0, t)[0]) / (2 * eps)
            assert abs(fd - g[name][i]) < 1e-6 * max(1.0, abs(fd)), (name, i, fd, g[name][i])


def test_zero_last_layer_is_the_identity():
    P = D.init_params(seed=1, scale3=0.0)
    j = _rand((3, 4, 4, 3), 14)
    assert np.array_equal(D.denoise(P, j, 0.7), j)


def test_adam_first_step_is_lr_times_sign():
    """With bias correction, m_hat / sqrt(v_hat) = g / |g| at step 1 (Kingma and Ba 2015)."""
    P = {"w": np.array([1.0, -2.0, 0.5])}
    g = {"w": np.array([0.3, -4.0, 1e-3])}
    m = {"w": np.zeros(3)}
    v = {"w": np.zeros(3)}
    D.adam_step(P, g, m, v, 1, lr=0.01, eps=0.0)
    assert np.allclose(P["w"], np.array([1.0, -2.0, 0.5]) - 0.01 * np.sign(g["w"]), rtol=0, atol=1e-15)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    a = np.concatenate([_rand(1000, 15) * 10 ** _rand(1000, 16),
                        [1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -3.0 - 2 ** -7, 0.0]])
    want = torch.tensor(a, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(D.to_bf16(a), want)


def test_denoised_step_with_the_identity_is_the_plain_step():
    """The oracle's two-pass s-step with denoise = identity reproduces the plain s-step (the
    second pass recomputes the level from the same current), trapping included."""
    from oracle import RefSim
    from paper_2509_16793_gb300 import workloads as W
    w = W.small_2d(nx=16, nzeta=48, ppc=2, a0=2.0, delta=1.5)
    a, b = RefSim(w), RefSim(w)
    for _ in range(3):
        da = a.step()
        db = b.step_denoised(lambda J: J)
        for k in ("field_energy", "kinetic_energy", "charge_flux"):
            assert db[k] == pytest.approx(da[k], rel=1e-13, abs=1e-300), k
        for k in ("n_trapped", "n_stored", "n_rejoined"):
            assert db[k] == da[k]
    assert np.abs(a.state() - b.state()).max() <= 1e-13 * np.abs(a.state()).max()
    assert da["n_trapped"] > 0 or a.stored.n > 0


def test_denoised_step_is_linear_in_the_current_change():
    """The field update is linear in the current and diagonal in the transverse modes: adding
    a uniform j_z offset in the second pass changes only the (kx, ky) = 0 mode of the state."""
    from oracle import RefSim
    from paper_2509_16793_gb300 import workloads as W
    w = W.small_2d(nx=16, nzeta=32, ppc=2, a0=1.0)
    a, b = RefSim(w), RefSim(w)
    a.step_denoised(lambda J: J)
    c = 1e-3

    def shift(J):
        J = J.copy()
        J[:, 2] += c
        return J
    b.step_denoised(shift)
    d = b.state() - a.state()
    d[:, :, 0, 0] = 0.0                       # the k = 0 column may change
    assert np.abs(d).max() <= 1e-13 * np.abs(a.state()).max()
