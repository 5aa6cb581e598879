"""Plain numpy oracle of the learned current denoiser (TEST INFRASTRUCTURE ONLY, like the rest
of oracle/: only tests/, __graft_entry__.smoke() and bench.py's baseline legs use it).

The paper's method deposits the current of every macroparticle; with few particles per cell
that current is noisy.  The denoiser is a small 3-D convolutional net applied to the current
j = (j_x, j_y, j_z) on the half-slice grid [nzeta][ny][nx] before the field update, trained on
pairs of runs of the method itself (few versus many particles per cell).  The paper has no
such component; its structure follows the benchmark spec: three 3x3x3 convolution layers,
16 hidden channels, ReLU between layers, in BF16 with FP32 accumulation on the GPU.

Conventions shared with the GPU path (each side implements them separately):
  * tensors are channel-last, X[z][y][x][c]; z is the zeta index (half-slices), y, x the
    transverse nodes;
  * a tap (dz, dy, dx) in {-1, 0, 1}^3 reads X[z + dz][y + dy][x + dx]; the transverse
    directions are periodic (the field solve's boundary condition), zeta is zero-padded
    (nothing outside the window);
  * weights W[dz + 1][dy + 1][dx + 1][c_in][c_out], bias b[c_out];
  * the net: x0 = j / scale, h1 = relu(conv1(x0)), h2 = relu(conv2(h1)), r = conv3(h2),
    denoised j = j + scale r (residual form: a zero last layer is the identity);
  * loss: mean over voxels and the 3 components of (x0 + r - t)^2, t = j_target / scale;
  * Adam (Kingma and Ba, ICLR 2015) with bias correction.
Everything here runs in FP64; the GPU rounds activations and weights to BF16, which the
parity tests account for.
"""
from __future__ import annotations

import itertools

import numpy as np

TAPS = list(itertools.product((-1, 0, 1), repeat=3))     # (dz, dy, dx), row-major order


def shifted(X, dz, dy, dx):
    """S[z][y][x] = X[z + dz][y + dy][x + dx]: periodic across, zero outside the window in z."""
    S = np.roll(X, shift=(-dy, -dx), axis=(1, 2))
    if dz == 0:
        return S
    out = np.zeros_like(S)
    if dz > 0:
        out[:-dz] = S[dz:]
    else:
        out[-dz:] = S[:dz]
    return out


def conv3d(X, W, b=None):
    """Y[z,y,x,o] = b[o] + sum over taps and input channels of X[z+dz,y+dy,x+dx,i] W[tap,i,o]."""
    nz, ny, nx, ci = X.shape
    co = W.shape[-1]
    Y = np.zeros((nz, ny, nx, co))
    for dz, dy, dx in TAPS:
        Y += shifted(X, dz, dy, dx) @ W[dz + 1, dy + 1, dx + 1]
    if b is not None:
        Y += b
    return Y


def conv3d_backward(X, W, dY):
    """Gradients of sum(dY * conv3d(X, W, b)) with respect to X, W and b."""
    dX = np.zeros_like(X)
    dW = np.zeros_like(W)
    for dz, dy, dx in TAPS:
        Wt = W[dz + 1, dy + 1, dx + 1]
        # Y[v] gets X[v + t] Wt: X[u] receives dY[u - t] Wt^T
        dX += shifted(dY, -dz, -dy, -dx) @ Wt.T
        dW[dz + 1, dy + 1, dx + 1] = np.einsum("zyxi,zyxo->io", shifted(X, dz, dy, dx), dY)
    return dX, dW, dY.sum(axis=(0, 1, 2))


def relu(a):
    return np.maximum(a, 0.0)


def init_params(seed=1, hidden=16, cin=3, scale3=0.0):
    """Seeded He-style initial weights (normal, std sqrt(2 / fan_in)); the last layer is scaled
    by scale3 (0: the net starts as the identity on j)."""
    rng = np.random.default_rng(seed)
    def w(ci, co, s=1.0):
        return rng.standard_normal((3, 3, 3, ci, co)) * np.sqrt(2.0 / (27 * ci)) * s
    return {"W1": w(cin, hidden), "b1": np.zeros(hidden),
            "W2": w(hidden, hidden), "b2": np.zeros(hidden),
            "W3": w(hidden, cin, scale3), "b3": np.zeros(cin)}


def forward(P, x0):
    """(r, cache): the net's correction r for the normalised current x0 [nz, ny, nx, 3]."""
    a1 = conv3d(x0, P["W1"], P["b1"])
    h1 = relu(a1)
    a2 = conv3d(h1, P["W2"], P["b2"])
    h2 = relu(a2)
    r = conv3d(h2, P["W3"], P["b3"])
    return r, (x0, a1, h1, a2, h2)


def loss_and_grad(P, x0, t):
    """Mean squared error of x0 + r against t and its gradients with respect to P."""
    r, (x0, a1, h1, a2, h2) = forward(P, x0)
    e = x0 + r - t
    n = e.size
    loss = float((e * e).sum() / n)
    dr = 2.0 * e / n
    g = {}
    dh2, g["W3"], g["b3"] = conv3d_backward(h2, P["W3"], dr)
    da2 = dh2 * (a2 > 0)
    dh1, g["W2"], g["b2"] = conv3d_backward(h1, P["W2"], da2)
    da1 = dh1 * (a1 > 0)
    _, g["W1"], g["b1"] = conv3d_backward(x0, P["W1"], da1)
    return loss, g


def adam_step(P, g, m, v, k, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (k = 1, 2, ... the step count) of every parameter, in place."""
    for name in P:
        m[name] = beta1 * m[name] + (1 - beta1) * g[name]
        v[name] = beta2 * v[name] + (1 - beta2) * g[name] ** 2
        mh = m[name] / (1 - beta1 ** k)
        vh = v[name] / (1 - beta2 ** k)
        P[name] = P[name] - lr * mh / (np.sqrt(vh) + eps)


def denoise(P, j, scale):
    """The denoised current j + scale r(j / scale), j [nz, ny, nx, 3]."""
    r, _ = forward(P, j / scale)
    return j + scale * r


def to_bf16(a):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    rounded = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return rounded.astype(np.uint32).view(np.float32).astype(np.float64)


def denoise_bf16(P, J, scale):
    """The denoiser at the GPU's rounding points, on a current J [nz, 3, ny, nx]: the input
    j/scale, the weights and the hidden activations rounded to BF16, biases, sums and the
    residual add in full precision."""
    j = np.asarray(J, np.float64).transpose(0, 2, 3, 1)
    Q = {k: (to_bf16(v) if k.startswith("W") else np.asarray(v, np.float32).astype(np.float64))
         for k, v in P.items()}
    x0 = to_bf16(j / scale)
    h1 = to_bf16(relu(conv3d(x0, Q["W1"], Q["b1"])))
    h2 = to_bf16(relu(conv3d(h1, Q["W2"], Q["b2"])))
    r = conv3d(h2, Q["W3"], Q["b3"])
    return (j + scale * r).transpose(0, 3, 1, 2)
