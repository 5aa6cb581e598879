"""Plain FP64 numpy oracle of one GEM-PIC s-step (arXiv 2509.16793).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Every function restates a passage of the
paper, cited by section / equation.  It is written for reading, not speed: no blocking, no
fusion, particle loops vectorised only over independent particles.

The paper is silent or garbled in places; the readings taken here are:
  * LyN uses (B_z0^1 + B_z1^1)/2 (the printed B_z0^0 is a typo; LxN has the same form).
  * eqall carries +i k_y (B_x0 + B_x1)/2, as in the continuous Eq. EzGu.
  * The lower index of the slice scheme is the zeta-slice: 0 = zeta_0, 1 = zeta_0 + h.
  * The unknown j^1_{-1/2} of Eqs. RxN/RyN is predicted as j^1_{+1/2}; once the true
    j^1_{-1/2} has been deposited (next zeta step) R^1 of that slice is corrected by
    -(Delta/4)(j_true - j_pred) (Sec. 4.1, predictor-corrector).  At slice 0, j_{-1/2} := j_{+1/2}.
  * Transverse boundaries are periodic; the x- and y-Nyquist modes are projected out.
  * The front ghost slice zeta_{N} has R = L = E_z = B_z = 0 and E = B = 0.
  * Particles (GT2, Sec. 5): u on half-slices, r_perp and s~ on slices; a deterministic
    two-pass Boris step resolves the implicit dependence of dt = h/(1 - v_z) on v_z.
  * Step length: -dzeta = min(d, (Delta - sigma)(1 - v_z)/v_z) with v_z taken before the
    step (Eq. trap2); a particle whose step is cut short is trapped and kept in the box with
    its weight unchanged.
  * Transverse shape: cloud-in-cell; j_perp by the 2-D Esirkepov decomposition of the
    transverse move across one slice, so that (rho - j_z) is conserved through the planes.
  * Plasma channel (Sec. 6, Eq. n_plasma): its axis is the grid's middle node (x_c, y_c) =
    (nx hx/2, ny hy/2), as for the laser; immobile ions carry no current in the slice
    equations, so the profile enters only through each fresh macroparticle's charge, taken
    at its injection position.
  * Particle law GT1 (Sec. 5, Eq. trap1; the default is GT2): the s-budget is the lab time,
    ds = |dzeta|/(1 - v_z), the step is min(d, (Delta - sigma)(1 - v_z)); a stored particle
    advances by the lab time Delta (zeta += Delta (v_z - 1)) and rejoins the zeta march when
    Delta (1 - v_z) >= h.  The current deposit is the same under both laws.
  * Variable Delta (Sec. 6 changes Delta along the run without saying how the change meets
    the stored set): the stored set's advance from s^k to s^{k+1} uses the Delta of s-step k,
    the one whose fields it gathers; after a change the stored set lags it by one s-step.
  * Stored (trapped / beam) particles are pushed along the slow coordinate s (Sec. 5.1, last
    paragraph) with the fields of the last completed level; a
    stored particle with Delta(1-v_z)/v_z >= h rejoins the zeta march at its slice.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Dict, List, Optional

import numpy as np

# ----------------------------------------------------------------------------------------
# Counter-based SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
# generators", OOPSLA 2014): output number c of the stream seeded with `seed` is
# mix(seed + (c + 1) * golden_gamma).  Fresh-particle offsets are drawn with it.
# ----------------------------------------------------------------------------------------
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, counter: np.ndarray) -> np.ndarray:
    """Output `counter` (uint64 array) of the SplitMix64 stream seeded with `seed`."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (counter.astype(np.uint64) + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform24(seed: int, counter: np.ndarray) -> np.ndarray:
    """Uniform [0, 1) with 24 random bits (exact in both FP32 and FP64)."""
    return (splitmix64(seed, counter) >> np.uint64(40)).astype(np.float64) * (2.0 ** -24)


def uniform53(seed: int, counter: np.ndarray) -> np.ndarray:
    """Uniform (0, 1] with 53 random bits: (top 53 bits + 1) / 2^53 (never 0, so that the
    logarithm of the Box-Muller transform is finite)."""
    return ((splitmix64(seed, counter) >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)


def box_muller(v0: np.ndarray, v1: np.ndarray):
    """Two independent standard normals from two uniforms on (0, 1] (Box and Muller, Ann.
    Math. Stat. 29 (1958) 610): radius sqrt(-2 ln v0), angle 2 pi v1."""
    r = np.sqrt(-2.0 * np.log(v0))
    return r * np.cos(2.0 * math.pi * v1), r * np.sin(2.0 * math.pi * v1)


def sample_beam(b, nx, ny, hx, hy, length):
    """Gaussian bunch of equal-charge macroparticles (beam particles of Sec. 5.1, placed in the
    box at creation).  Density n_peak exp(-r^2/(2 sr^2) - (zeta - zc)^2/(2 sz^2)) around the
    grid's middle node; macroparticle i uses SplitMix64 outputs 4 i .. 4 i + 3 of the stream
    b.seed as uniforms on (0, 1] and the Box-Muller pairs (g0, g1), (g2, g3):
    x = x_c + sr g0, y = y_c + sr g1 (periodic), zeta = zc + sz g2, gamma (1 + spread g3) along
    +z, no transverse momentum.  Returns (x, y, zeta, u [3, N], Q) of the macroparticles with
    0 < zeta <= length; each carries total charge / n_macro."""
    i = np.arange(int(b.n_macro), dtype=np.uint64)
    v = [uniform53(int(b.seed), np.uint64(4) * i + np.uint64(j)) for j in range(4)]
    g0, g1 = box_muller(v[0], v[1])
    g2, g3 = box_muller(v[2], v[3])
    lx, ly = nx * hx, ny * hy
    x = np.mod(0.5 * lx + b.sigma_r * g0, lx)
    y = np.mod(0.5 * ly + b.sigma_r * g1, ly) if ny > 1 else np.zeros(i.size)
    zeta = b.zeta_center + b.sigma_z * g2
    gam = b.gamma * (1.0 + b.rel_spread * g3)
    uz = np.sqrt(np.maximum(gam * gam - 1.0, 0.0))
    if ny > 1:
        total = b.charge * b.n_peak * (2.0 * math.pi) ** 1.5 * b.sigma_r ** 2 * b.sigma_z
    else:
        total = b.charge * b.n_peak * 2.0 * math.pi * b.sigma_r * b.sigma_z
    keep = (zeta > 0.0) & (zeta <= length)
    n = int(keep.sum())
    u = np.stack([np.zeros(n), np.zeros(n), uz[keep]])
    return x[keep], y[keep], zeta[keep], u, np.full(n, total / max(int(b.n_macro), 1))


# ----------------------------------------------------------------------------------------
# Transverse spectral transform (Sec. 3.1: 2-D Fourier transform in (x, y), d/dx -> i k_x).
# Layout: [..., ky (ny), kx (nx/2)]; the kx-Nyquist column is dropped and the ky-Nyquist row
# is zeroed.  Staggered currents (stored at x + hx/2 or y + hy/2) are shifted to the nodes.
# ----------------------------------------------------------------------------------------
class Spectral:
    def __init__(self, nx: int, ny: int, hx: float, hy: float):
        self.nx, self.ny = nx, ny
        self.kx = 2.0 * math.pi * np.arange(nx // 2) / (nx * hx)            # [nx/2]
        self.ky = 2.0 * math.pi * np.fft.fftfreq(ny, d=hy)                   # [ny]
        self.mask = np.ones((ny, nx // 2))
        if ny > 1:
            self.mask[ny // 2, :] = 0.0
        self.shift_x = np.exp(-0.5j * self.kx * hx)[None, :]                 # x + hx/2 -> x
        self.shift_y = np.exp(-0.5j * self.ky * hy)[:, None]                 # y + hy/2 -> y

    def forward(self, a: np.ndarray, stagger: str = "") -> np.ndarray:
        """Real [ny, nx] -> spectral [ny, nx/2] (DFT, unnormalised)."""
        F = np.fft.fft(np.fft.rfft(a, axis=-1), axis=-2)[..., : self.nx // 2]
        if "x" in stagger:
            F = F * self.shift_x
        if "y" in stagger:
            F = F * self.shift_y
        return F * self.mask

    def inverse(self, F: np.ndarray) -> np.ndarray:
        """Spectral [ny, nx/2] -> real [ny, nx] (inverse DFT with 1/N)."""
        full = np.concatenate([F, np.zeros(F.shape[:-1] + (1,), complex)], axis=-1)
        return np.fft.irfft(np.fft.ifft(full, axis=-2), n=self.nx, axis=-1)


# ----------------------------------------------------------------------------------------
# Per-mode slice update, Sec. 4.1 Eqs. RxN, RyN, LxN, LyN, the B_z equation and eqall.
# Solved as a dense 6x6 complex system for (Rx0, Ry0, Lx0, Ly0, Bz0, Ez0) at level s^1.
# E_x = (R_x+L_x)/2, B_y = (R_x-L_x)/2, E_y = (R_y+L_y)/2, B_x = (L_y-R_y)/2 (Eqs. Rx-Ly).
# The R equations are multiplied through by Delta so that Delta = 0 gives R^1 = R^0.
# ----------------------------------------------------------------------------------------
RX, RY, LX, LY, BZ, EZ = range(6)


def slice_solve_dense(kx, ky, h, delta, new1, old0, j0m, j0p, j1m, j1p, jz1p):
    """Solve the slice system for every mode.

    kx, ky: wavenumbers broadcast to the mode shape; new1: dict of level-1 values at slice 1
    (keys Rx, Ry, Lx, Ly, Bz, Ez); old0: dict of level-0 values at slice 0 (Rx, Ry, Ez, Bz);
    j0m/j0p/j1m/j1p: (jx, jy) tuples of the level-0/1 currents at -1/2 and +1/2;
    jz1p: level-1 j_z at +1/2.  Returns the six unknowns, each of the mode shape.
    """
    shape = np.broadcast(kx, ky, new1["Rx"]).shape
    kx = np.broadcast_to(kx, shape).ravel()
    ky = np.broadcast_to(ky, shape).ravel()
    M = kx.size
    i = 1j
    A = np.zeros((M, 6, 6), complex)
    b = np.zeros((M, 6), complex)

    def f(x):
        return np.broadcast_to(x, shape).ravel()

    Rx1, Ry1, Lx1, Ly1 = f(new1["Rx"]), f(new1["Ry"]), f(new1["Lx"]), f(new1["Ly"])
    Bz1, Ez1 = f(new1["Bz"]), f(new1["Ez"])
    Rxo, Ryo, Ezo, Bzo = f(old0["Rx"]), f(old0["Ry"]), f(old0["Ez"]), f(old0["Bz"])
    jx0m, jy0m = f(j0m[0]), f(j0m[1])
    jx0p, jy0p = f(j0p[0]), f(j0p[1])
    jx1m, jy1m = f(j1m[0]), f(j1m[1])
    jx1p, jy1p = f(j1p[0]), f(j1p[1])
    jz1 = f(jz1p)

    # RxN * Delta: Rx0 - Delta/2 (i kx Ez0 + i ky Bz0) = Rxo + Delta/2 (i kx Ezo + i ky Bzo) - Delta Jx/4
    A[:, 0, RX] = 1.0
    A[:, 0, EZ] = -0.5 * delta * i * kx
    A[:, 0, BZ] = -0.5 * delta * i * ky
    b[:, 0] = Rxo + 0.5 * delta * (i * kx * Ezo + i * ky * Bzo) \
        - 0.25 * delta * (jx1m + jx0m + jx1p + jx0p)
    # RyN * Delta: Ry0 - Delta/2 (i ky Ez0 - i kx Bz0) = Ryo + Delta/2 (i ky Ezo - i kx Bzo) - Delta Jy/4
    A[:, 1, RY] = 1.0
    A[:, 1, EZ] = -0.5 * delta * i * ky
    A[:, 1, BZ] = +0.5 * delta * i * kx
    b[:, 1] = Ryo + 0.5 * delta * (i * ky * Ezo - i * kx * Bzo) \
        - 0.25 * delta * (jy1m + jy0m + jy1p + jy0p)
    # LxN: 2 (Lx1 - Lx0)/h = i kx (Ez1 + Ez0)/2 - i ky (Bz0 + Bz1)/2 + jx_{+1/2}
    A[:, 2, LX] = -2.0 / h
    A[:, 2, EZ] = -0.5 * i * kx
    A[:, 2, BZ] = +0.5 * i * ky
    b[:, 2] = -2.0 * Lx1 / h + 0.5 * i * kx * Ez1 - 0.5 * i * ky * Bz1 + jx1p
    # LyN (read with B_z0^1 + B_z1^1): 2 (Ly1 - Ly0)/h = i ky (Ez1 + Ez0)/2 + i kx (Bz0 + Bz1)/2 + jy_{+1/2}
    A[:, 3, LY] = -2.0 / h
    A[:, 3, EZ] = -0.5 * i * ky
    A[:, 3, BZ] = -0.5 * i * kx
    b[:, 3] = -2.0 * Ly1 / h + 0.5 * i * ky * Ez1 + 0.5 * i * kx * Bz1 + jy1p
    # B_z: (Bz1 - Bz0)/h = i kx (Ey0 + Ey1)/2 - i ky (Ex0 + Ex1)/2
    A[:, 4, BZ] = -1.0 / h
    A[:, 4, RY] = -0.25 * i * kx
    A[:, 4, LY] = -0.25 * i * kx
    A[:, 4, RX] = +0.25 * i * ky
    A[:, 4, LX] = +0.25 * i * ky
    b[:, 4] = -Bz1 / h + 0.25 * i * kx * (Ry1 + Ly1) - 0.25 * i * ky * (Rx1 + Lx1)
    # eqall (read with +i ky): (Ez1 - Ez0)/h = -i kx (By0 + By1)/2 + i ky (Bx0 + Bx1)/2 + jz_{+1/2}
    A[:, 5, EZ] = -1.0 / h
    A[:, 5, RX] = +0.25 * i * kx
    A[:, 5, LX] = -0.25 * i * kx
    A[:, 5, LY] = -0.25 * i * ky
    A[:, 5, RY] = +0.25 * i * ky
    b[:, 5] = -Ez1 / h - 0.25 * i * kx * (Rx1 - Lx1) + 0.25 * i * ky * (Ly1 - Ry1) + jz1

    x = np.linalg.solve(A, b[..., None])[..., 0]
    return {k: x[:, idx].reshape(shape) for k, idx in
            (("Rx", RX), ("Ry", RY), ("Lx", LX), ("Ly", LY), ("Bz", BZ), ("Ez", EZ))}


def fields_from_characteristics(s):
    """E and B from R, L, E_z, B_z (Eqs. Rx, Ry, Lx, Ly)."""
    return {"Ex": 0.5 * (s["Rx"] + s["Lx"]), "Ey": 0.5 * (s["Ry"] + s["Ly"]), "Ez": s["Ez"],
            "Bx": 0.5 * (s["Ly"] - s["Ry"]), "By": 0.5 * (s["Rx"] - s["Lx"]), "Bz": s["Bz"]}


FIELD_NAMES = ("Ex", "Ey", "Ez", "Bx", "By", "Bz")


# ----------------------------------------------------------------------------------------
# Particle dynamics.  du/dt = (q/m)(E + u x B / gamma) (Sec. 3, normalised Vlasov force).
# ----------------------------------------------------------------------------------------
def gamma_of(u):
    return np.sqrt(1.0 + u[0] ** 2 + u[1] ** 2 + u[2] ** 2)


def gamma_minus_uz(u, g):
    """gamma - u_z, written as (1 + u_perp^2)/(gamma + u_z) where u_z > 0 (same quantity)."""
    perp = 1.0 + u[0] ** 2 + u[1] ** 2
    return np.where(u[2] > 0.0, perp / (g + np.maximum(u[2], 0.0)), g - u[2])


def boris(u, E, B, qm, dt):
    """Relativistic Boris rotation of u over lab time dt (arrays [3, N])."""
    a = 0.5 * qm * dt
    um = u + a * E
    gm = np.sqrt(1.0 + (um ** 2).sum(0))
    t = a * B / gm
    up = um + np.cross(um, t, axis=0)
    s = 2.0 * t / (1.0 + (t ** 2).sum(0))
    upl = um + np.cross(up, s, axis=0)
    return upl + a * E


def zeta_push(u, E, B, qm, hc):
    """One step of length hc along -zeta (GT2 characteristics, Eq. after Vlasov2):
    dp/dzeta = F/(v_z - 1), dr/dzeta = v_perp/(v_z - 1), ds~/dzeta = v_z/(v_z - 1).
    Lab time of the step dt = hc gamma/(gamma - u_z); two passes evaluate it at the step's
    mean momentum.  Returns (u_new, dx, dy, ds~)."""
    g0 = gamma_of(u)
    dt1 = hc * g0 / gamma_minus_uz(u, g0)
    us = boris(u, E, B, qm, dt1)
    ub = 0.5 * (u + us)
    gb = gamma_of(ub)
    dt2 = hc * gb / gamma_minus_uz(ub, gb)
    un = boris(u, E, B, qm, dt2)
    gn = gamma_of(un)
    den = gamma_minus_uz(un, gn)
    return un, hc * un[0] / den, hc * un[1] / den, hc * un[2] / den


# ----------------------------------------------------------------------------------------
# Shapes: cloud-in-cell on the transverse nodes x_i = i hx (periodic).
# ----------------------------------------------------------------------------------------
def cic_gather(F, X, Y):
    """Interpolate node values F [ny, nx] at positions X, Y in cell units."""
    ny, nx = F.shape
    i0 = np.floor(X)
    fx = X - i0
    i0 = i0.astype(np.int64)
    if ny == 1:
        return (1.0 - fx) * F[0, i0 % nx] + fx * F[0, (i0 + 1) % nx]
    j0 = np.floor(Y)
    fy = Y - j0
    j0 = j0.astype(np.int64)
    out = np.zeros_like(X)
    for dj, wy in ((0, 1.0 - fy), (1, fy)):
        for di, wx in ((0, 1.0 - fx), (1, fx)):
            out += wx * wy * F[(j0 + dj) % ny, (i0 + di) % nx]
    return out


def _shape3(Xp, base):
    """CIC weights of position Xp on the three nodes base, base+1, base+2."""
    return [np.maximum(0.0, 1.0 - np.abs(Xp - (base + a))) for a in range(3)]


def _scatter(plane, jj, ii, val):
    ny, nx = plane.shape
    idx = (jj % ny) * nx + (ii % nx)
    plane += np.bincount(idx.ravel(), weights=val.ravel(), minlength=nx * ny).reshape(ny, nx)


def esirkepov_deposit(jx, jy, X0, Y0, X1, Y1, w, h, hx, hy, dy_out=None):
    """Charge-conserving transverse current of moves (X0,Y0) -> (X1,Y1) (cell units).

    2-D Esirkepov (Esirkepov, Comput. Phys. Commun. 135 (2001) 144) with CIC shapes:
    W_x = (S1x - S0x)(S0y + S1y)/2, W_y = (S1y - S0y)(S0x + S1x)/2 and
    J_x(a + 1/2) = J_x(a - 1/2) - (w hx / h) W_x(a), so that (D_new - D_old) + h div J = 0
    with D = w S.  jx is stored on x-edges (index i <-> x = (i + 1/2) hx), jy on y-edges in
    3-D.  In 2-D (ny == 1) the y-current is out of plane: w (dy/h) (S0x + S1x)/2 on the nodes,
    dy_out being the particle's y displacement.  Moves longer than one cell are split into
    equal sub-moves.
    """
    ny, nx = jx.shape
    dX = X1 - X0
    dY = Y1 - Y0 if ny > 1 else np.zeros_like(dX)
    nsub = np.maximum(1, np.ceil(np.maximum(np.abs(dX), np.abs(dY)))).astype(np.int64)
    for ns in np.unique(nsub):
        sel = nsub == ns
        for s in range(ns):
            xa = X0[sel] + dX[sel] * (s / ns)
            xb = X0[sel] + dX[sel] * ((s + 1) / ns)
            wsel = w[sel]
            bx = np.floor(np.minimum(xa, xb))
            S0x, S1x = _shape3(xa, bx), _shape3(xb, bx)
            ibx = bx.astype(np.int64)
            if ny == 1:
                cum = np.zeros_like(xa)
                for a in range(2):
                    cum = cum + (S1x[a] - S0x[a])
                    _scatter(jx, np.zeros_like(ibx), ibx + a, -(wsel * hx / h) * cum)
                if dy_out is not None:
                    dyv = dy_out[sel] / ns
                    for a in range(3):
                        _scatter(jy, np.zeros_like(ibx), ibx + a,
                                 wsel * (dyv / h) * 0.5 * (S0x[a] + S1x[a]))
                continue
            ya = Y0[sel] + dY[sel] * (s / ns)
            yb = Y0[sel] + dY[sel] * ((s + 1) / ns)
            by = np.floor(np.minimum(ya, yb))
            S0y, S1y = _shape3(ya, by), _shape3(yb, by)
            iby = by.astype(np.int64)
            for b in range(3):
                cum = np.zeros_like(xa)
                for a in range(2):
                    cum = cum + (S1x[a] - S0x[a]) * 0.5 * (S0y[b] + S1y[b])
                    _scatter(jx, iby + b, ibx + a, -(wsel * hx / h) * cum)
            for a in range(3):
                cum = np.zeros_like(xa)
                for b in range(2):
                    cum = cum + (S1y[b] - S0y[b]) * 0.5 * (S0x[a] + S1x[a])
                    _scatter(jy, iby + b, ibx + a, -(wsel * hy / h) * cum)


def cic_deposit(plane, X, Y, val):
    """Deposit val on the nodes of plane with CIC weights at (X, Y) (cell units)."""
    ny, nx = plane.shape
    i0 = np.floor(X)
    fx = X - i0
    i0 = i0.astype(np.int64)
    if ny == 1:
        _scatter(plane, np.zeros_like(i0), i0, (1.0 - fx) * val)
        _scatter(plane, np.zeros_like(i0), i0 + 1, fx * val)
        return
    j0 = np.floor(Y)
    fy = Y - j0
    j0 = j0.astype(np.int64)
    for dj, wy in ((0, 1.0 - fy), (1, fy)):
        for di, wx in ((0, 1.0 - fx), (1, fx)):
            _scatter(plane, j0 + dj, i0 + di, wx * wy * val)


# ----------------------------------------------------------------------------------------
# Gauss's law on a slice plane (a diagnostic: the scheme does not conserve it while
# dR/ds != 0).  With d E_z/d zeta taken from Eq. EzGu, div E - rho = d_x L_x + d_y L_y -
# (rho - j_z), L_x = E_x - B_y, L_y = E_y + B_x (Eqs. Lx, Ly).
# ----------------------------------------------------------------------------------------
def gauss_residual(F, D, hx, hy):
    """max over the nodes of |d_x L_x + d_y L_y - D| for the real-space fields F [6, ny, nx]
    (E_x, E_y, E_z, B_x, B_y, B_z) of one plane and its (rho - j_z) density D [ny, nx];
    central differences across (periodic), no y-derivative in 2-D (ny == 1)."""
    Lx = F[0] - F[4]
    div = (np.roll(Lx, -1, axis=1) - np.roll(Lx, 1, axis=1)) / (2.0 * hx)
    if F.shape[1] > 1:
        Ly = F[1] + F[3]
        div = div + (np.roll(Ly, -1, axis=0) - np.roll(Ly, 1, axis=0)) / (2.0 * hy)
    return float(np.abs(div - D).max())


# ----------------------------------------------------------------------------------------
# Plasma channel, Sec. 6 Eq. n_plasma.
# ----------------------------------------------------------------------------------------
def channel_profile(ch, dx, dy):
    """n(r_perp) / n0 of the Gaussian channel: n = n0 [1 + (n1 - n0)/n0 exp(-r^2/R_ch^2)],
    with r^2 = dx^2 + dy^2 measured from the channel axis; ch.n1_over_n0 = n1/n0,
    ch.radius = R_ch."""
    n0 = 1.0
    n1 = ch.n1_over_n0 * n0
    r2 = np.asarray(dx) ** 2 + np.asarray(dy) ** 2
    return (n0 * (1.0 + (n1 - n0) / n0 * np.exp(-r2 / ch.radius ** 2))) / n0


# ----------------------------------------------------------------------------------------
# The simulation.
# ----------------------------------------------------------------------------------------
@dataclass
class Particles:
    """Particle set: absolute transverse position (x, y), zeta, momentum u [3, N], s~ budget
    used in this s-step (sigma), charge Q, species index.  For streaming particles `dist` is
    the zeta distance to the next slice plane (h, or less for a particle that rejoins)."""
    x: np.ndarray
    y: np.ndarray
    zeta: np.ndarray
    u: np.ndarray
    sigma: np.ndarray
    Q: np.ndarray
    sp: np.ndarray
    dist: np.ndarray

    @staticmethod
    def empty():
        z = np.zeros(0)
        return Particles(z, z.copy(), z.copy(), np.zeros((3, 0)), z.copy(), z.copy(),
                         np.zeros(0, np.int64), z.copy())

    @property
    def n(self):
        return self.x.size

    def select(self, m):
        return Particles(self.x[m], self.y[m], self.zeta[m], self.u[:, m], self.sigma[m],
                         self.Q[m], self.sp[m], self.dist[m])

    @staticmethod
    def concat(parts):
        parts = [p for p in parts if p.n > 0]
        if not parts:
            return Particles.empty()
        return Particles(*(np.concatenate([getattr(p, f) for p in parts], axis=-1)
                           for f in ("x", "y", "zeta", "u", "sigma", "Q", "sp", "dist")))


class RefSim:
    """FP64 GEM-PIC, GT2 particle law, universal reduced Maxwell system (Secs. 3-4).

    State between s-steps (what the scheme needs at s^0, Sec. 4.1): spectral R_x, R_y, E_z,
    B_z on the slices zeta_n = n h (n = 0..N-1) and j_x, j_y on the half-slices
    zeta_{n+1/2} (index n), plus the stored (trapped / beam) particles and the real-space
    fields of the last level (they push the stored particles).
    """

    def __init__(self, w):
        self.w = w
        self.nx, self.ny, self.nz = w.nx, w.ny, w.nzeta
        self.hx, self.hy, self.h = w.hx, w.hy, w.h
        self.delta = w.delta
        # zeta grid: slab n between planes n and n+1 has thickness hz[n]; plane n sits at
        # zp[n] (plane 0 at the back).  Uniform: hz = h.  Variable (Sec. 6 refines the back
        # of the window): every use of h below takes the thickness of the slab it concerns.
        self.varh = w.hz is not None
        if self.varh:
            self.hz = np.asarray(w.hz, dtype=float)
            if self.hz.shape != (self.nz,) or not np.all(self.hz > 0) or not np.all(np.isfinite(self.hz)):
                raise ValueError("hz holds nzeta positive slab thicknesses")
            self.zp = np.concatenate([[0.0], np.cumsum(self.hz)])
        else:
            self.hz = np.full(self.nz, self.h)
            self.zp = np.arange(self.nz + 1) * self.h
        if w.particle_law not in ("GT1", "GT2"):
            raise ValueError("particle_law is GT1 or GT2 (Sec. 5)")
        self.gt1 = w.particle_law == "GT1"
        # Delta of the next advance of the stored set: that of the last completed s-step
        # (the level-0 set-up counts as one, with the Delta of creation)
        self.delta_stored = self.delta
        self.sp = Spectral(self.nx, self.ny, self.hx, self.hy)
        self.KX = self.sp.kx[None, :]
        self.KY = self.sp.ky[:, None]
        shp = (self.nz, self.ny, self.nx // 2)
        self.S = {k: np.zeros(shp, complex) for k in ("Rx", "Ry", "Ez", "Bz", "jx", "jy")}
        self.fields_rs = np.zeros((self.nz, 6, self.ny, self.nx))
        self.step_index = 0
        self.diag: Dict = {}
        densest = max(1.0, w.channel.n1_over_n0) if w.channel is not None else 1.0
        if w.omega_p2 * densest * self.delta * self.hz.max() > 4.0 * (1.0 + 1e-12):
            raise ValueError("Delta h omega_p^2 > 4: outside the stability bound (Sec. 4.2)")
        # species of the particles: the injected ones, then a slot of the bunch's own if no
        # injected species has its charge and mass
        self.species = list(w.species)
        self.beam_species = None
        if w.beam is not None:
            b = w.beam
            for si, s in enumerate(w.species):
                if s.charge == b.charge and s.mass == b.mass:
                    self.beam_species = si
                    break
            if self.beam_species is None:
                self.beam_species = len(self.species)
                self.species.append(type("BeamSpecies", (), dict(charge=b.charge, mass=b.mass))())
        # neutralising background of the injected species (immobile ions): -sum_s q_s n_s f(r)
        # on the nodes, f the channel profile; it carries no current
        qn = sum(s.charge * s.density for s in w.species)
        xi = np.arange(self.nx) * self.hx - 0.5 * self.nx * self.hx
        yj = (np.arange(self.ny) * self.hy - 0.5 * self.ny * self.hy) if self.ny > 1 else np.zeros(1)
        prof = (channel_profile(w.channel, xi[None, :], yj[:, None]) if w.channel is not None
                else np.ones((self.ny, self.nx)))
        self.rho_bg = -qn * prof
        self.stored = Particles.empty()
        if w.stored is not None and w.stored.n > 0:
            st = w.stored
            self.stored = Particles(st.x.astype(float).copy(), st.y.astype(float).copy(),
                                    st.zeta.astype(float).copy(),
                                    np.stack([st.ux, st.uy, st.uz]).astype(float),
                                    np.zeros(st.n), st.weight.astype(float).copy(),
                                    st.species.astype(np.int64).copy(), np.zeros(st.n))
        if w.beam is not None and w.beam.n_macro > 0:
            bx, by, bz, bu, bq = sample_beam(w.beam, self.nx, self.ny, self.hx, self.hy,
                                             self.zp[self.nz])
            nb = bx.size
            self.stored = Particles.concat([self.stored, Particles(
                bx, by, bz, bu, np.zeros(nb), bq, np.full(nb, self.beam_species, np.int64),
                np.zeros(nb))])
        self._init_laser()
        # Delta = 0 consistency march (R^1 = R^0 exactly): fills E_z, B_z (and L) for the
        # initial laser and the real-space fields of level 0.
        self._march(delta_field=0.0, inject=False, joiners=Particles.empty(),
                    jbeam=self._zero_jbeam())

    def set_delta(self, delta):
        """Sec. 6: Delta may change along the run.  The s-steps after this call use the new
        Delta in the slice update (Sec. 4.1), the fresh weight Q_f (Sec. 5.1) and the
        particles' s-budget (Sec. 5); stored particles keep their charge.  The stored set is
        advanced to the next level with the Delta of the s-step that produced the fields it
        uses (the previous one), so after a change it lags the new Delta by one s-step."""
        densest = max(1.0, self.w.channel.n1_over_n0) if self.w.channel is not None else 1.0
        if not (delta >= 0.0) or not math.isfinite(delta):
            raise ValueError("Delta must be finite and >= 0")
        if self.w.omega_p2 * densest * delta * self.hz.max() > 4.0 * (1.0 + 1e-12):
            raise ValueError("Delta h omega_p^2 > 4: outside the stability bound (Sec. 4.2)")
        self.delta = float(delta)

    # -- initial condition: forward wave R = 2E, L = 0 (Eqs. Rx/Ry, E_laser) ------------------
    def _init_laser(self):
        L = self.w.laser
        if L is None:
            return
        xi = np.arange(self.nx) * self.hx - 0.5 * self.nx * self.hx
        yj = (np.arange(self.ny) * self.hy - 0.5 * self.ny * self.hy) if self.ny > 1 else np.zeros(1)
        r2 = yj[:, None] ** 2 + xi[None, :] ** 2
        comp = "Rx" if L.pol == 0 else "Ry"
        for n in range(self.nz):
            phi = self.zp[n] - L.zeta_center
            E = L.a0 * math.cos(phi) * math.exp(-phi * phi / L.duration ** 2) * np.exp(-r2 / L.waist ** 2)
            self.S[comp][n] = self.sp.forward(2.0 * E)

    def _slab(self, zeta):
        """Slab m with zp[m] < zeta <= zp[m+1] and the offset (zeta - zp[m]) / hz[m]."""
        if self.varh:
            m = np.searchsorted(self.zp, zeta, side="left").astype(np.int64) - 1
            mc = np.clip(m, 0, self.nz - 1)
            return m, (zeta - self.zp[mc]) / self.hz[mc]
        m = np.ceil(zeta / self.h).astype(np.int64) - 1
        return m, zeta / self.h - m

    def _zero_jbeam(self):
        return np.zeros((self.nz, 3, self.ny, self.nx))

    # -- fresh particles at the front ghost slice (Sec. 5.1, Q_f = q n hx hy Delta) -----------
    def _inject(self):
        w = self.w
        ncell = self.nx * self.ny
        nlayer = sum(s.ppc for s in w.species) * ncell
        parts = []
        off = 0
        for si, s in enumerate(w.species):
            cell = np.repeat(np.arange(ncell), s.ppc)
            k = np.tile(np.arange(s.ppc), ncell)
            g = off + cell * s.ppc + k
            c = (np.uint64(self.step_index) * np.uint64(nlayer) + g.astype(np.uint64)) * np.uint64(2)
            ox = uniform24(w.seed, c)
            oy = uniform24(w.seed, c + np.uint64(1))
            i = cell % self.nx
            j = cell // self.nx
            x = (i + ox) * self.hx
            y = (j + oy) * self.hy if self.ny > 1 else np.zeros(cell.size)
            n = cell.size
            Q = s.charge * s.density * self.hx * self.hy * self.delta / s.ppc
            if w.channel is not None:
                Q = Q * channel_profile(w.channel, x - 0.5 * self.nx * self.hx,
                                        y - 0.5 * self.ny * self.hy if self.ny > 1 else y)
            parts.append(Particles(x, y, np.full(n, self.zp[self.nz]), np.zeros((3, n)),
                                   np.zeros(n), np.broadcast_to(Q, (n,)).copy(),
                                   np.full(n, si, np.int64),
                                   np.full(n, self.hz[self.nz - 1])))
            off += ncell * s.ppc
        return Particles.concat(parts)

    def _qm(self, sp):
        return np.array([s.charge / s.mass for s in self.species])[sp]

    def _mass(self, sp):
        return np.array([s.mass for s in self.species])[sp]

    def _charge(self, sp):
        return np.array([s.charge for s in self.species])[sp]

    # -- stored set along s (Sec. 5.1, last paragraph) --------------------------------------
    def _gather_stored(self, x, y, zeta):
        """E, B [6, N] at the absolute positions (x, y, zeta) from the real-space fields of the
        last completed level: CIC across, linear in zeta between the slices m and m + 1 of the
        slab holding zeta (the ghost slice in front of the window is field-free)."""
        m, fz = self._slab(zeta)
        X, Y = x / self.hx, y / self.hy
        Efld = np.zeros((6, x.size))
        for c in range(6):
            lo = np.zeros(x.size)
            hi = np.zeros(x.size)
            for mm in np.unique(m):
                sel = m == mm
                lo[sel] = cic_gather(self.fields_rs[mm, c], X[sel], Y[sel])
                if mm + 1 < self.nz:
                    hi[sel] = cic_gather(self.fields_rs[mm + 1, c], X[sel], Y[sel])
            Efld[c] = (1.0 - fz) * lo + fz * hi
        return Efld

    def _beam_cells(self, zeta):
        """Half-slices receiving the beam current of a particle at zeta (Sec. 5.1, j = Q v/
        (hx hy h)): i0 with weight 1 - f and i0 + 1 with weight f, linear between the
        half-slice centres zeta_{i+1/2} = zp[i] + hz[i]/2 (the grid extended by one slab of
        the end thickness on either side)."""
        if self.varh:
            c = np.concatenate([[-0.5 * self.hz[0]], self.zp[:-1] + 0.5 * self.hz,
                                [self.zp[-1] + 0.5 * self.hz[-1]]])
            k = np.searchsorted(c, zeta, side="right") - 1   # c[k] <= zeta < c[k+1]
            return k - 1, (zeta - c[k]) / (c[k + 1] - c[k])
        t = zeta / self.h - 0.5
        i0 = np.floor(t).astype(np.int64)
        return i0, t - i0

    def _stored_push(self):
        """Advance the stored particles from s^k to s^{k+1} with the fields of level k.
        Returns (particles that rejoin the zeta march, beam current j^{k+1} on half-slices)."""
        jbeam = self._zero_jbeam()
        P = self.stored
        nremoved = 0
        if P.n == 0:
            return Particles.empty(), jbeam, 0
        D = self.delta_stored
        ms, _ = self._slab(P.zeta)
        h = self.hz[np.clip(ms, 0, self.nz - 1)]        # thickness of each particle's slab
        g = gamma_of(P.u)
        gmu = gamma_minus_uz(P.u, g)
        if self.gt1:
            # GT1: one s-step is the lab time Delta; the particle stays stored while it moves
            # less than one cell along zeta in it, Delta (1 - v_z) < h
            spush = D * gmu < h * g
        else:
            spush = (P.u[2] > 0.0) & (D * gmu < h * np.maximum(P.u[2], 0.0))
        # rejoiners: their zeta march starts at their position, budget 0, first step to the
        # plane below them.
        R = P.select(~spush)
        m, _ = self._slab(R.zeta)
        R.dist = R.zeta - (self.zp[m] if self.varh else m * self.h)
        R.sigma = np.zeros(R.n)
        S = P.select(spush)
        Efld = self._gather_stored(S.x, S.y, S.zeta)
        u = S.u
        g = gamma_of(u)
        if self.gt1:
            # GT1: dt = Delta; r_perp += Delta v_perp, zeta += Delta (v_z - 1)
            un = boris(u, Efld[:3], Efld[3:], self._qm(S.sp), D)
            gn = gamma_of(un)
            fwd = np.ones(S.n, bool)
            S.u = un
            S.x = (S.x + D * un[0] / gn) % (self.nx * self.hx)
            if self.ny > 1:
                S.y = (S.y + D * un[1] / gn) % (self.ny * self.hy)
            S.zeta = S.zeta - D * gamma_minus_uz(un, gn) / gn
        else:
            # GT2: the s-step is the propagation distance Delta, dt = Delta / v_z
            dt = D * g / u[2]
            un = boris(u, Efld[:3], Efld[3:], self._qm(S.sp), dt)
            gn = gamma_of(un)
            fwd = un[2] > 0.0
            safe_uz = np.where(fwd, un[2], 1.0)
            S.u = un
            S.x = np.where(fwd, (S.x + D * un[0] / safe_uz) % (self.nx * self.hx), S.x)
            if self.ny > 1:
                S.y = np.where(fwd, (S.y + D * un[1] / safe_uz) % (self.ny * self.hy), S.y)
            S.zeta = np.where(fwd, S.zeta - D * gamma_minus_uz(un, gn) / safe_uz, S.zeta)
        keep = S.zeta > 0.0
        nremoved = int((~keep).sum())
        S = S.select(keep)
        fwd = fwd[keep]
        gn = gn[keep]
        # beam current j = Q v / (hx hy h) on half-slice nodes (Sec. 5.1, j = q n v)
        if S.n:
            D3 = S.select(fwd)
            gd = gn[fwd]
            i0, f = self._beam_cells(D3.zeta)
            if self.varh:
                # the density of half-slice i is charge / (hx hy hz[i]) (the grid extended by
                # one slab of the end thickness on either side)
                hpad = np.concatenate([[self.hz[0]], self.hz, [self.hz[-1]]])
                amp = D3.Q / (self.hx * self.hy * gd)
                inv_h = lambda ii: 1.0 / hpad[np.clip(ii + 1, 0, self.nz + 1)]
            else:
                amp = D3.Q / (self.hx * self.hy * self.h * gd)
                inv_h = lambda ii: 1.0
            X, Y = D3.x / self.hx, D3.y / self.hy
            for ii, wz in ((i0, 1.0 - f), (i0 + 1, f)):
                ok = (ii >= 0) & (ii < self.nz)
                for iz in np.unique(ii[ok]):
                    sel = ok & (ii == iz)
                    a = amp[sel] * wz[sel] * inv_h(iz)
                    cic_deposit(jbeam[iz, 0], X[sel] - 0.5, Y[sel], a * D3.u[0, sel])
                    if self.ny > 1:
                        cic_deposit(jbeam[iz, 1], X[sel], Y[sel] - 0.5, a * D3.u[1, sel])
                    else:
                        cic_deposit(jbeam[iz, 1], X[sel], Y[sel], a * D3.u[1, sel])
                    cic_deposit(jbeam[iz, 2], X[sel], Y[sel], a * D3.u[2, sel])
        self.stored = S
        return R, jbeam, nremoved

    # -- the zeta march at level s^1 (Sec. 4.1: from the front of the window towards the back) -------
    def _march(self, delta_field, inject, joiners, jbeam, current_hook=None):
        nx, ny, nz = self.nx, self.ny, self.nz
        old = {k: v.copy() for k, v in self.S.items()}
        D = self.delta
        zero = np.zeros((ny, nx // 2), complex)
        new1 = {k: zero for k in ("Rx", "Ry", "Lx", "Ly", "Bz", "Ez")}   # ghost slice
        F1 = np.zeros((6, ny, nx))
        jprev = None
        P = self._inject() if inject else Particles.empty()
        trapped: List[Particles] = []
        field_energy = 0.0
        kinetic = 0.0
        charge_flux = 0.0
        continuity = 0.0          # max over slabs and nodes of the discrete continuity residual
        gauss = 0.0               # max over slices and nodes of the Gauss residual
        onaxis = np.zeros(nz)
        if joiners.n:
            jm, _ = self._slab(joiners.zeta)
        for n in range(nz - 1, -1, -1):
            h = self.hz[n]                                  # slab n: planes n and n+1
            if joiners.n:
                P = Particles.concat([P, joiners.select(jm == n)])
            jx = np.zeros((ny, nx))
            jy = np.zeros((ny, nx))
            jz = np.zeros((ny, nx))
            Dn = np.zeros((ny, nx))
            if P.n:
                X0, Y0 = P.x / self.hx, P.y / self.hy
                E = np.stack([cic_gather(F1[c], X0, Y0) for c in range(3)])
                B = np.stack([cic_gather(F1[c], X0, Y0) for c in range(3, 6)])
                g = gamma_of(P.u)
                gmu = gamma_minus_uz(P.u, g)
                uzp = np.maximum(P.u[2], 0.0)
                if self.gt1:
                    # Eq. trap1: s = ct advances by the lab time |dzeta|/(1 - v_z); the step
                    # is min(d, (Delta - sigma)(1 - v_z)), 1 - v_z = (gamma - u_z)/gamma
                    hlim = (D - P.sigma) * gmu / g
                else:
                    # Eq. trap2: the step is min(d, (Delta - sigma)(1 - v_z)/v_z) for v_z > 0
                    hlim = np.where(P.u[2] > 0.0, (D - P.sigma) * gmu / np.where(uzp > 0, uzp, 1.0), np.inf)
                hlim = np.maximum(hlim, 0.0)
                trap = hlim < P.dist
                hc = np.where(trap, hlim, P.dist)
                un, dx, dy, ds = zeta_push(P.u, E, B, self._qm(P.sp), hc)
                wgt = P.Q / (self.hx * self.hy * D)            # D-weight q n / ppc of Sec. 5.1
                X1 = X0 + dx / self.hx
                Y1 = Y0 + dy / self.hy if ny > 1 else Y0
                esirkepov_deposit(jx, jy, X0, Y0, X1, Y1, wgt, h, self.hx, self.hy,
                                  dy_out=dy if ny == 1 else None)
                cic_deposit(jz, X1, Y1, wgt * ds / h)
                reach = ~trap
                cic_deposit(Dn, X1[reach], Y1[reach], wgt[reach])
                # discrete continuity of this slab's deposit (Sec. 5.1; rho - j_z conserved
                # through the planes): (D(start) - D(end))/h = div j_perp on every node, with D
                # the CIC density of w at the start and end of each particle's move
                Dd = np.zeros((ny, nx))
                cic_deposit(Dd, X0, Y0, wgt)
                cic_deposit(Dd, X1 % nx, (Y1 % ny) if ny > 1 else Y1, -wgt)
                div = (jx - np.roll(jx, 1, axis=1)) / self.hx
                if ny > 1:
                    div = div + (jy - np.roll(jy, 1, axis=0)) / self.hy
                continuity = max(continuity, float(np.abs(Dd / h - div).max()))
                gn = gamma_of(un)
                dtl = hc * gn / gamma_minus_uz(un, gn)
                kinetic += float(np.sum((P.Q / self._charge(P.sp)) * self._mass(P.sp) * (gn - 1.0) * dtl / D))
                charge_flux += float(np.sum(wgt[reach])) * self.hx * self.hy * h
                P.u = un
                P.x = (X1 * self.hx) % (nx * self.hx)
                if ny > 1:
                    P.y = (Y1 * self.hy) % (ny * self.hy)
                # the s-budget: s~ = z under GT2 (ds~ = v_z dt), s = ct under GT1 (ds = dt)
                P.sigma = P.sigma + (dtl if self.gt1 else ds)
                P.zeta = self.zp[n] + (P.dist - hc) if self.varh else n * h + (P.dist - hc)
                if trap.any():
                    T = P.select(trap)
                    trapped.append(T)
                P = P.select(~trap)
                P.dist = np.full(P.n, self.hz[n - 1] if n > 0 else h)
                P.zeta = np.full(P.n, self.zp[n] if self.varh else n * h)
            jx += jbeam[n, 0]
            jy += jbeam[n, 1]
            jz += jbeam[n, 2]
            if current_hook is not None:            # record or replace the half-slice's current
                jx, jy, jz = current_hook(n, jx, jy, jz)
            # transform the currents at the half-slice n + 1/2
            Jx = self.sp.forward(jx, "x")
            Jy = self.sp.forward(jy, "y" if ny > 1 else "")
            Jz = self.sp.forward(jz)
            # corrector: R of slice n+1 was built with j_{n+1/2} := j_{n+3/2}
            if n + 1 < nz:
                new1 = dict(new1)
                new1["Rx"] = new1["Rx"] - 0.25 * delta_field * (Jx - jprev[0])
                new1["Ry"] = new1["Ry"] - 0.25 * delta_field * (Jy - jprev[1])
                self.S["Rx"][n + 1] = new1["Rx"]
                self.S["Ry"][n + 1] = new1["Ry"]
            o0 = {k: old[k][n] for k in ("Rx", "Ry", "Ez", "Bz")}
            j0p = (old["jx"][n], old["jy"][n])
            j0m = (old["jx"][n - 1], old["jy"][n - 1]) if n > 0 else j0p
            j1p = (Jx, Jy)
            j1m = j1p                                               # predictor
            sol = slice_solve_dense(self.KX, self.KY, h, delta_field, new1, o0, j0m, j0p, j1m, j1p, Jz)
            sol = {k: v * self.sp.mask for k, v in sol.items()}
            self.S["Rx"][n], self.S["Ry"][n] = sol["Rx"], sol["Ry"]
            self.S["Ez"][n], self.S["Bz"][n] = sol["Ez"], sol["Bz"]
            self.S["jx"][n], self.S["jy"][n] = Jx, Jy
            fl = fields_from_characteristics(sol)
            F0 = np.stack([self.sp.inverse(fl[name]) for name in FIELD_NAMES])
            self.fields_rs[n] = F0
            # Gauss's law on plane n (not conserved by the scheme while dR/ds != 0): with
            # d E_z/d zeta from Eq. EzGu, div E - rho = d_x L_x + d_y L_y - (rho - j_z),
            # L_x = E_x - B_y, L_y = E_y + B_x; central differences across; rho - j_z is the
            # CIC density of the particles reaching plane n plus the neutralising background
            gauss = max(gauss, gauss_residual(F0, Dn + self.rho_bg, self.hx, self.hy))
            field_energy += 0.5 * float(np.sum(F0 ** 2)) * self.hx * self.hy * h
            onaxis[n] = F0[2, ny // 2, nx // 2]
            new1 = sol
            F1 = F0
            jprev = (Jx, Jy)
        # particles that reached the back plane leave the box (Sec. 5, left boundary)
        T = Particles.concat(trapped)
        self.stored = Particles.concat([self.stored, T])
        stored_ke = 0.0
        if self.stored.n:
            g = gamma_of(self.stored.u)
            stored_ke = float(np.sum((self.stored.Q / self._charge(self.stored.sp))
                                     * self._mass(self.stored.sp) * (g - 1.0)))
        return dict(field_energy=field_energy, kinetic_energy=kinetic + stored_ke,
                    stored_kinetic_energy=stored_ke,
                    charge_flux=charge_flux, continuity_residual=continuity,
                    gauss_residual=gauss,
                    onaxis_ez=onaxis, n_trapped=T.n,
                    n_stored=self.stored.n)

    # -- one s-step ---------------------------------------------------------------------
    def step(self, n: int = 1):
        for _ in range(n):
            joiners, jbeam, nrem = self._stored_push()
            d = self._march(delta_field=self.delta, inject=True, joiners=joiners, jbeam=jbeam)
            self.delta_stored = self.delta
            d["n_rejoined"] = joiners.n
            d["n_stored_removed"] = nrem
            self.step_index += 1
            d["step"] = self.step_index
            self.diag = d
        return self.diag

    # -- one s-step with a current denoiser (two passes) --------------------------------------
    def step_denoised(self, denoise):
        """The denoised s-step of the library: the first pass marches the particles with the
        plain deposit and records the current J [nz, 3, ny, nx] of every half-slice; the
        second recomputes the level from the unchanged old one with denoise(J) in place of the
        deposit (no particles), so the stored set is pushed at the next s-step with its
        fields.  Diagnostics: fields and stored set from the second pass, the streaming
        particles from the first."""
        joiners, jbeam, nrem = self._stored_push()
        old = {k: v.copy() for k, v in self.S.items()}
        J = np.zeros((self.nz, 3, self.ny, self.nx))

        def record(n, jx, jy, jz):
            J[n, 0], J[n, 1], J[n, 2] = jx, jy, jz
            return jx, jy, jz
        d1 = self._march(delta_field=self.delta, inject=True, joiners=joiners, jbeam=jbeam,
                         current_hook=record)
        self.S = old
        Jd = denoise(J)

        def replace(n, jx, jy, jz):
            return Jd[n, 0].copy(), Jd[n, 1].copy(), Jd[n, 2].copy()
        d3 = self._march(delta_field=self.delta, inject=False, joiners=Particles.empty(),
                         jbeam=self._zero_jbeam(), current_hook=replace)
        self.delta_stored = self.delta
        d = dict(d3)
        for key in ("kinetic_energy", "charge_flux", "n_trapped", "continuity_residual"):
            d[key] = d1[key]
        d["n_rejoined"] = joiners.n
        d["n_stored_removed"] = nrem
        self.step_index += 1
        d["step"] = self.step_index
        d["current"] = J
        self.diag = d
        return d

    # -- exports in the canonical layout used for comparisons ---------------------------------
    def state(self) -> np.ndarray:
        """Spectral state [6, nzeta, ny, nx/2] complex: Rx, Ry, Ez, Bz (slices), jx, jy
        (half-slices, index n <-> n + 1/2)."""
        return np.stack([self.S[k] for k in ("Rx", "Ry", "Ez", "Bz", "jx", "jy")])

    def stored_particles(self):
        P = self.stored
        return dict(x=P.x.copy(), y=P.y.copy(), zeta=P.zeta.copy(), ux=P.u[0].copy(),
                    uy=P.u[1].copy(), uz=P.u[2].copy(), weight=P.Q.copy(), species=P.sp.copy())
