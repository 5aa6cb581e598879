"""Seeded synthetic workloads for the GEM-PIC hot path.

This module is the one thing the CUDA path and the FP64 oracle share: plain parameter
records and seeded input arrays.  It holds none of the method's arithmetic (no push, no
deposit, no field update) and imports nothing from the rest of the package.

Units are the paper's normalised units (Sec. 3): lengths in c/omega_0, time in 1/omega_0,
fields in m c omega_0 / e, densities in n_cr.  With omega_0 = omega_L the laser wavelength is
lambda_L = 2*pi and an electron plasma of density n has omega_p^2 = n.

The stand-in workloads follow the paper's LWFA set-up (Sec. 6: Gaussian x-polarised laser
driver, Eq. E_laser; cold uniform background plasma swept by the moving window; fresh
macroparticles injected at the front every s-step, Sec. 5.1).  The
paper's own run (150x150x180 um, 12 h on 432 cores) is not a dataset; these seeded configs
stand in for it.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import List, Optional

import numpy as np

LAMBDA_L = 2.0 * math.pi          # laser wavelength for omega_0 = omega_L
SEED = 20250916                   # default seed of every workload


@dataclass
class Species:
    """One background species injected fresh at the front of the window every s-step.

    charge, mass in units of e, m_e; density in n_cr; ppc macroparticles per transverse cell.
    """
    charge: float = -1.0
    mass: float = 1.0
    density: float = 0.005
    ppc: int = 4


@dataclass
class Laser:
    """Driver E = e_pol a0 cos(phi) exp(-phi^2/T^2) exp(-r^2/w0^2), phi = zeta - zeta_c (Eq. E_laser).

    duration is T of the paper's exp(-phi^2/T^2) envelope; waist is R (1/e field radius);
    pol 0 = x, 1 = y.  The transverse centre is the middle node of the grid.
    """
    a0: float = 1.0
    waist: float = 8.0 * LAMBDA_L
    duration: float = 10.0 * LAMBDA_L / math.sqrt(2.0 * math.log(2.0))
    zeta_center: float = 0.0
    pol: int = 0


@dataclass
class Channel:
    """Transverse plasma channel (Sec. 6, Eq. n_plasma): every species' density is scaled by
    1 + (n1/n0 - 1) exp(-r^2/R_ch^2), r the transverse distance from the grid's middle node
    (2-D: |x - x_c|)."""
    n1_over_n0: float = 0.25            # Sec. 6: n1 = n0 / 4
    radius: float = 95.5 * LAMBDA_L     # Sec. 6: R_ch = 76.4 um at lambda = 0.8 um


@dataclass
class Beam:
    """Gaussian bunch placed in the box at creation (PWFA-style driver, Sec. 5.1 beam
    particles): density n_peak exp(-r^2/(2 sigma_r^2) - (zeta - zeta_center)^2/(2 sigma_z^2)),
    r from the grid's middle node, cold, gamma (1 + rel_spread N(0, 1)) along +z, n_macro
    equal-charge macroparticles.  A parameter record only: the library and the oracle each
    sample it from the bunch's own counter-based SplitMix64 stream `seed`."""
    charge: float = -1.0
    mass: float = 1.0
    n_peak: float = 0.01
    sigma_r: float = 1.0
    sigma_z: float = 1.0
    zeta_center: float = 0.0
    gamma: float = 1000.0
    rel_spread: float = 1e-3
    n_macro: int = 1024
    seed: int = SEED + 1


@dataclass
class StoredParticles:
    """Macroparticles placed inside the box at creation (beam / driver bunch, Sec. 5.1 Q_b).

    Positions are absolute (x, y, zeta), momenta u = p/(m c), weight is the macroparticle
    charge Q (sign included), species indexes the workload's species list for q/m.
    """
    x: np.ndarray
    y: np.ndarray
    zeta: np.ndarray
    ux: np.ndarray
    uy: np.ndarray
    uz: np.ndarray
    weight: np.ndarray
    species: np.ndarray

    @property
    def n(self) -> int:
        return int(self.x.shape[0])


@dataclass
class Workload:
    """A GEM-PIC run: grid, s-step Delta, species, driver, seed and precision."""
    name: str
    nx: int
    ny: int                      # ny == 1 -> 2-D slab (x, zeta), y-invariant
    nzeta: int
    hx: float
    hy: float                    # 2-D: hy = 1 (per unit length in y)
    h: float
    delta: float
    species: List[Species] = field(default_factory=list)
    laser: Optional[Laser] = None
    seed: int = SEED
    precision: int = 64          # 64 or 32
    steps: int = 1
    stored: Optional[StoredParticles] = None
    snapshot: bool = False       # keep real-space fields of the last s-step
    channel: Optional[Channel] = None   # None: uniform density
    particle_law: str = "GT2"    # "GT2" (Eq. trap2, s~ = z) or "GT1" (Eq. trap1, s = ct)
    hz: Optional[np.ndarray] = None     # nzeta slab thicknesses (back to front); None: h
    residual: bool = False       # report the deposit's continuity residual (2-D)
    beam: Optional[Beam] = None  # Gaussian bunch sampled in the box at creation
    capture_current: bool = False  # keep the current of the last s-step of each call

    @property
    def ncells(self) -> int:
        return self.nx * self.ny * self.nzeta

    @property
    def pushes_per_step(self) -> int:
        """Streaming pushes per s-step: every fresh particle crosses every slice once."""
        return sum(sp.ppc for sp in self.species) * self.nx * self.ny * self.nzeta

    @property
    def omega_p2(self) -> float:
        return sum(sp.charge ** 2 * sp.density / sp.mass for sp in self.species)

    def with_(self, **kw) -> "Workload":
        return replace(self, **kw)


def refined_h(nzeta: int, h_front: float, ratio: float, back_fraction: float = 1.0 / 3.0,
              width: float = 0.1) -> np.ndarray:
    """Slab thicknesses refined at the back of the window (Sec. 6: 6.3 nm over the back third,
    where the bubble's back wall sits, 50 nm in front): h_front / ratio behind, h_front in
    front, joined smoothly by a tanh over `width` of the window.  Index 0 is the back slab."""
    x = (np.arange(nzeta) + 0.5) / nzeta
    t = 0.5 * (1.0 + np.tanh((x - back_fraction) / width))
    return h_front / ratio + (h_front - h_front / ratio) * t


def fwhm_to_T(fwhm_intensity: float) -> float:
    """T of exp(-phi^2/T^2) for a given intensity FWHM (intensity ~ exp(-2 phi^2/T^2))."""
    return fwhm_intensity / math.sqrt(2.0 * math.log(2.0))


def lwfa_2d_128x256(precision: int = 64, steps: int = 200) -> Workload:
    """2-D (x, zeta) LWFA: 128 x 256, dzeta = lambda/20, dx = lambda/2, n0 = 0.005 n_cr,
    4 ppc, a0 = 1, 10 lambda/c FWHM, waist 8 lambda, Delta at the stability limit
    Delta h omega_p^2 = 4 (Sec. 4.2)."""
    h = LAMBDA_L / 20.0
    n0 = 0.005
    L = 256 * h
    return Workload(
        name="lwfa2d_128x256_ppc4", nx=128, ny=1, nzeta=256, hx=LAMBDA_L / 2.0, hy=1.0, h=h,
        delta=4.0 / (n0 * h), species=[Species(-1.0, 1.0, n0, 4)],
        laser=Laser(a0=1.0, waist=8.0 * LAMBDA_L, duration=fwhm_to_T(10.0 * LAMBDA_L),
                    zeta_center=0.6 * L),
        precision=precision, steps=steps)


def scan_2d(n: int = 64, seed: int = SEED, precision: int = 32, steps: int = 500) -> List[Workload]:
    """Batched parameter scan: n independent 2-D (x, zeta) instances with nx drawn from
    {128, 256, 512} and nzeta from {256, 512, 1024, 2048}, a0 ~ U[0.5, 3], n0 log-uniform on
    [1e-3, 1e-2] n_cr, 4 ppc, dzeta = lambda/20, dx = lambda/2, Delta at each instance's
    stability limit Delta h omega_p^2 = 4, and the laser of the 2-D workload (10 lambda/c
    FWHM, waist 8 lambda) centred at 0.6 of the window.  Draws from a seeded generator;
    instance i uses seed + i for its injection offsets."""
    rng = np.random.default_rng(seed)
    h = LAMBDA_L / 20.0
    out = []
    for i in range(n):
        nx = int(rng.choice([128, 256, 512]))
        nz = int(rng.choice([256, 512, 1024, 2048]))
        a0 = float(rng.uniform(0.5, 3.0))
        n0 = float(10.0 ** rng.uniform(-3.0, -2.0))
        L = nz * h
        out.append(Workload(
            name=f"scan{i}_{nx}x{nz}", nx=nx, ny=1, nzeta=nz, hx=LAMBDA_L / 2.0, hy=1.0, h=h,
            delta=4.0 / (n0 * h), species=[Species(-1.0, 1.0, n0, 4)],
            laser=Laser(a0=a0, waist=8.0 * LAMBDA_L, duration=fwhm_to_T(10.0 * LAMBDA_L),
                        zeta_center=0.6 * L),
            seed=seed + i, precision=precision, steps=steps))
    return out


def lwfa_3d_128x128x1024(precision: int = 32, steps: int = 2000) -> Workload:
    """3-D LWFA: 128 x 128 x 1024, dzeta = lambda/20, dx = dy = lambda/4, n0 = 0.002 n_cr,
    2 ppc (33.5 M pushes per s-step), a0 = 2.5, 8 lambda/c FWHM, waist 10 lambda.
    Delta = min(4/(omega_p^2 h), Z_R/10) with Z_R = pi w0^2/lambda."""
    h = LAMBDA_L / 20.0
    n0 = 0.002
    w0 = 10.0 * LAMBDA_L
    zr = math.pi * w0 * w0 / LAMBDA_L
    T = fwhm_to_T(8.0 * LAMBDA_L)
    L = 1024 * h
    return Workload(
        name="lwfa3d_128x128x1024_ppc2", nx=128, ny=128, nzeta=1024, hx=LAMBDA_L / 4.0,
        hy=LAMBDA_L / 4.0, h=h, delta=min(4.0 / (n0 * h), zr / 10.0),
        species=[Species(-1.0, 1.0, n0, 2)],
        laser=Laser(a0=2.5, waist=w0, duration=T, zeta_center=L - 2.0 * T),
        precision=precision, steps=steps)


def lwfa_3d_128x128x512(ppc: int = 1, precision: int = 32, steps: int = 200) -> Workload:
    """The denoiser's 3-D LWFA: the laser and plasma of the 128 x 128 x 1024 workload
    (dzeta = lambda/20, dx = dy = lambda/4, n0 = 0.002 n_cr, a0 = 2.5, 8 lambda/c FWHM, waist
    10 lambda, the same Delta) on a 512-slice window, at ppc particles per cell (1 for the
    sparse run the denoiser cleans, 16 for the dense run it is trained towards)."""
    w = lwfa_3d_128x128x1024(precision=precision, steps=steps)
    L = 512 * w.h
    return w.with_(name=f"lwfa3d_128x128x512_ppc{ppc}", nzeta=512,
                   species=[Species(-1.0, 1.0, w.species[0].density, ppc)],
                   laser=Laser(**{**w.laser.__dict__, "zeta_center": L - 2.0 * w.laser.duration}))


def pwfa_3d_128x128x768(precision: int = 32, steps: int = 1000, n_macro: int = 1 << 20) -> Workload:
    """Beam-driven wakefield (units omega_0 = omega_p, so n0 = 1): background electrons and
    mobile protons (m = 1836), 2 + 2 per cell, cold, injected at the front; an electron drive
    bunch n_b = 2 n0, sigma_r = 0.5, sigma_z = 1 c/omega_p, gamma = 2000 with 1e-3 relative
    spread, n_macro equal-charge macroparticles, centred 3 sigma_z behind the front; window
    12 x 12 x 15.36 c/omega_p, h = 1/50, Delta = 10 (about 40 s-steps per betatron period
    2 pi sqrt(2 gamma)).  The transverse grid is 128 x 128 (hx = 12/128), the largest square
    power-of-two grid one cluster marches; the 192 x 192 grid of the same box is not (its
    transforms are not powers of two)."""
    n0 = 1.0
    h = 1.0 / 50.0
    hx = 12.0 / 128.0
    L = 768 * h
    return Workload(
        name="pwfa3d_128x128x768_ppc2x2", nx=128, ny=128, nzeta=768, hx=hx, hy=hx, h=h,
        delta=10.0, species=[Species(-1.0, 1.0, n0, 2), Species(1.0, 1836.0, n0, 2)],
        laser=None, precision=precision, steps=steps,
        beam=Beam(charge=-1.0, mass=1.0, n_peak=2.0 * n0, sigma_r=0.5, sigma_z=1.0,
                  zeta_center=L - 3.0, gamma=2000.0, rel_spread=1e-3, n_macro=n_macro,
                  seed=SEED + 3))


def small_3d(nx: int = 16, ny: int = 16, nzeta: int = 48, ppc: int = 2, precision: int = 64,
             a0: float = 1.5, n0: float = 0.01, delta: Optional[float] = None,
             steps: int = 2) -> Workload:
    """Scaled-down 3-D LWFA used for parity: same physics, grid small enough for the oracle."""
    h = LAMBDA_L / 16.0
    hx = LAMBDA_L / 2.0
    w0 = 2.5 * LAMBDA_L
    T = fwhm_to_T(1.5 * LAMBDA_L)
    L = nzeta * h
    if delta is None:
        delta = min(4.0 / (n0 * h), 40.0)
    return Workload(
        name=f"lwfa3d_{nx}x{ny}x{nzeta}_ppc{ppc}", nx=nx, ny=ny, nzeta=nzeta, hx=hx, hy=hx, h=h,
        delta=delta, species=[Species(-1.0, 1.0, n0, ppc)],
        laser=Laser(a0=a0, waist=w0, duration=T, zeta_center=L - 2.2 * T),
        precision=precision, steps=steps)


def small_2d(nx: int = 32, nzeta: int = 64, ppc: int = 3, precision: int = 64, a0: float = 1.0,
             n0: float = 0.01, delta: Optional[float] = None, steps: int = 3) -> Workload:
    """Scaled-down 2-D (x, zeta) LWFA for parity tests."""
    h = LAMBDA_L / 16.0
    hx = LAMBDA_L / 2.0
    T = fwhm_to_T(1.5 * LAMBDA_L)
    L = nzeta * h
    if delta is None:
        delta = 4.0 / (n0 * h)
    return Workload(
        name=f"lwfa2d_{nx}x{nzeta}_ppc{ppc}", nx=nx, ny=1, nzeta=nzeta, hx=hx, hy=1.0, h=h,
        delta=delta, species=[Species(-1.0, 1.0, n0, ppc)],
        laser=Laser(a0=a0, waist=3.0 * LAMBDA_L, duration=T, zeta_center=L - 2.2 * T),
        precision=precision, steps=steps)


def gaussian_bunch(w: Workload, n_macro: int, n_peak: float, sigma_r: float, sigma_z: float,
                   zeta_center: float, gamma: float, rel_spread: float, species: int = 0,
                   seed: int = SEED) -> StoredParticles:
    """Seeded Gaussian driver bunch placed in the box (PWFA-style driver).

    Equal-weight macroparticles; the total charge equals that of the density profile
    n_peak exp(-r^2/(2 sr^2) - (zeta-zc)^2/(2 sz^2)) times the species charge.
    """
    rng = np.random.default_rng(seed)
    q = w.species[species].charge
    xc = 0.5 * w.nx * w.hx
    yc = 0.5 * w.ny * w.hy if w.ny > 1 else 0.0
    if w.ny > 1:
        total = q * n_peak * (2.0 * math.pi) ** 1.5 * sigma_r * sigma_r * sigma_z
        y = yc + sigma_r * rng.standard_normal(n_macro)
    else:
        total = q * n_peak * (2.0 * math.pi) * sigma_r * sigma_z
        y = np.zeros(n_macro)
    x = xc + sigma_r * rng.standard_normal(n_macro)
    zeta = zeta_center + sigma_z * rng.standard_normal(n_macro)
    g = gamma * (1.0 + rel_spread * rng.standard_normal(n_macro))
    uz = np.sqrt(g * g - 1.0)
    zero = np.zeros(n_macro)
    keep = (zeta > 0.0) & (zeta < w.nzeta * w.h)
    wgt = np.full(n_macro, total / n_macro)
    return StoredParticles(x=x[keep], y=y[keep], zeta=zeta[keep], ux=zero[keep].copy(),
                           uy=zero[keep].copy(), uz=uz[keep], weight=wgt[keep],
                           species=np.full(int(keep.sum()), species, dtype=np.int32))
