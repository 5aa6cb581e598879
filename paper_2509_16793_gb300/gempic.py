"""Thin ctypes binding of libgempic.so (include/gempic.h).

Argument marshalling only: every step of the GEM-PIC path runs in the library's CUDA
kernels.  The functions keep the C names (gempic_create, gempic_step, ...); `Sim` wraps one
simulation handle.  There is no fallback: if libgempic.so is missing or no GPU is present,
`load()` raises.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import (POINTER, Structure, c_char_p, c_double, c_int32, c_int64, c_size_t,
                    c_uint32, c_uint64, c_void_p, byref)
from typing import Optional

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libgempic.so")

GEMPIC_FLAG_DIAG = 1
GEMPIC_FLAG_SNAPSHOT = 2
GEMPIC_FLAG_GT1 = 4
GEMPIC_FLAG_RESIDUAL = 8
GEMPIC_FLAG_CURRENT = 16
STATUS = {0: "GEMPIC_OK", -1: "GEMPIC_EINVAL", -2: "GEMPIC_ENOMEM", -3: "GEMPIC_ECUDA",
          -4: "GEMPIC_EUNSTABLE", -5: "GEMPIC_ETIMEOUT", -6: "GEMPIC_ESTATE",
          -7: "GEMPIC_EOVERFLOW", -8: "GEMPIC_ENONFINITE"}
FIELDS = {"Ex": 0, "Ey": 1, "Ez": 2, "Bx": 3, "By": 4, "Bz": 5, "jx": 6, "jy": 7, "jz": 8}


class GempicError(RuntimeError):
    def __init__(self, status: int, what: str, msg: str = ""):
        super().__init__(f"{what}: {STATUS.get(status, status)} ({msg})")
        self.status = status


class gempic_grid(Structure):
    _fields_ = [("nx", c_int32), ("ny", c_int32), ("nzeta", c_int32),
                ("hx", c_double), ("hy", c_double), ("h", c_double)]


class gempic_species(Structure):
    _fields_ = [("charge", c_double), ("mass", c_double), ("density", c_double),
                ("ppc", c_int32), ("reserved", c_int32)]


class gempic_laser(Structure):
    _fields_ = [("a0", c_double), ("waist", c_double), ("duration", c_double),
                ("zeta_center", c_double), ("pol", c_int32), ("reserved", c_int32),
                ("fwhm_intensity", c_double)]


class gempic_beam(Structure):
    _fields_ = [("charge", c_double), ("mass", c_double), ("n_peak", c_double),
                ("sigma_r", c_double), ("sigma_z", c_double), ("zeta_center", c_double),
                ("gamma", c_double), ("rel_spread", c_double), ("n_macro", c_int64),
                ("seed", c_uint64)]


class gempic_channel(Structure):
    _fields_ = [("n1_over_n0", c_double), ("radius", c_double)]


class gempic_config(Structure):
    _fields_ = [("grid", gempic_grid), ("delta", c_double), ("precision", c_int32),
                ("flags", c_uint32), ("seed", c_uint64), ("nspecies", c_int32),
                ("cluster_ctas", c_int32), ("species", POINTER(gempic_species)),
                ("laser", POINTER(gempic_laser)), ("stored_bucket_capacity", c_int32),
                ("particle_headroom", c_int32), ("pipeline_depth", c_int32),
                ("reserved", c_int32), ("cuda_stream", c_void_p),
                ("channel", POINTER(gempic_channel)), ("hz", POINTER(c_double)),
                ("beam", POINTER(gempic_beam))]


class gempic_diag(Structure):
    _fields_ = [("step", c_int64), ("field_energy", c_double), ("kinetic_energy", c_double),
                ("charge_flux", c_double), ("n_trapped", c_int64), ("n_stored", c_int64),
                ("n_rejoined", c_int64), ("pushes", c_int64),
                ("continuity_residual", c_double), ("gauss_residual", c_double),
                ("stored_kinetic_energy", c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


# exported symbols and their signatures (include/gempic.h)
SIGNATURES = {
    "gempic_create": (c_int32, [POINTER(gempic_config), POINTER(c_void_p)]),
    "gempic_add_particles": (c_int32, [c_void_p, c_int64] + [c_void_p] * 8),
    "gempic_step": (c_int32, [c_void_p, c_int32]),
    "gempic_step_async": (c_int32, [c_void_p, c_int32]),
    "gempic_sync": (c_int32, [c_void_p]),
    "gempic_set_wait_limit": (c_int32, [c_void_p, c_int64]),
    "gempic_set_delta": (c_int32, [c_void_p, c_double]),
    "gempic_step_host": (c_int32, [c_void_p, c_int32, c_void_p, c_void_p, c_size_t, POINTER(gempic_diag)]),
    "gempic_step_streamed": (c_int32, [c_void_p, c_int32, c_void_p, c_size_t, POINTER(gempic_diag)]),
    "gempic_state_bytes": (c_size_t, [c_void_p]),
    "gempic_get_state": (c_int32, [c_void_p, c_void_p, c_size_t, c_int32]),
    "gempic_set_state": (c_int32, [c_void_p, c_void_p, c_size_t, c_int32]),
    "gempic_get_fields": (c_int32, [c_void_p, c_int32, c_void_p, c_size_t, c_int32]),
    "gempic_get_particles": (c_int32, [c_void_p, c_int32, POINTER(c_int64)] + [c_void_p] * 8),
    "gempic_get_diagnostics": (c_int32, [c_void_p, POINTER(gempic_diag)]),
    "gempic_get_onaxis_ez": (c_int32, [c_void_p, c_void_p, c_int32]),
    "gempic_launch_count": (c_int64, [c_void_p]),
    "gempic_launch_shape": (c_int32, [c_void_p] + [POINTER(c_int32)] * 4),
    "gempic_step_noalloc": (c_int32, [POINTER(gempic_config), c_int64, c_void_p, c_size_t,
                                       POINTER(gempic_diag), c_void_p]),
    "gempic_batch_create": (c_int32, [POINTER(gempic_config), c_int32, POINTER(c_void_p)]),
    "gempic_batch_step_async": (c_int32, [c_void_p, c_int32]),
    "gempic_batch_sync": (c_int32, [c_void_p]),
    "gempic_batch_step": (c_int32, [c_void_p, c_int32]),
    "gempic_batch_size": (c_int32, [c_void_p]),
    "gempic_batch_sim": (c_void_p, [c_void_p, c_int32]),
    "gempic_batch_stream": (c_void_p, [c_void_p, c_int32]),
    "gempic_batch_tuning": (c_int32, [c_void_p, c_int32, POINTER(c_int32), POINTER(c_double)]),
    "gempic_batch_destroy": (None, [c_void_p]),
    "gempic_probe_fp32_fma": (c_int32, [c_void_p, c_int32, POINTER(c_double), POINTER(c_double)]),
    "gempic_denoiser_param_count": (c_size_t, []),
    "gempic_denoiser_create": (c_int32, [c_void_p, c_double, POINTER(c_void_p)]),
    "gempic_denoiser_set_params": (c_int32, [c_void_p, c_void_p, c_size_t]),
    "gempic_denoiser_get_params": (c_int32, [c_void_p, c_void_p, c_size_t]),
    "gempic_denoiser_apply": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_int32, c_int32,
                                        c_void_p]),
    "gempic_denoiser_grad": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_int32, c_int32,
                                       c_int32, POINTER(c_double), c_void_p, c_void_p]),
    "gempic_denoiser_train_step": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_int32,
                                             c_int32, c_int32, c_double, POINTER(c_double),
                                             c_void_p]),
    "gempic_denoiser_destroy": (None, [c_void_p]),
    "gempic_set_denoiser": (c_int32, [c_void_p, c_void_p]),
    "gempic_get_current": (c_int32, [c_void_p, c_void_p, c_size_t, c_int32]),
    "gempic_strerror": (c_char_p, [c_int32]),
    "gempic_destroy": (None, [c_void_p]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libgempic.so and declare its signatures (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(st: int, what: str):
    if st != 0:
        raise GempicError(st, what, load().gempic_strerror(st).decode())


def _ptr(a) -> int:
    """Raw pointer of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def config_from_workload(w, *, flags: int = GEMPIC_FLAG_DIAG, cluster_ctas: int = 0,
                         pipeline_depth: int = 0, bucket_capacity: int = 0,
                         headroom: int = 0, stream: Optional[int] = None,
                         laser_fwhm: Optional[float] = None):
    """gempic_config for a paper_2509_16793_gb300.workloads.Workload (plus the arrays it
    points to, returned so that they outlive the create call).  laser_fwhm: pass the laser's
    intensity FWHM instead of its T (the library converts)."""
    n = len(w.species)
    sp = (gempic_species * max(n, 1))()
    for i, s in enumerate(w.species):
        sp[i] = gempic_species(s.charge, s.mass, s.density, s.ppc, 0)
    las = None
    if w.laser is not None:
        L = w.laser
        if laser_fwhm is None:
            las = gempic_laser(L.a0, L.waist, L.duration, L.zeta_center, L.pol, 0, 0.0)
        else:
            las = gempic_laser(L.a0, L.waist, 0.0, L.zeta_center, L.pol, 0, float(laser_fwhm))
    bm = None
    if w.beam is not None:
        b = w.beam
        bm = gempic_beam(b.charge, b.mass, b.n_peak, b.sigma_r, b.sigma_z, b.zeta_center,
                         b.gamma, b.rel_spread, int(b.n_macro), int(b.seed))
    hz = None
    if w.hz is not None:
        hz = np.ascontiguousarray(w.hz, dtype=np.float64)
        if hz.shape != (w.nzeta,):
            raise ValueError("hz holds nzeta slab thicknesses")
    ch = None
    if w.channel is not None:
        ch = gempic_channel(w.channel.n1_over_n0, w.channel.radius)
    if w.snapshot:
        flags |= GEMPIC_FLAG_SNAPSHOT
    if w.particle_law not in ("GT1", "GT2"):
        raise ValueError("particle_law is GT1 or GT2")
    if w.particle_law == "GT1":
        flags |= GEMPIC_FLAG_GT1
    if w.residual:
        flags |= GEMPIC_FLAG_RESIDUAL
    if getattr(w, "capture_current", False):
        flags |= GEMPIC_FLAG_CURRENT
    cfg = gempic_config(
        grid=gempic_grid(w.nx, w.ny, w.nzeta, w.hx, w.hy, w.h), delta=w.delta,
        precision=w.precision, flags=flags, seed=w.seed, nspecies=n, cluster_ctas=cluster_ctas,
        species=ctypes.cast(sp, POINTER(gempic_species)),
        laser=ctypes.pointer(las) if las is not None else None,
        stored_bucket_capacity=bucket_capacity, particle_headroom=headroom,
        pipeline_depth=pipeline_depth, reserved=0, cuda_stream=stream,
        channel=ctypes.pointer(ch) if ch is not None else None,
        hz=hz.ctypes.data_as(POINTER(c_double)) if hz is not None else None,
        beam=ctypes.pointer(bm) if bm is not None else None)
    return cfg, (sp, las, ch, hz, bm)


def gempic_probe_fp32_fma(iters: int = 200000, stream: Optional[int] = None):
    """Measured FP32 FMA throughput: (TFLOP/s, kernel ms)."""
    t, ms = c_double(), c_double()
    _check(load().gempic_probe_fp32_fma(stream, int(iters), byref(t), byref(ms)),
           "gempic_probe_fp32_fma")
    return t.value, ms.value


def gempic_step_noalloc(w, step: int, state, onaxis: bool = False, stream: Optional[int] = None,
                        cluster_ctas: int = 0):
    """One allocation-free s-step on a caller-owned device state (torch tensor in the layout of
    gempic_get_state).  Returns (status, diagnostics dict, on-axis E_z or None)."""
    lib = load()
    cfg, keep = config_from_workload(w, cluster_ctas=cluster_ctas, stream=stream)
    d = gempic_diag()
    ez = np.empty(w.nzeta) if onaxis else None
    st = lib.gempic_step_noalloc(byref(cfg), step, state.data_ptr(),
                                 state.numel() * state.element_size(), byref(d),
                                 ez.ctypes.data if ez is not None else None)
    del keep
    return st, d.as_dict(), ez


class Sim:
    """One GEM-PIC simulation on the GPU (gempic_create ... gempic_destroy)."""

    def __init__(self, w, **kw):
        lib = load()
        cfg, self._keep = config_from_workload(w, **kw)
        h = c_void_p()
        _check(lib.gempic_create(byref(cfg), byref(h)), "gempic_create")
        self._attach(lib, w, h, owned=True)

    @classmethod
    def borrowed(cls, w, handle):
        """A view of a simulation owned elsewhere (an instance of a Batch)."""
        self = cls.__new__(cls)
        self._attach(load(), w, c_void_p(handle), owned=False)
        return self

    def _attach(self, lib, w, h, owned):
        self.w = w
        self.lib = lib
        self.h = h
        self.owned = owned
        self.dtype = np.complex128 if w.precision == 64 else np.complex64
        self.rdtype = np.float64 if w.precision == 64 else np.float32
        if w.stored is not None and w.stored.n > 0:
            st = w.stored
            arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in
                    (st.x, st.y, st.zeta, st.ux, st.uy, st.uz, st.weight)]
            spc = np.ascontiguousarray(st.species, dtype=np.int32)
            _check(lib.gempic_add_particles(self.h, st.n, *[a.ctypes.data for a in arrs],
                                            spc.ctypes.data), "gempic_add_particles")

    def gempic_step(self, n: int = 1):
        _check(self.lib.gempic_step(self.h, n), "gempic_step")

    step = gempic_step

    def gempic_step_async(self, n: int = 1):
        _check(self.lib.gempic_step_async(self.h, n), "gempic_step_async")

    step_async = gempic_step_async

    def gempic_sync(self):
        _check(self.lib.gempic_sync(self.h), "gempic_sync")

    sync = gempic_sync

    def gempic_set_delta(self, delta: float):
        _check(self.lib.gempic_set_delta(self.h, float(delta)), "gempic_set_delta")

    set_delta = gempic_set_delta

    def gempic_set_denoiser(self, d):
        """Denoised s-steps with the Denoiser d (None: plain steps).  Keeps a reference."""
        _check(self.lib.gempic_set_denoiser(self.h, d.h if d is not None else None),
               "gempic_set_denoiser")
        self._denoiser = d

    set_denoiser = gempic_set_denoiser

    def gempic_get_current(self, out=None):
        """The plain current of the last s-step, [nzeta, 3, ny, nx]: into a device tensor
        `out`, or a new host array."""
        w = self.w
        if out is not None and hasattr(out, "data_ptr") and out.is_cuda:
            _check(self.lib.gempic_get_current(self.h, out.data_ptr(),
                                               out.numel() * out.element_size(), 1),
                   "gempic_get_current")
            return out
        a = np.empty((w.nzeta, 3, w.ny, w.nx), self.rdtype)
        _check(self.lib.gempic_get_current(self.h, a.ctypes.data, a.nbytes, 0), "gempic_get_current")
        return a

    current = gempic_get_current

    def gempic_set_wait_limit(self, polls: int):
        _check(self.lib.gempic_set_wait_limit(self.h, int(polls)), "gempic_set_wait_limit")

    set_wait_limit = gempic_set_wait_limit

    def state_bytes(self) -> int:
        return int(self.lib.gempic_state_bytes(self.h))

    def state_shape(self):
        w = self.w
        return (6, w.nzeta, w.ny, w.nx // 2)

    def gempic_get_state(self, out=None) -> np.ndarray:
        """Spectral state [6, nzeta, ny, nx/2] (Rx, Ry, Ez, Bz, jx, jy) on the host, or into
        `out`: a device tensor, or a C-contiguous host buffer of state_bytes() bytes (any
        dtype; its bytes are written)."""
        if out is not None and hasattr(out, "data_ptr") and out.is_cuda:
            _check(self.lib.gempic_get_state(self.h, out.data_ptr(), self.state_bytes(), 1), "gempic_get_state")
            return out
        if out is not None:
            if out.nbytes < self.state_bytes() or not out.flags["C_CONTIGUOUS"]:
                raise ValueError("out must be C-contiguous with state_bytes() bytes")
            _check(self.lib.gempic_get_state(self.h, out.ctypes.data, out.nbytes, 0), "gempic_get_state")
            return out
        a = np.empty(self.state_shape(), self.dtype)
        _check(self.lib.gempic_get_state(self.h, a.ctypes.data, a.nbytes, 0), "gempic_get_state")
        return a

    state = gempic_get_state

    def gempic_set_state(self, a):
        """From a device tensor, a host array of the state (converted to its dtype), or a raw
        C-contiguous host buffer of exactly state_bytes() bytes in another dtype."""
        if hasattr(a, "data_ptr") and a.is_cuda:
            _check(self.lib.gempic_set_state(self.h, a.data_ptr(), self.state_bytes(), 1), "gempic_set_state")
            return
        if not (a.dtype != self.dtype and a.nbytes == self.state_bytes() and a.flags["C_CONTIGUOUS"]):
            a = np.ascontiguousarray(a, self.dtype)
        _check(self.lib.gempic_set_state(self.h, a.ctypes.data, a.nbytes, 0), "gempic_set_state")

    set_state = gempic_set_state

    def gempic_step_host(self, n: int, state_in: Optional[np.ndarray], state_out: Optional[np.ndarray]):
        d = gempic_diag()
        nb = self.state_bytes()
        _check(self.lib.gempic_step_host(self.h, n, _ptr(state_in), _ptr(state_out), nb, byref(d)),
               "gempic_step_host")
        return d.as_dict()

    def gempic_step_streamed(self, n: int, host_state, diagnostics: bool = True):
        """n s-steps with the state streamed through `host_state` (a C-contiguous host buffer
        of state_bytes() bytes in the layout of gempic_get_state: the first s-step's input,
        the last one's result on return).  Returns the diagnostics of each s-step."""
        nb = self.state_bytes()
        if host_state.nbytes < nb:
            raise ValueError(f"host_state holds {host_state.nbytes} bytes, the state {nb}")
        d = (gempic_diag * max(n, 1))()
        _check(self.lib.gempic_step_streamed(self.h, n, _ptr(host_state), host_state.nbytes,
                                             d if diagnostics else None), "gempic_step_streamed")
        return [d[i].as_dict() for i in range(n)] if diagnostics else None

    step_streamed = gempic_step_streamed

    def gempic_get_fields(self, comp) -> np.ndarray:
        c = FIELDS[comp] if isinstance(comp, str) else int(comp)
        w = self.w
        a = np.empty((w.nzeta, w.ny, w.nx), self.rdtype)
        _check(self.lib.gempic_get_fields(self.h, c, a.ctypes.data, a.nbytes, 0), "gempic_get_fields")
        return a

    fields = gempic_get_fields

    def gempic_get_particles(self, kind: int = 0) -> dict:
        n = c_int64(0)
        st = self.lib.gempic_get_particles(self.h, kind, byref(n), *([None] * 8))
        if st not in (0, -1):
            _check(st, "gempic_get_particles")
        cnt = n.value
        out = {k: np.empty(cnt) for k in ("x", "y", "zeta", "ux", "uy", "uz", "weight")}
        out["species"] = np.empty(cnt, np.int32)
        n = c_int64(cnt)
        _check(self.lib.gempic_get_particles(
            self.h, kind, byref(n), *[out[k].ctypes.data for k in
                                      ("x", "y", "zeta", "ux", "uy", "uz", "weight", "species")]),
            "gempic_get_particles")
        return out

    particles = gempic_get_particles

    def gempic_get_diagnostics(self) -> dict:
        d = gempic_diag()
        _check(self.lib.gempic_get_diagnostics(self.h, byref(d)), "gempic_get_diagnostics")
        return d.as_dict()

    diagnostics = gempic_get_diagnostics

    def gempic_get_onaxis_ez(self) -> np.ndarray:
        a = np.empty(self.w.nzeta)
        _check(self.lib.gempic_get_onaxis_ez(self.h, a.ctypes.data, a.size), "gempic_get_onaxis_ez")
        return a

    onaxis_ez = gempic_get_onaxis_ez

    def launch_count(self) -> int:
        return int(self.lib.gempic_launch_count(self.h))

    def launch_shape(self) -> dict:
        v = [c_int32() for _ in range(4)]
        _check(self.lib.gempic_launch_shape(self.h, *[byref(x) for x in v]), "gempic_launch_shape")
        return dict(cluster_ctas=v[0].value, threads=v[1].value, smem_bytes=v[2].value,
                    pipeline=v[3].value)

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            if getattr(self, "owned", True):
                self.lib.gempic_destroy(self.h)
            self.h = c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Batch:
    """Independent simulations stepped side by side (gempic_batch_create ...
    gempic_batch_destroy); `sims[i]` is a view of instance i for the query calls."""

    def __init__(self, workloads, **kw):
        lib = load()
        n = len(workloads)
        cfgs = (gempic_config * n)()
        self._keep = []
        for i, w in enumerate(workloads):
            c, k = config_from_workload(w, **kw)
            cfgs[i] = c
            self._keep.append(k)
        h = c_void_p()
        _check(lib.gempic_batch_create(cfgs, n, byref(h)), "gempic_batch_create")
        self.lib = lib
        self.h = h
        self.workloads = list(workloads)
        self.sims = [Sim.borrowed(w, lib.gempic_batch_sim(h, i)) for i, w in enumerate(workloads)]

    def __len__(self):
        return int(self.lib.gempic_batch_size(self.h))

    def gempic_batch_step(self, n: int = 1):
        _check(self.lib.gempic_batch_step(self.h, n), "gempic_batch_step")

    step = gempic_batch_step

    def gempic_batch_step_async(self, n: int = 1):
        _check(self.lib.gempic_batch_step_async(self.h, n), "gempic_batch_step_async")

    step_async = gempic_batch_step_async

    def gempic_batch_sync(self):
        _check(self.lib.gempic_batch_sync(self.h), "gempic_batch_sync")

    sync = gempic_batch_sync

    def gempic_batch_tuning(self, i: int):
        """(threads per CTA of the launch, measured ms per s-step of instance i's class)."""
        nt, ms = c_int32(), c_double()
        _check(self.lib.gempic_batch_tuning(self.h, i, byref(nt), byref(ms)), "gempic_batch_tuning")
        return nt.value, ms.value

    tuning = gempic_batch_tuning

    def gempic_batch_stream(self, i: int) -> int:
        return int(self.lib.gempic_batch_stream(self.h, i) or 0)

    stream = gempic_batch_stream

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            for v in self.sims:
                v.h = c_void_p()
            self.lib.gempic_batch_destroy(self.h)
            self.h = c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Denoiser:
    """The learned current denoiser (gempic_denoiser_create ... gempic_denoiser_destroy).
    Currents are device FP32 tensors [nz, 3, ny, nx]; parameters a host FP32 vector."""

    def __init__(self, params: Optional[np.ndarray] = None, scale: float = 1.0):
        self.lib = load()
        self.n = int(self.lib.gempic_denoiser_param_count())
        h = c_void_p()
        p = None
        if params is not None:
            p = np.ascontiguousarray(params, dtype=np.float32)
            if p.size != self.n:
                raise ValueError(f"expected {self.n} parameters")
        _check(self.lib.gempic_denoiser_create(p.ctypes.data if p is not None else None,
                                               float(scale), byref(h)), "gempic_denoiser_create")
        self.h = h
        self.scale = float(scale)

    def set_params(self, params: np.ndarray):
        p = np.ascontiguousarray(params, dtype=np.float32)
        _check(self.lib.gempic_denoiser_set_params(self.h, p.ctypes.data, p.size),
               "gempic_denoiser_set_params")

    def params(self) -> np.ndarray:
        p = np.empty(self.n, np.float32)
        _check(self.lib.gempic_denoiser_get_params(self.h, p.ctypes.data, p.size),
               "gempic_denoiser_get_params")
        return p

    @staticmethod
    def _dims(j):
        nz, c, ny, nx = j.shape
        if c != 3 or not j.is_cuda or not j.is_contiguous():
            raise ValueError("currents are contiguous device tensors [nz, 3, ny, nx]")
        return nx, ny, nz

    def apply(self, j, out=None, stream: Optional[int] = None):
        import torch
        nx, ny, nz = self._dims(j)
        out = torch.empty_like(j) if out is None else out
        _check(self.lib.gempic_denoiser_apply(self.h, j.data_ptr(), out.data_ptr(), nx, ny, nz,
                                              stream), "gempic_denoiser_apply")
        return out

    def grad(self, j, target, z_margin: int = 0, stream: Optional[int] = None):
        nx, ny, nz = self._dims(j)
        loss = c_double()
        g = np.empty(self.n, np.float32)
        _check(self.lib.gempic_denoiser_grad(self.h, j.data_ptr(), target.data_ptr(), nx, ny, nz,
                                             z_margin, byref(loss), g.ctypes.data, stream),
               "gempic_denoiser_grad")
        return loss.value, g

    def train_step(self, j, target, lr: float, z_margin: int = 0, stream: Optional[int] = None):
        nx, ny, nz = self._dims(j)
        loss = c_double()
        _check(self.lib.gempic_denoiser_train_step(self.h, j.data_ptr(), target.data_ptr(), nx, ny,
                                                   nz, z_margin, float(lr), byref(loss), stream),
               "gempic_denoiser_train_step")
        return loss.value

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.gempic_denoiser_destroy(self.h)
            self.h = c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def denoiser_params_to_vector(P) -> np.ndarray:
    """Pack a dict of W1, b1, W2, b2, W3, b3 (shapes [3,3,3,ci,co] and [co]) into the library's
    parameter vector (tap, input channel, output channel order)."""
    parts = []
    for l in (1, 2, 3):
        parts.append(np.asarray(P[f"W{l}"], np.float32).reshape(-1))
        parts.append(np.asarray(P[f"b{l}"], np.float32).reshape(-1))
    return np.concatenate(parts)


def denoiser_vector_to_params(v: np.ndarray, hidden: int = 16, cin: int = 3) -> dict:
    shapes = [(cin, hidden), (hidden, hidden), (hidden, cin)]
    P, o = {}, 0
    for l, (ci, co) in enumerate(shapes, start=1):
        n = 27 * ci * co
        P[f"W{l}"] = np.asarray(v[o:o + n], np.float64).reshape(3, 3, 3, ci, co)
        o += n
        P[f"b{l}"] = np.asarray(v[o:o + co], np.float64)
        o += co
    return P
