"""Thin Python binding of ``libboris.so`` (C ABI in ``include/boris.h``).

Argument marshalling only: every step of the demag and LLG path runs in the
CUDA kernels of the library.  Tensors are torch CUDA tensors (device memory
and streams); the library is loaded from this package's directory and its
absence is an error, never a fallback.
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass, field

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libboris.so")

BORIS_OK = 0
STATUS = {0: "OK", -1: "INVALID_ARG", -2: "OOM", -3: "CUDA", -4: "UNSUPPORTED_SIZE", -5: "TIMEOUT",
          -6: "STEP_CONTROL"}
FLAG_F32, FLAG_F64, FLAG_FP16_TC, FLAG_BF16_TC = 0x0, 0x1, 0x2, 0x4
RK4, RKF45 = 0, 1

MU0 = 4e-7 * math.pi
#: gamma = mu0 g muB / hbar with the electron g-factor (Eq. 1, g_rel = 1), m/(A s)
GAMMA = MU0 * 2.00231930436256 * 9.2740100783e-24 / 1.054571817e-34

#: entry points declared in include/boris.h
EXPORTS = ["boris_demag_plan", "boris_multimesh_plan", "boris_plan_multimesh_info", "boris_demag_apply", "boris_demag_apply_f64", "boris_demag_apply_noalloc",
           "boris_demag_adjoint",
           "boris_llg_step", "boris_llg_step_f64", "boris_llg_run_graph", "boris_llg_step_backward", "boris_llg_step_backward_f64", "boris_llg_run_host", "boris_llg_run_rkf45", "boris_energy",
           "boris_energy_terms", "boris_set_field_terms", "boris_demag_plan_pbc",
           "boris_thermal_set_step", "boris_philox4x32_10", "boris_oersted_plan", "boris_oersted_apply",
           "boris_sync_status", "boris_last_error", "boris_plan_padded", "boris_plan_schedule", "boris_plan_device_bytes",
           "boris_profile_enable", "boris_profile_read", "boris_plan_destroy"]
KERNEL_CLASSES = ["x_r2c", "yz_conv", "x_c2r", "llg_stage", "other", "y_fwd", "z_conv", "y_inv", "x_c2r_rk4"]


class BorisError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (STATUS.get(code, "?"), code, msg))
        self.code = code


class LLGParamsC(ctypes.Structure):
    _fields_ = [("Ms_map", ctypes.c_void_p), ("Ms", ctypes.c_double), ("A", ctypes.c_double),
                ("alpha", ctypes.c_double), ("gamma", ctypes.c_double), ("Ku_map", ctypes.c_void_p),
                ("Ku", ctypes.c_double), ("easy", ctypes.c_double * 3), ("Hext", ctypes.c_double * 3),
                ("method", ctypes.c_int), ("tol", ctypes.c_double), ("dt_min", ctypes.c_double),
                ("dt_max", ctypes.c_double)]


DMI_KINDS = {"none": 0, "bulk": 1, "interfacial": 2}


class FieldTermsC(ctypes.Structure):
    _fields_ = [("K2", ctypes.c_double), ("Kc1", ctypes.c_double), ("Kc2", ctypes.c_double),
                ("cubic_e1", ctypes.c_double * 3), ("cubic_e2", ctypes.c_double * 3), ("dmi", ctypes.c_int),
                ("D", ctypes.c_double), ("J1", ctypes.c_double), ("J2", ctypes.c_double),
                ("temperature", ctypes.c_double), ("seed", ctypes.c_ulonglong), ("H_add", ctypes.c_void_p)]


@dataclass
class FieldTerms:
    """Further Table 1 terms and the Eq. 5 surface exchange (boris_field_terms)."""
    K2: float = 0.0
    Kc1: float = 0.0
    Kc2: float = 0.0
    cubic_e1: tuple = (1.0, 0.0, 0.0)
    cubic_e2: tuple = (0.0, 1.0, 0.0)
    dmi: str = "none"
    D: float = 0.0
    J1: float = 0.0
    J2: float = 0.0
    temperature: float = 0.0
    seed: int = 0
    H_add: object = None  # torch CUDA tensor [3][nz][ny][nx] of the plan's precision, or None

    def c(self) -> FieldTermsC:
        t = FieldTermsC()
        t.K2, t.Kc1, t.Kc2 = self.K2, self.Kc1, self.Kc2
        t.cubic_e1 = (ctypes.c_double * 3)(*self.cubic_e1)
        t.cubic_e2 = (ctypes.c_double * 3)(*self.cubic_e2)
        t.dmi = DMI_KINDS[self.dmi]
        t.D, t.J1, t.J2 = self.D, self.J1, self.J2
        t.temperature, t.seed = self.temperature, self.seed
        t.H_add = self.H_add.data_ptr() if self.H_add is not None else None
        return t


_lib = None


def lib():
    """Load libboris.so; raises if it was not built (no CPU fallback exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libboris.so is not built: run __graft_entry__.build() (needs nvcc)")
        L = ctypes.CDLL(LIB_PATH)
        i, d, vp, u = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_uint
        P = ctypes.POINTER
        L.boris_demag_plan.argtypes = [i, i, i, d, d, d, u, vp, P(vp)]
        L.boris_demag_plan_pbc.argtypes = [i, i, i, d, d, d, P(i), u, vp, P(vp)]
        L.boris_demag_apply.argtypes = [vp, vp, vp]
        L.boris_multimesh_plan.argtypes = [i, vp, vp, vp, u, vp, P(vp)]
        L.boris_plan_multimesh_info.argtypes = [vp, P(i)]
        L.boris_demag_apply_f64.argtypes = [vp, vp, vp]
        L.boris_demag_adjoint.argtypes = [vp, vp, vp]
        L.boris_demag_apply_noalloc.argtypes = [vp, vp, vp]
        L.boris_llg_step.argtypes = [vp, vp, P(LLGParamsC), P(d)]
        L.boris_llg_step_f64.argtypes = [vp, vp, P(LLGParamsC), P(d)]
        L.boris_llg_step_backward.argtypes = [vp, vp, P(LLGParamsC), d, vp, vp, vp, vp]
        L.boris_llg_step_backward_f64.argtypes = [vp, vp, P(LLGParamsC), d, vp, vp, vp, vp]
        L.boris_llg_run_host.argtypes = [vp, vp, P(LLGParamsC), d, i]
        L.boris_llg_run_graph.argtypes = [vp, vp, P(LLGParamsC), d, i]
        L.boris_llg_run_rkf45.argtypes = [vp, vp, P(LLGParamsC), P(d), i, P(d)]
        L.boris_energy.argtypes = [vp, vp, P(LLGParamsC), P(d)]
        L.boris_energy_terms.argtypes = [vp, vp, P(LLGParamsC), P(d)]
        L.boris_set_field_terms.argtypes = [vp, P(FieldTermsC)]
        L.boris_thermal_set_step.argtypes = [vp, ctypes.c_ulonglong]
        L.boris_philox4x32_10.argtypes = [vp, vp, vp, i, vp]
        L.boris_oersted_plan.argtypes = [i, i, i, d, d, d, vp, P(vp)]
        L.boris_oersted_apply.argtypes = [vp, vp, vp]
        L.boris_sync_status.argtypes = [vp]
        L.boris_last_error.restype = ctypes.c_char_p
        L.boris_plan_padded.argtypes = [vp, P(i)]
        L.boris_plan_schedule.argtypes = [vp, P(i)]
        L.boris_plan_device_bytes.restype = ctypes.c_size_t
        L.boris_plan_device_bytes.argtypes = [vp]
        L.boris_plan_destroy.argtypes = [vp]
        L.boris_profile_enable.argtypes = [vp, i]
        L.boris_profile_read.argtypes = [vp, P(d), P(ctypes.c_longlong), P(ctypes.c_longlong)]
        for name in EXPORTS:
            if name not in ("boris_last_error", "boris_plan_device_bytes", "boris_plan_destroy"):
                getattr(L, name).restype = i
        L.boris_plan_destroy.restype = None
        _lib = L
    return _lib


def philox4x32_10(ctr, key, stream=None):
    """Device Philox4x32-10 words (boris_philox4x32_10): ctr an int32 CUDA
    tensor [n][4] and key [n][2] holding the 32-bit words; returns [n][4]."""
    import torch
    assert ctr.is_cuda and ctr.dtype == torch.int32 and key.dtype == torch.int32
    ctr, key = ctr.contiguous(), key.contiguous()
    n = ctr.shape[0]
    assert tuple(ctr.shape) == (n, 4) and tuple(key.shape) == (n, 2)
    out = torch.empty((n, 4), dtype=torch.int32, device=ctr.device)
    st = stream if stream is not None else torch.cuda.current_stream().cuda_stream
    check(lib().boris_philox4x32_10(ctr.data_ptr(), key.data_ptr(), out.data_ptr(), n, st))
    return out


def check(rc):
    if rc != BORIS_OK:
        raise BorisError(rc, lib().boris_last_error().decode())
    return rc


@dataclass
class LLGParams:
    Ms: float = 8e5
    A: float = 1.3e-11
    alpha: float = 0.02
    gamma: float = GAMMA
    Ku: float = 0.0
    easy: tuple = (0.0, 0.0, 1.0)
    Hext: tuple = (0.0, 0.0, 0.0)
    method: int = RK4
    tol: float = 1e-5
    dt_min: float = 1e-16
    dt_max: float = 1e-12
    Ms_map: object = None  # torch CUDA tensor [nz][ny][nx] or None
    Ku_map: object = None

    def c(self) -> LLGParamsC:
        p = LLGParamsC()
        p.Ms_map = self.Ms_map.data_ptr() if self.Ms_map is not None else None
        p.Ms = self.Ms
        p.A = self.A
        p.alpha = self.alpha
        p.gamma = self.gamma
        p.Ku_map = self.Ku_map.data_ptr() if self.Ku_map is not None else None
        p.Ku = self.Ku
        p.easy = (ctypes.c_double * 3)(*self.easy)
        p.Hext = (ctypes.c_double * 3)(*self.Hext)
        p.method = self.method
        p.tol = self.tol
        p.dt_min = self.dt_min
        p.dt_max = self.dt_max
        return p


def _ptr(t, dtype, shape=None):
    import torch
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError("expected dtype %s, got %s" % (dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError("expected shape %s, got %s" % (tuple(shape), tuple(t.shape)))
    return ctypes.c_void_p(t.data_ptr())


class Plan:
    """A demag + LLG plan for an nx x ny x nz mesh of dx x dy x dz cells."""

    def __init__(self, nx, ny, nz, dx, dy, dz, fp64: bool = False, stream=None, tc: str | None = None,
                 images=None):
        """images: periodic images per axis (x, y, z), 0 for an open axis
        (boris_demag_plan_pbc); None for no periodic axis."""
        import torch
        self.shape = (nx, ny, nz)
        self.cell = (dx, dy, dz)
        self.fp64 = fp64
        self.dtype = torch.float64 if fp64 else torch.float32
        st = stream if stream is not None else torch.cuda.current_stream()
        self.stream = st
        h = ctypes.c_void_p()
        flags = FLAG_F64 if fp64 else FLAG_F32
        if tc is not None:
            flags |= {"fp16": FLAG_FP16_TC, "bf16": FLAG_BF16_TC}[tc]
        self.tc = tc
        self.images = tuple(images) if images is not None else (0, 0, 0)
        if images is not None:
            im = (ctypes.c_int * 3)(*[int(v) for v in images])
            check(lib().boris_demag_plan_pbc(nx, ny, nz, dx, dy, dz, im, flags, ctypes.c_void_p(st.cuda_stream),
                                             ctypes.byref(h)))
        else:
            check(lib().boris_demag_plan(nx, ny, nz, dx, dy, dz, flags, ctypes.c_void_p(st.cuda_stream),
                                         ctypes.byref(h)))
        self._h = h

    @property
    def field_shape(self):
        nx, ny, nz = self.shape
        return (3, nz, ny, nx)

    @property
    def map_shape(self):
        nx, ny, nz = self.shape
        return (nz, ny, nx)

    def padded(self):
        out = (ctypes.c_int * 3)()
        check(lib().boris_plan_padded(self._h, out))
        return tuple(out)

    def schedule(self):
        """(kind, CTAs per cluster, threads, shared bytes) of the fused y-z pass."""
        out = (ctypes.c_int * 4)()
        check(lib().boris_plan_schedule(self._h, out))
        return tuple(out)

    def device_bytes(self) -> int:
        return int(lib().boris_plan_device_bytes(self._h))

    def apply(self, M, out=None):
        """H = -N * M (device tensors [3][nz][ny][nx])."""
        import torch
        if out is None:
            out = torch.empty(self.field_shape, dtype=self.dtype, device=M.device)
        fn = lib().boris_demag_apply_f64 if self.fp64 else lib().boris_demag_apply
        check(fn(self._h, _ptr(M, self.dtype, self.field_shape), _ptr(out, self.dtype, self.field_shape)))
        return out

    def adjoint(self, gH, out=None):
        import torch
        if out is None:
            out = torch.empty(self.field_shape, dtype=self.dtype, device=gH.device)
        if self.fp64:
            raise NotImplementedError("adjoint is FP32")
        check(lib().boris_demag_adjoint(self._h, _ptr(gH, self.dtype, self.field_shape),
                                        _ptr(out, self.dtype, self.field_shape)))
        return out

    def _params(self, prm: LLGParams):
        for mp in (prm.Ms_map, prm.Ku_map):
            if mp is not None:
                _ptr(mp, self.dtype, self.map_shape)
        return prm.c()

    def llg_step(self, m, prm: LLGParams, dt: float) -> float:
        """Advance m in place by one RK4 step (returns dt) or one accepted RKF45 step
        (returns the controller's next dt)."""
        c = self._params(prm)
        h = ctypes.c_double(dt)
        fn = lib().boris_llg_step_f64 if self.fp64 else lib().boris_llg_step
        check(fn(self._h, _ptr(m, self.dtype, self.field_shape), ctypes.byref(c), ctypes.byref(h)))
        return h.value

    def llg_step_backward(self, m_in, prm: LLGParams, dt: float, g_out, g_in=None, g_Ms=None, g_Ku=None):
        """g_in = dL/dm_in of one RK4 step from g_out = dL/dm_out; ADDS dL/dMs and
        dL/dKu into g_Ms / g_Ku when given (tensors [nz][ny][nx])."""
        import torch
        if g_in is None:
            g_in = torch.empty_like(g_out)
        c = self._params(prm)
        gms = _ptr(g_Ms, self.dtype, self.map_shape) if g_Ms is not None else None
        gku = _ptr(g_Ku, self.dtype, self.map_shape) if g_Ku is not None else None
        fn = lib().boris_llg_step_backward_f64 if self.fp64 else lib().boris_llg_step_backward
        check(fn(self._h, _ptr(m_in, self.dtype, self.field_shape), ctypes.byref(c), float(dt),
                 _ptr(g_out, self.dtype, self.field_shape), _ptr(g_in, self.dtype, self.field_shape), gms, gku))
        return g_in

    def llg_run_graph(self, m, prm: LLGParams, dt: float, nsteps: int):
        """nsteps RK4 steps replayed from a captured CUDA graph (FP32 plans)."""
        c = self._params(prm)
        check(lib().boris_llg_run_graph(self._h, _ptr(m, self.dtype, self.field_shape), ctypes.byref(c), float(dt),
                                        int(nsteps)))

    def llg_run_rkf45(self, m, prm: LLGParams, dt: float, nsteps: int):
        """nsteps accepted RKF45 steps with device-side step control (FP32 plans);
        one synchronisation at the end.  Returns (next dt, simulated time)."""
        c = self._params(prm)
        h, t = ctypes.c_double(dt), ctypes.c_double(0.0)
        check(lib().boris_llg_run_rkf45(self._h, _ptr(m, self.dtype, self.field_shape), ctypes.byref(c),
                                        ctypes.byref(h), int(nsteps), ctypes.byref(t)))
        return h.value, t.value

    def llg_run_host(self, m_host, prm: LLGParams, dt: float, nsteps: int):
        """m_host: CPU float32 tensor (pinned for speed), updated in place."""
        if m_host.is_cuda or m_host.dtype.itemsize != 4 or not m_host.is_contiguous():
            raise ValueError("expected a contiguous CPU float32 tensor")
        c = self._params(prm)
        check(lib().boris_llg_run_host(self._h, ctypes.c_void_p(m_host.data_ptr()), ctypes.byref(c),
                                       float(dt), int(nsteps)))

    def energy(self, m, prm: LLGParams):
        c = self._params(prm)
        out = (ctypes.c_double * 4)()
        check(lib().boris_energy(self._h, _ptr(m, self.dtype, self.field_shape), ctypes.byref(c), out))
        return tuple(out)

    def set_field_terms(self, terms: "FieldTerms | None"):
        """Set (or with None clear) the further field terms of the plan."""
        if terms is None:
            check(lib().boris_set_field_terms(self._h, None))
        else:
            c = terms.c()
            check(lib().boris_set_field_terms(self._h, ctypes.byref(c)))

    def thermal_set_step(self, step: int):
        check(lib().boris_thermal_set_step(self._h, int(step)))

    def energy_terms(self, m, prm: LLGParams):
        """(E_demag, E_exchange, E_anisotropy, E_Zeeman, E_DMI) in J."""
        c = self._params(prm)
        out = (ctypes.c_double * 5)()
        check(lib().boris_energy_terms(self._h, _ptr(m, self.dtype, self.field_shape), ctypes.byref(c), out))
        return tuple(out)

    def profile(self, on: bool):
        check(lib().boris_profile_enable(self._h, 1 if on else 0))

    def profile_read(self):
        """{kernel class: (ms, timed launches)}, total launches since the last read."""
        ms = (ctypes.c_double * len(KERNEL_CLASSES))()
        cnt = (ctypes.c_longlong * len(KERNEL_CLASSES))()
        tot = ctypes.c_longlong()
        check(lib().boris_profile_read(self._h, ms, cnt, ctypes.byref(tot)))
        return {k: (ms[i], cnt[i]) for i, k in enumerate(KERNEL_CLASSES)}, tot.value

    def sync_status(self):
        return check(lib().boris_sync_status(self._h))

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().boris_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class OerstedPlan:
    """Oersted field H = K * J of a current density on an nx x ny x nz mesh
    (boris_oersted_plan / boris_oersted_apply), FP32."""

    def __init__(self, nx, ny, nz, dx, dy, dz, stream=None):
        import torch
        self.shape = (nx, ny, nz)
        self.dtype = torch.float32
        st = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        check(lib().boris_oersted_plan(nx, ny, nz, dx, dy, dz, ctypes.c_void_p(st.cuda_stream), ctypes.byref(h)))
        self._h = h

    @property
    def field_shape(self):
        nx, ny, nz = self.shape
        return (3, nz, ny, nx)

    def apply(self, J, out=None):
        import torch
        if out is None:
            out = torch.empty(self.field_shape, dtype=torch.float32, device=J.device)
        check(lib().boris_oersted_apply(self._h, _ptr(J, torch.float32, self.field_shape),
                                        _ptr(out, torch.float32, self.field_shape)))
        return out

    def profile(self, on: bool):
        check(lib().boris_profile_enable(self._h, 1 if on else 0))

    def profile_read(self):
        ms = (ctypes.c_double * len(KERNEL_CLASSES))()
        cnt = (ctypes.c_longlong * len(KERNEL_CLASSES))()
        tot = ctypes.c_longlong()
        check(lib().boris_profile_read(self._h, ms, cnt, ctypes.byref(tot)))
        return {k: (ms[i], cnt[i]) for i, k in enumerate(KERNEL_CLASSES)}, tot.value

    def sync_status(self):
        return check(lib().boris_sync_status(self._h))

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().boris_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MultiPlan(Plan):
    """Multi-mesh plan (Eq. 4): layers[i] = (nx, ny, nz) cells of size
    cells[i] = (hx, hy, hz) with lower corner origins[i] = (x, y, z), m.
    Fields are the layers' SoA [3][nz][ny][nx] arrays concatenated in layer
    order (flat tensors of 3 * total cells); maps likewise (total cells)."""

    def __init__(self, layers, cells, origins, stream=None):
        import numpy as np
        import torch
        self.layers = [tuple(int(v) for v in l) for l in layers]
        self.fp64 = False
        self.tc = None
        self.dtype = torch.float32
        self.total = sum(nx * ny * nz for nx, ny, nz in self.layers)
        st = stream if stream is not None else torch.cuda.current_stream()
        self.stream = st
        nxyz = np.ascontiguousarray(np.array(self.layers, dtype=np.int32).reshape(-1))
        hxyz = np.ascontiguousarray(np.array(cells, dtype=np.float64).reshape(-1))
        org = np.ascontiguousarray(np.array(origins, dtype=np.float64).reshape(-1))
        h = ctypes.c_void_p()
        check(lib().boris_multimesh_plan(len(self.layers), nxyz.ctypes.data_as(ctypes.c_void_p),
                                         hxyz.ctypes.data_as(ctypes.c_void_p), org.ctypes.data_as(ctypes.c_void_p),
                                         FLAG_F32, ctypes.c_void_p(st.cuda_stream), ctypes.byref(h)))
        self._h = h
        self.shape = None

    @property
    def field_shape(self):
        return (3 * self.total,)

    @property
    def map_shape(self):
        return (self.total,)

    def info(self):
        """(z planes, distinct inter-plane spectra, frame nx, frame ny)."""
        out = (ctypes.c_int * 4)()
        check(lib().boris_plan_multimesh_info(self._h, out))
        return tuple(out)
