"""Thin ctypes binding of libwave (include/wave.h).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of libwave.so.  torch supplies device memory (workspaces are uint8
tensors) and the current CUDA stream.  Importing this module raises if the
library has not been built; nothing here falls back to CPU code.

Grid shapes are C order, slowest axis first: (ny, nx) in 2D, (nz, ny, nx) in
3D; cell indices are flat C-order indices.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass
from typing import List, Optional, Sequence

import torch

from . import build as _build

if not os.path.exists(_build.LIB):
    raise ImportError(
        f"libwave.so is not built ({_build.LIB}); run `python -c \"import __graft_entry__ as g; g.build()\"`")

_lib = C.CDLL(_build.LIB)

# ---- enums (include/wave.h) ------------------------------------------------
PHYSICS = {"velocity": 0, "density": 1}
BC = {"dirichlet": 0, "neumann": 1}
STORAGE = {"f32": 0, "bf16": 1, "f16": 2}
OBJECTIVE = {"l2": 0, "patch": 1}
MODE = {"superposition": 0, "exact": 1, "symmetric": 2, "reverse": 3}
GRAD_WRT = {"mass": 0, "param": 1}
WAVELET = {"ricker": 0, "sine_burst": 1}


class GridDesc(C.Structure):
    _fields_ = [("ndim", C.c_int32), ("order", C.c_int32), ("n", C.c_int64 * 3), ("h", C.c_double),
                ("dt", C.c_double), ("physics", C.c_int32), ("bc", C.c_int32), ("storage", C.c_int32),
                ("kahan", C.c_int32)]


class ShotDesc(C.Structure):
    _fields_ = [("src_cell", C.c_int64), ("nt", C.c_int32), ("nrec", C.c_int32), ("wavelet_dev", C.c_void_p),
                ("rec_cells_dev", C.c_void_p), ("observed_dev", C.c_void_p), ("traces_dev", C.c_void_p)]


class GradOpts(C.Structure):
    _fields_ = [("objective", C.c_int32), ("mode", C.c_int32), ("batched", C.c_int32), ("grad_wrt", C.c_int32),
                ("patch_sign", C.c_double), ("k", C.c_double), ("k_ratio", C.c_double)]


_vp = C.c_void_p
_sz = C.c_size_t
_i32 = C.c_int32
_st = C.c_int


def _sig(name, res, *args):
    f = getattr(_lib, name)
    f.restype = res
    f.argtypes = list(args)
    return f


_status_string = _sig("wave_status_string", C.c_char_p, _st)
_last_error = _sig("wave_last_error", C.c_char_p)
_launch_count = _sig("wave_launch_count", C.c_uint64)
_cfl_dt = _sig("wave_cfl_dt", C.c_double, _i32, _i32, C.c_double, C.c_double, C.c_double)
_wavelet = _sig("wave_wavelet", _st, _i32, C.c_double, _i32, C.c_double, C.c_double, _i32, _vp, _vp)
_model_ws = _sig("wave_model_workspace_size", _st, C.POINTER(GridDesc), C.POINTER(_sz))
_model_create = _sig("wave_model_create", _st, C.POINTER(GridDesc), _vp, _vp, _sz, _vp, C.POINTER(_vp))
_model_destroy = _sig("wave_model_destroy", _st, _vp)
_model_set_block = _sig("wave_model_set_block", _st, _vp, C.c_int64)
_model_get_block = _sig("wave_model_get_block", _st, _vp, C.POINTER(C.c_int64))
_model_set_tiling = _sig("wave_model_set_tiling", _st, _vp, C.c_int64, _i32, _i32, _i32)
_model_set_schedule = _sig("wave_model_set_schedule", _st, _vp, _i32)
_model_check = _sig("wave_model_check", _st, _vp, _vp)
_model_set_param = _sig("wave_model_set_param", _st, _vp, _vp, _vp)
_model_set_debug = _sig("wave_model_set_debug", _st, _vp, _i32, C.c_int64)
_model_pitch = _sig("wave_model_pitch", _st, _vp, C.POINTER(C.c_int64))
_step = _sig("wave_step", _st, _vp, _i32, C.POINTER(_vp), C.POINTER(_vp), C.POINTER(C.c_float), _vp, _vp, _vp)
_fwd_ws = _sig("wave_forward_workspace_size", _st, _vp, C.POINTER(ShotDesc), _i32, C.POINTER(_sz))
_forward = _sig("wave_forward", _st, _vp, C.POINTER(ShotDesc), _i32, _vp, _vp, _vp, _sz, _vp)
_grad_ws = _sig("wave_gradient_workspace_size", _st, _vp, C.POINTER(ShotDesc), _i32, C.POINTER(GradOpts),
                C.POINTER(_sz))
_adjoint_sensitivity = _sig("wave_adjoint_sensitivity", _st, _vp, C.POINTER(ShotDesc), _i32, C.POINTER(GradOpts),
                            _vp, _vp, _vp, _vp, _vp, _sz, _vp)


class GradMetrics(C.Structure):
    _fields_ = [("misfit", C.c_double), ("k", C.c_double), ("grad_l2", C.c_double), ("forward_ms", C.c_double),
                ("adjoint_ms", C.c_double), ("total_ms", C.c_double), ("step_bytes", C.c_double),
                ("cell_updates", C.c_double), ("step_launches", C.c_int64)]


_set_metrics = _sig("wave_model_set_metrics", _st, _vp, _i32)
_metrics_read = _sig("wave_gradient_metrics_read", _st, _vp, C.POINTER(GradMetrics))
_timing_enable = _sig("wave_timing_enable", _st, _i32)
_timing_read = _sig("wave_timing_read", _st, C.POINTER(C.c_double), C.POINTER(C.c_uint64), C.POINTER(C.c_double))
_misfit_scratch = _sig("wave_misfit_scratch_size", _sz, C.c_int64)
_misfit = _sig("misfit", _st, _vp, _vp, C.c_int64, C.c_double, C.c_double, _vp, _vp, _sz, _vp)


class WaveError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = _status_string(status).decode()
        extra = _last_error().decode() if status == 4 else ""
        super().__init__(f"{where}: {msg} ({status}) {extra}".strip())
        self.status = status


def _check(status: int, where: str):
    if status != 0:
        raise WaveError(status, where)


def launch_count() -> int:
    """Kernels launched by libwave in this process."""
    return int(_launch_count())


def timing_enable(on: bool = True):
    """Bracket every step-kernel launch with CUDA events (resets the counters)."""
    _check(_timing_enable(int(bool(on))), "wave_timing_enable")


def timing_read():
    """(total step-kernel ms, timed launches, algorithmic bytes) since enabling."""
    ms, n, b = C.c_double(0), C.c_uint64(0), C.c_double(0)
    _check(_timing_read(C.byref(ms), C.byref(n), C.byref(b)), "wave_timing_read")
    return float(ms.value), int(n.value), float(b.value)


def status_string(status: int) -> str:
    return _status_string(status).decode()


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return _vp(s.cuda_stream)


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else _vp(t.data_ptr())


def _workspace(nbytes: int, device) -> torch.Tensor:
    # torch's allocator returns 512-byte aligned blocks; one extra byte keeps
    # zero-size requests valid.
    return torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device)


def cfl_dt(ndim: int, order: int, h: float, vmax: float, fraction: float = 0.5) -> float:
    dt = _cfl_dt(ndim, order, h, vmax, fraction)
    if dt <= 0:
        raise ValueError("invalid arguments to cfl_dt")
    return dt


def wavelet(kind: str, freq: float, dt: float, nt: int, nc: int = 2, psi0: float = 1.0,
            device="cuda", stream=None) -> torch.Tensor:
    out = torch.empty(nt + 1, dtype=torch.float32, device=device)
    _check(_wavelet(WAVELET[kind], freq, nc, psi0, dt, nt, _ptr(out), _stream(stream)), "wave_wavelet")
    return out


def misfit(syn: torch.Tensor, obs: Optional[torch.Tensor], dt: float, weight: float = 1.0,
           stream=None) -> torch.Tensor:
    """0.5 * weight * dt * sum (syn - obs)^2 in FP64 (device scalar)."""
    syn = syn.contiguous()
    if obs is not None:
        obs = obs.contiguous()
        if obs.numel() != syn.numel():
            raise ValueError("syn and obs differ in size")
    out = torch.empty(1, dtype=torch.float64, device=syn.device)
    scratch = _workspace(_misfit_scratch(syn.numel()), syn.device)
    _check(_misfit(_ptr(syn), _ptr(obs), syn.numel(), dt, weight, _ptr(out), _ptr(scratch),
                   scratch.numel(), _stream(stream)), "misfit")
    return out


@dataclass
class Shot:
    """A point source (flat cell index + wavelet samples psi(n dt), n=0..nt)
    with receivers (flat indices) and, for gradients, observed traces
    [nrec, nt+1] (None = zero data)."""
    src: int
    wavelet: torch.Tensor
    rec: torch.Tensor
    observed: Optional[torch.Tensor] = None

    @property
    def nt(self) -> int:
        return int(self.wavelet.numel()) - 1

    @property
    def nrec(self) -> int:
        return int(self.rec.numel())


def _shot_descs(shots: Sequence[Shot], traces: Optional[List[torch.Tensor]] = None):
    arr = (ShotDesc * len(shots))()
    for i, s in enumerate(shots):
        if s.wavelet.dtype != torch.float32 or not s.wavelet.is_cuda:
            raise TypeError("wavelet must be a CUDA float32 tensor")
        if s.rec.dtype != torch.int64 or not s.rec.is_cuda:
            raise TypeError("receivers must be a CUDA int64 tensor")
        if s.observed is not None and (s.observed.dtype != torch.float32 or not s.observed.is_cuda or
                                       tuple(s.observed.shape) != (s.nrec, s.nt + 1) or
                                       not s.observed.is_contiguous()):
            raise TypeError("observed must be a contiguous CUDA float32 [nrec, nt+1] tensor")
        if not s.wavelet.is_contiguous() or not s.rec.is_contiguous():
            raise TypeError("wavelet and receivers must be contiguous")
        arr[i].src_cell = int(s.src)
        arr[i].nt = s.nt
        arr[i].nrec = s.nrec
        arr[i].wavelet_dev = s.wavelet.data_ptr()
        arr[i].rec_cells_dev = s.rec.data_ptr() if s.nrec else None
        arr[i].observed_dev = s.observed.data_ptr() if s.observed is not None else None
        arr[i].traces_dev = traces[i].data_ptr() if traces is not None and s.nrec else None
    return arr


class Model:
    """A discretised medium resident on the GPU (wave_model)."""

    def __init__(self, param: torch.Tensor, h: float, dt: float, order: int = 2, physics: str = "velocity",
                 bc: str = "dirichlet", storage: str = "f32", kahan: bool = False, stream=None):
        if not param.is_cuda or param.dtype != torch.float32:
            raise TypeError("param must be a CUDA float32 tensor")
        self.param = param.contiguous()
        self.shape = tuple(self.param.shape)
        nd = len(self.shape)
        if nd not in (2, 3):
            raise ValueError("2D or 3D grids only")
        d = GridDesc()
        d.ndim = nd
        d.order = order
        rev = list(reversed(self.shape)) + [1] * (3 - nd)
        for i in range(3):
            d.n[i] = int(rev[i])
        d.h, d.dt = float(h), float(dt)
        d.physics, d.bc, d.storage = PHYSICS[physics], BC[bc], STORAGE[storage]
        d.kahan = int(bool(kahan))
        self.desc = d
        self.h, self.dt, self.order, self.physics, self.bc = h, dt, order, physics, bc
        self.storage, self.kahan = storage, kahan
        self.cta_order = 1   # the library's default launch order (plane-major)
        nbytes = _sz(0)
        _check(_model_ws(C.byref(d), C.byref(nbytes)), "wave_model_workspace_size")
        self._ws = _workspace(nbytes.value, self.param.device)
        h_ = _vp()
        _check(_model_create(C.byref(d), _ptr(self.param), _ptr(self._ws), self._ws.numel(), _stream(stream),
                             C.byref(h_)), "wave_model_create")
        self._h = h_
        self._fws = None
        self._gws = None
        self.grad_norm = None   # device FP64 ||grad||_2 of the last gradient call

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            _model_destroy(h)
            self._h = None

    @property
    def ncells(self) -> int:
        n = 1
        for s in self.shape:
            n *= s
        return n

    def set_block(self, zblock: int):
        _check(_model_set_block(self._h, int(zblock)), "wave_model_set_block")

    def set_tiling(self, zblock: int, tile_rows: int = 8, ring_depth: int = 3, pipeline: int = 0):
        _check(_model_set_tiling(self._h, int(zblock), int(tile_rows), int(ring_depth), int(pipeline)),
               "wave_model_set_tiling")

    def set_schedule(self, cta_order: int = 1):
        """Launch order of the 3D step CTAs: 0 z-block fastest, 1 plane-major (wave_model_set_schedule)."""
        _check(_model_set_schedule(self._h, int(cta_order)), "wave_model_set_schedule")
        self.cta_order = int(cta_order)

    def set_metrics(self, on: bool = True):
        """Record per-pass CUDA events in later gradient calls (wave_model_set_metrics)."""
        _check(_set_metrics(self._h, int(bool(on))), "wave_model_set_metrics")

    def metrics(self) -> dict:
        """Figures of the last gradient call (waits for it): misfit, k, grad_l2,
        forward_ms, adjoint_ms, total_ms, step_bytes, cell_updates,
        step_launches.  Raises WaveError(WAVE_ENONFINITE) on a NaN/Inf result."""
        m = GradMetrics()
        _check(_metrics_read(self._h, C.byref(m)), "wave_gradient_metrics_read")
        return {n: getattr(m, n) for n, _ in GradMetrics._fields_}

    def check(self, stream=None) -> int:
        """Wait for the stream; WAVE_ETIMEOUT (5) if a bounded device wait gave up,
        WAVE_EUNSTABLE (2) / WAVE_ENONFINITE (6) for an unstable or non-finite
        parameter of the last set_param."""
        return int(_model_check(self._h, _stream(stream)))

    def set_param(self, param: torch.Tensor, stream=None):
        """Replace the parameter grid (same shape) without a host wait; check()
        reports an unstable or non-finite value."""
        if not param.is_cuda or param.dtype != torch.float32 or tuple(param.shape) != self.shape:
            raise TypeError("param must be a CUDA float32 tensor of the model's shape")
        self.param = param.contiguous()
        _check(_model_set_param(self._h, _ptr(self.param), _stream(stream)), "wave_model_set_param")

    def set_debug(self, stall_pipeline: bool, wait_limit_cycles: int = 4_000_000_000):
        _check(_model_set_debug(self._h, int(bool(stall_pipeline)), int(wait_limit_cycles)), "wave_model_set_debug")

    def get_block(self) -> int:
        v = C.c_int64(0)
        _check(_model_get_block(self._h, C.byref(v)), "wave_model_get_block")
        return int(v.value)

    @property
    def pitch(self) -> int:
        """Row pitch of the resident grids (nx rounded up to 128 cells)."""
        v = C.c_int64(0)
        _check(_model_pitch(self._h, C.byref(v)), "wave_model_pitch")
        return int(v.value)

    def pitched_shape(self) -> tuple:
        return tuple(self.shape[:-1]) + (self.pitch,)

    def step(self, cur: Sequence[torch.Tensor], prev: Sequence[torch.Tensor], acc: Optional[torch.Tensor] = None,
             comp: Optional[torch.Tensor] = None, acc_sign: Optional[Sequence[float]] = None, stream=None):
        """One leapfrog step of len(cur) fields (wave_step): prev[f] <- u^{n+1};
        acc += acc_sign[f] (u^{n+1} - u^n)^2 if acc is given.  All grids are
        pitched ([..., pitch], see pitched_shape) and contiguous."""
        if len(cur) != len(prev) or not 1 <= len(cur) <= 32:
            raise ValueError("cur and prev need the same number (1..32) of fields")
        shp = self.pitched_shape()
        level_dtype = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}[self.storage]
        for t, dt in [(t, level_dtype) for t in list(cur) + list(prev)] + \
                [(t, torch.float32) for t in (acc, comp) if t is not None]:
            if not t.is_cuda or not t.is_contiguous() or tuple(t.shape) != shp or t.dtype != dt:
                raise ValueError(f"grids must be contiguous CUDA {dt} tensors of shape {shp}")
        n = len(cur)
        ca = (_vp * n)(*[t.data_ptr() for t in cur])
        pa = (_vp * n)(*[t.data_ptr() for t in prev])
        sg = (C.c_float * n)(*[float(v) for v in acc_sign]) if acc_sign is not None else None
        _check(_step(self._h, n, ca, pa, sg, _ptr(acc), _ptr(comp), _stream(stream)), "wave_step")

    def _ensure(self, attr, nbytes):
        ws = getattr(self, attr)
        if ws is None or ws.numel() < nbytes:
            ws = _workspace(nbytes, self.param.device)
            setattr(self, attr, ws)
        return ws

    def forward(self, shots: Sequence[Shot], init: Optional[torch.Tensor] = None, return_final: bool = False,
                stream=None):
        """Traces [nrec, nt+1] per shot (levels 0..nt), and optionally the last
        shot's final levels (u^N, u^{N+1}) as a [2, *shape] tensor."""
        dev = self.param.device
        traces = [torch.empty((s.nrec, s.nt + 1), dtype=torch.float32, device=dev) for s in shots]
        arr = _shot_descs(shots, traces)
        nbytes = _sz(0)
        _check(_fwd_ws(self._h, arr, len(shots), C.byref(nbytes)), "wave_forward_workspace_size")
        ws = self._ensure("_fws", nbytes.value)
        final = torch.empty((2,) + self.shape, dtype=torch.float32, device=dev) if return_final else None
        if init is not None:
            init = init.contiguous().to(torch.float32)
            if tuple(init.shape) != (2,) + self.shape:
                raise ValueError("init must be [2, *shape]")
        _check(_forward(self._h, arr, len(shots), _ptr(init), _ptr(final), _ptr(ws), ws.numel(), _stream(stream)),
               "wave_forward")
        return (traces, final) if return_final else traces

    def gradient(self, shots: Sequence[Shot], objective: str = "l2", k: Optional[float] = None,
                 k_ratio: Optional[float] = None, mode: str = "superposition", batched: bool = False,
                 grad_wrt: str = "mass", patch_sign: float = 1.0, stream=None, out: Optional[torch.Tensor] = None):
        """Algorithm 1.  Returns (grad [*shape] float32, misfit [1] float64, k [1] float64);
        self.grad_norm receives ||grad||_2 (FP64 device reduction, [1] float64).

        mode: "superposition" (Algorithm 1), "exact" (adjoint over the stored
        forward history), "symmetric" (mean of the +k and -k superposition
        results: exact, two more grids) or "reverse" (u reconstructed backward
        beside the adjoint field: exact, two more grids, k returned as 0)."""
        dev = self.param.device
        o = GradOpts()
        o.objective, o.mode, o.batched, o.grad_wrt = OBJECTIVE[objective], MODE[mode], int(bool(batched)), \
            GRAD_WRT[grad_wrt]
        o.patch_sign = float(patch_sign)
        o.k = float(k) if k is not None else 0.0
        o.k_ratio = float(k_ratio) if k_ratio is not None else 0.0
        arr = _shot_descs(shots)
        nbytes = _sz(0)
        _check(_grad_ws(self._h, arr, len(shots), C.byref(o), C.byref(nbytes)), "wave_gradient_workspace_size")
        ws = self._ensure("_gws", nbytes.value)
        grad = out if out is not None else torch.empty(self.shape, dtype=torch.float32, device=dev)
        mis = torch.empty(1, dtype=torch.float64, device=dev)
        kd = torch.empty(1, dtype=torch.float64, device=dev)
        norm = torch.empty(1, dtype=torch.float64, device=dev)
        _check(_adjoint_sensitivity(self._h, arr, len(shots), C.byref(o), _ptr(grad), _ptr(mis), _ptr(kd),
                                    _ptr(norm), _ptr(ws), ws.numel(), _stream(stream)), "wave_adjoint_sensitivity")
        self.grad_norm = norm
        return grad, mis, kd
