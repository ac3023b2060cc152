"""Python face of the CUDA CBS library: plans, sources and solves on torch device tensors.

Torch supplies device memory and the stream; every computation runs in libcbs.so through
the C ABI (include/cbs.h).  Fields are torch.complex64 tensors of shape (3, nz, ny, nx) on
the plan's device; permittivity and gradient are float32 (nz, ny, nx).
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np
import torch

from . import _lib as L


@dataclass
class PlaneWave:
    """Current sheet on plane z_plane (-1: first interior plane) launching pol exp(ik|z - z_s|)."""
    pol: Sequence[complex] = (1.0, 0.0, 0.0)
    z_plane: int = -1


@dataclass
class PointSource:
    """Raw source value pol at voxel r0 = (x, y, z); a dipole p is pol = p / pitch^3."""
    r0: Sequence[int]
    pol: Sequence[complex] = (1.0, 0.0, 0.0)


@dataclass
class UserSource:
    """Arbitrary source S, complex64 (3, nz, ny, nx) on the device."""
    S: torch.Tensor


@dataclass
class Stats:
    iters: int
    rel_resid: float
    resid0: float
    seconds: float
    status: int

    @property
    def converged(self) -> bool:
        return self.status == L.CBS_OK


def _stats(s: L.cbs_stats) -> Stats:
    return Stats(s.iters, s.rel_resid, s.resid0, s.seconds, s.status)


def _ptr(t: torch.Tensor) -> int:
    return t.data_ptr()


def _field_like(shape, device) -> torch.Tensor:
    nz, ny, nx = shape
    return torch.empty((3, nz, ny, nx), dtype=torch.complex64, device=device)


class CBSPlan:
    """A solver for one grid: owns the potential, the k-space workspace and the launch plan."""

    def __init__(self, nx: int, ny: int, nz: int, pitch: float, lam: float, n_bg: float = 1.0,
                 pad_lo=(0, 0, 0), pad_hi=None, tol: float = 1e-6, max_iter: int = 100000,
                 check_every: int = 32, device=None, stream: Optional[torch.cuda.Stream] = None,
                 layer_round_trip: float = 0.0, layer_power: float = 0.0, layer_corner_max: bool = False):
        """Absorbing layers: layer_round_trip (the amplitude a normally incident plane wave keeps
        after crossing a layer and back; 0 selects 1e-4), layer_power (ramp exponent; 0 selects
        2) and layer_corner_max (where layers overlap the largest applies instead of the sum);
        see cbs_plan_desc in include/cbs.h."""
        self.lib = L.lib()
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        if pad_hi is None:
            pad_hi = pad_lo
        self.shape = (nz, ny, nx)
        self.nx, self.ny, self.nz = nx, ny, nz
        self.pitch, self.lam, self.n_bg = pitch, lam, n_bg
        self.pad_lo, self.pad_hi = tuple(pad_lo), tuple(pad_hi)
        with torch.cuda.device(self.device):
            s = stream if stream is not None else torch.cuda.current_stream(self.device)
            d = L.cbs_plan_desc(nx, ny, nz, pitch, lam, n_bg, (ctypes.c_int * 3)(*pad_lo),
                                (ctypes.c_int * 3)(*pad_hi), tol, max_iter, check_every,
                                ctypes.c_void_p(s.cuda_stream), float(layer_round_trip), float(layer_power),
                                1 if layer_corner_max else 0)
            h = ctypes.c_void_p()
            L.check(self.lib.cbs_plan(ctypes.byref(h), ctypes.byref(d)))
        self.handle = h
        self.stream = s

    # -- lifetime --------------------------------------------------------------------------
    def close(self):
        if getattr(self, "handle", None):
            self.lib.cbs_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- set-up ----------------------------------------------------------------------------
    def _check_field(self, E: torch.Tensor, name: str):
        nz, ny, nx = self.shape
        if E.dtype != torch.complex64 or tuple(E.shape) != (3, nz, ny, nx) or not E.is_contiguous() \
                or E.device != self.device:
            raise ValueError(f"{name} must be a contiguous complex64 (3, {nz}, {ny}, {nx}) tensor on {self.device}")

    def set_permittivity(self, eps: torch.Tensor):
        if eps.dtype != torch.float32 or tuple(eps.shape) != self.shape or not eps.is_contiguous() \
                or eps.device != self.device:
            raise ValueError(f"eps must be a contiguous float32 {self.shape} tensor on {self.device}")
        self._eps = eps
        L.check(self.lib.cbs_set_permittivity(self.handle, ctypes.c_void_p(_ptr(eps))))

    def splitting(self):
        k0 = ctypes.c_double()
        ep = ctypes.c_double()
        L.check(self.lib.cbs_get_splitting(self.handle, ctypes.byref(k0), ctypes.byref(ep)))
        return k0.value, ep.value

    def set_solver(self, tol: float, max_iter: int, check_every: int = 32):
        L.check(self.lib.cbs_set_solver(self.handle, tol, max_iter, check_every))

    def set_profiling(self, on: bool):
        L.check(self.lib.cbs_set_profiling(self.handle, 1 if on else 0))

    def set_time_limit(self, seconds: float):
        """Wall-clock limit of later solves (0: none); checked after each block of
        check_every iterations, a solve past it ends with status CBS_ERR_TIME_LIMIT."""
        L.check(self.lib.cbs_set_time_limit(self.handle, float(seconds)))

    def pass_times(self, reset: bool = False):
        """{pass name: (summed ms, timed launches)} since the last reset."""
        ms = (ctypes.c_double * 5)()
        n = (ctypes.c_longlong * 5)()
        L.check(self.lib.cbs_pass_times(self.handle, ctypes.byref(ms), ctypes.byref(n), 1 if reset else 0))
        return {name: (ms[i], n[i]) for i, name in enumerate(L.PASS_NAMES)}

    # -- solves ----------------------------------------------------------------------------
    def _source(self, src, warm: bool) -> L.cbs_source:
        s = L.cbs_source()
        s.warm_start = int(warm)
        s.z_plane = -1
        if isinstance(src, PlaneWave):
            s.kind = L.CBS_SRC_PLANE_WAVE
            pol = src.pol
            s.z_plane = src.z_plane
        elif isinstance(src, PointSource):
            s.kind = L.CBS_SRC_POINT
            pol = src.pol
            for i in range(3):
                s.r0[i] = int(src.r0[i])
        elif isinstance(src, UserSource):
            self._check_field(src.S, "S")
            s.kind = L.CBS_SRC_USER
            s.user_src_dev = _ptr(src.S)
            pol = (0, 0, 0)
        else:
            raise TypeError(type(src))
        for i in range(3):
            p = complex(pol[i])
            s.pol[i][0] = p.real
            s.pol[i][1] = p.imag
        return s

    def forward(self, source, E: Optional[torch.Tensor] = None, warm_start: int = 0):
        """Solve for the field of `source`; returns (E, Stats).  warm_start: 0 starts from
        zero; 1 from E with residuals relative to this run's first; 2 from E with residuals
        relative to a start from zero (stops early for a close guess).  Raises on errors
        other than 'not converged', 'stagnated' and 'time limit' (then Stats.status says
        which)."""
        if E is None:
            if warm_start:
                raise ValueError("warm_start needs E")
            E = _field_like(self.shape, self.device)
        self._check_field(E, "E")
        s = self._source(source, int(warm_start))
        st = L.cbs_stats()
        L.check(self.lib.cbs_forward(self.handle, ctypes.byref(s), ctypes.c_void_p(_ptr(E)),
                                     ctypes.byref(st)), allow=L.NONFATAL)
        return E, _stats(st)

    def adjoint(self, r0, E: torch.Tensor, E_adj: Optional[torch.Tensor] = None):
        """Adjoint field of |E(r0)|^2; returns (E_adj, Stats)."""
        self._check_field(E, "E")
        if E_adj is None:
            E_adj = _field_like(self.shape, self.device)
        self._check_field(E_adj, "E_adj")
        r = (ctypes.c_int * 3)(*[int(v) for v in r0])
        st = L.cbs_stats()
        L.check(self.lib.cbs_adjoint(self.handle, ctypes.byref(r), ctypes.c_void_p(_ptr(E)),
                                     ctypes.c_void_p(_ptr(E_adj)), ctypes.byref(st)),
                allow=L.NONFATAL)
        return E_adj, _stats(st)

    def gradient(self, E: torch.Tensor, E_adj: torch.Tensor, r0=None, grad: Optional[torch.Tensor] = None):
        """dL/d eps_r = 2 k_vac^2 Re[E_adj . E] (float32 (nz, ny, nx)) and, with r0, |E(r0)|^2."""
        self._check_field(E, "E")
        self._check_field(E_adj, "E_adj")
        if grad is None:
            grad = torch.empty(self.shape, dtype=torch.float32, device=self.device)
        obj = ctypes.c_double(float("nan"))
        r = (ctypes.c_int * 3)(*[int(v) for v in r0]) if r0 is not None else None
        L.check(self.lib.cbs_gradient(self.handle, ctypes.c_void_p(_ptr(E)), ctypes.c_void_p(_ptr(E_adj)),
                                      ctypes.byref(r) if r is not None else None,
                                      ctypes.c_void_p(_ptr(grad)), ctypes.byref(obj) if r is not None else None))
        return grad, (obj.value if r0 is not None else None)

    def objective(self, E: torch.Tensor, r0) -> float:
        """|E(r0)|^2 (FP64 on the device)."""
        self._check_field(E, "E")
        r = (ctypes.c_int * 3)(*[int(v) for v in r0])
        obj = ctypes.c_double()
        L.check(self.lib.cbs_objective(self.handle, ctypes.c_void_p(_ptr(E)), ctypes.byref(r), ctypes.byref(obj)))
        return obj.value

    def design_step_host(self, eps_host: np.ndarray, source, r0, grad_host: Optional[np.ndarray] = None):
        """Forward + adjoint + gradient from host memory (the library copies in and out).
        Returns (grad_host, objective, fwd Stats, adj Stats)."""
        eps_host = np.ascontiguousarray(eps_host, dtype=np.float32)
        if eps_host.shape != self.shape:
            raise ValueError("eps_host shape")
        if grad_host is None:
            grad_host = np.empty(self.shape, dtype=np.float32)
        s = self._source(source, False)
        r = (ctypes.c_int * 3)(*[int(v) for v in r0])
        obj = ctypes.c_double()
        f, a = L.cbs_stats(), L.cbs_stats()
        L.check(self.lib.cbs_design_step_host(
            self.handle, ctypes.c_void_p(eps_host.ctypes.data), ctypes.byref(s), ctypes.byref(r),
            ctypes.c_void_p(grad_host.ctypes.data), ctypes.byref(obj), ctypes.byref(f), ctypes.byref(a)))
        return grad_host, obj.value, _stats(f), _stats(a)
