"""ctypes binding of libcbs.so (the C ABI in include/cbs.h), with the same names.

Argument marshalling only: every step of a solve runs in the CUDA library.  Importing this
module loads the library and raises if it is missing; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, Structure, c_double, c_float, c_int, c_void_p

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libcbs.so")

CBS_OK = 0
CBS_ERR_ARG = -1
CBS_ERR_OOM = -2
CBS_ERR_NOT_CONVERGED = -3
CBS_ERR_DIVERGED = -4
CBS_ERR_CUDA = -5
CBS_ERR_STATE = -6
CBS_ERR_STAGNATED = -7
CBS_ERR_TIME_LIMIT = -8
# solves that end with the last iterate in E and raise nothing in the binding
NONFATAL = (CBS_OK, CBS_ERR_NOT_CONVERGED, CBS_ERR_STAGNATED, CBS_ERR_TIME_LIMIT)

CBS_SRC_PLANE_WAVE = 0
CBS_SRC_POINT = 1
CBS_SRC_USER = 2

# Every symbol include/cbs.h declares.
EXPORTS = ("cbs_plan", "cbs_set_permittivity", "cbs_get_splitting", "cbs_set_solver",
           "cbs_forward", "cbs_adjoint", "cbs_gradient", "cbs_objective", "cbs_design_step_host",
           "cbs_set_profiling", "cbs_pass_times", "cbs_set_time_limit", "cbs_splitting_noalloc", "cbs_destroy",
           "cbs_last_error", "cbs_design_create", "cbs_design_destroy", "cbs_design_reset",
           "cbs_design_get_state", "cbs_design_set_state",
           "cbs_design_permittivity", "cbs_design_height_gradient", "cbs_design_adam", "cbs_design_step",
           "cbs_server_create", "cbs_server_destroy", "cbs_server_submit", "cbs_server_take", "cbs_server_info",
           "cbs_server_sharing",
           "cbs_selftest_wait_timeout")

# cbs_pass_times slots: the series' first forward x pass (launched once per series, not
# timed), then the four kernels of every iteration
PASS_NAMES = ("k_xpass_fwd", "k_ypass_fwd", "k_zpass_green", "k_ypass_inv", "k_xpass_inv_fwd")


class cbs_plan_desc(Structure):
    _fields_ = [("nx", c_int), ("ny", c_int), ("nz", c_int),
                ("pitch_m", c_double), ("lambda_m", c_double), ("n_bg", c_double),
                ("pad_lo", c_int * 3), ("pad_hi", c_int * 3),
                ("tol", c_double), ("max_iter", c_int), ("check_every", c_int),
                ("cuda_stream", c_void_p),
                ("layer_round_trip", c_double), ("layer_power", c_double), ("layer_corner_max", c_int)]


class cbs_source(Structure):
    _fields_ = [("kind", c_int), ("pol", (c_double * 2) * 3), ("z_plane", c_int),
                ("r0", c_int * 3), ("user_src_dev", c_void_p), ("warm_start", c_int)]


class cbs_stats(Structure):
    _fields_ = [("iters", c_int), ("rel_resid", c_double), ("resid0", c_double),
                ("seconds", c_double), ("status", c_int)]


class cbs_design_desc(Structure):
    _fields_ = [("z_base", c_int), ("n_lens", c_double), ("aperture_um", c_double), ("h_max_um", c_double),
                ("sigma_um", c_double), ("mirror", c_int), ("alpha", c_double), ("beta1", c_double),
                ("beta2", c_double), ("adam_eps", c_double)]


class cbs_server_desc(Structure):
    _fields_ = [("hbm_budget_bytes", c_double), ("max_active", c_int), ("tol", c_double), ("max_iter", c_int),
                ("check_every", c_int)]


class cbs_request(Structure):
    _fields_ = [("nx", c_int), ("ny", c_int), ("nz", c_int),
                ("pitch_m", c_double), ("lambda_m", c_double), ("n_bg", c_double),
                ("pad_lo", c_int * 3), ("pad_hi", c_int * 3),
                ("layer_round_trip", c_double), ("layer_power", c_double), ("layer_corner_max", c_int),
                ("eps_host", c_void_p), ("eps_dev", c_void_p), ("src", cbs_source), ("adjoint", c_int),
                ("r0", c_int * 3), ("E_host", c_void_p), ("E_dev", c_void_p), ("grad_host", c_void_p),
                ("grad_dev", c_void_p)]


class cbs_result(Structure):
    _fields_ = [("id", ctypes.c_longlong), ("status", c_int), ("objective", c_double),
                ("fwd", cbs_stats), ("adj", cbs_stats), ("t_submit", c_double), ("t_admit", c_double),
                ("t_done", c_double), ("error", ctypes.c_char * 192)]


class CBSError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"CBS error {code}: {msg}")
        self.code = code


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python -m paper_2506_15411_gb300.build`")
    lib = ctypes.CDLL(path)
    P = c_void_p
    sig = {
        "cbs_plan": (c_int, [POINTER(c_void_p), POINTER(cbs_plan_desc)]),
        "cbs_set_permittivity": (c_int, [P, P]),
        "cbs_get_splitting": (c_int, [P, POINTER(c_double), POINTER(c_double)]),
        "cbs_set_solver": (c_int, [P, c_double, c_int, c_int]),
        "cbs_set_time_limit": (c_int, [P, c_double]),
        "cbs_forward": (c_int, [P, POINTER(cbs_source), P, POINTER(cbs_stats)]),
        "cbs_adjoint": (c_int, [P, POINTER(c_int * 3), P, P, POINTER(cbs_stats)]),
        "cbs_gradient": (c_int, [P, P, P, POINTER(c_int * 3), P, POINTER(c_double)]),
        "cbs_objective": (c_int, [P, P, POINTER(c_int * 3), POINTER(c_double)]),
        "cbs_design_step_host": (c_int, [P, P, POINTER(cbs_source), POINTER(c_int * 3), P,
                                         POINTER(c_double), POINTER(cbs_stats), POINTER(cbs_stats)]),
        "cbs_set_profiling": (c_int, [P, c_int]),
        "cbs_pass_times": (c_int, [P, POINTER(c_double * 5), POINTER(ctypes.c_longlong * 5), c_int]),
        "cbs_splitting_noalloc": (c_int, [POINTER(cbs_plan_desc), P, POINTER(c_double), POINTER(c_double)]),
        "cbs_destroy": (None, [P]),
        "cbs_selftest_wait_timeout": (c_int, [POINTER(c_int)]),
        "cbs_server_create": (c_int, [POINTER(c_void_p), POINTER(cbs_server_desc)]),
        "cbs_server_destroy": (None, [P]),
        "cbs_server_submit": (c_int, [P, POINTER(cbs_request), POINTER(ctypes.c_longlong)]),
        "cbs_server_take": (c_int, [P, POINTER(cbs_result), c_int, c_double, POINTER(c_int)]),
        "cbs_server_info": (c_int, [P, POINTER(ctypes.c_longlong), POINTER(ctypes.c_longlong), POINTER(c_double)]),
        "cbs_server_sharing": (c_int, [P, POINTER(ctypes.c_longlong), POINTER(ctypes.c_longlong), POINTER(c_int)]),
        "cbs_design_create": (c_int, [POINTER(c_void_p), P, POINTER(cbs_design_desc)]),
        "cbs_design_destroy": (None, [P]),
        "cbs_design_reset": (c_int, [P]),
        "cbs_design_get_state": (c_int, [P, P, P, POINTER(c_int)]),
        "cbs_design_set_state": (c_int, [P, P, P, c_int]),
        "cbs_design_permittivity": (c_int, [P, P, P, P]),
        "cbs_design_height_gradient": (c_int, [P, P, P, P]),
        "cbs_design_adam": (c_int, [P, P, P]),
        "cbs_design_step": (c_int, [P, P, POINTER(cbs_source), POINTER(c_int * 3), P, P, P, POINTER(c_double),
                                    POINTER(cbs_stats), POINTER(cbs_stats)]),
        "cbs_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        _lib = load()
    return _lib


def check(rc: int, allow=(CBS_OK,)) -> int:
    if rc not in allow:
        raise CBSError(rc, lib().cbs_last_error().decode())
    return rc
