"""The C ABI without a GPU: the library builds for sm_103a, loads, exports every function
include/cbs.h declares, and the ctypes structures match the C layout (checked with gcc)."""
from __future__ import annotations

import ctypes
import os
import re
import subprocess

from paper_2506_15411_gb300 import _lib as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cbs.h")


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\*)\s+(cbs_\w+)\s*\(", text, re.M)))


def test_header_and_binding_agree():
    assert declared_functions() == sorted(L.EXPORTS)


def test_library_exports_every_declared_symbol(built_lib):
    out = subprocess.run(["nm", "-D", "--defined-only", built_lib], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(cbs_\w+)", out))
    missing = set(declared_functions()) - exported
    assert not missing, missing
    lib = L.load(built_lib)
    for name in declared_functions():
        assert hasattr(lib, name)
    assert lib.cbs_last_error() == b""


def test_struct_layout_matches_c(tmp_path, built_lib):
    src = tmp_path / "layout.c"
    src.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "cbs.h"
#define F(T, m) printf(#T " " #m " %zu\n", offsetof(T, m))
int main(void) {
  printf("cbs_plan_desc size %zu\n", sizeof(cbs_plan_desc));
  printf("cbs_source size %zu\n", sizeof(cbs_source));
  printf("cbs_stats size %zu\n", sizeof(cbs_stats));
  printf("cbs_design_desc size %zu\n", sizeof(cbs_design_desc));
  printf("cbs_server_desc size %zu\n", sizeof(cbs_server_desc));
  printf("cbs_request size %zu\n", sizeof(cbs_request));
  printf("cbs_result size %zu\n", sizeof(cbs_result));
  F(cbs_plan_desc, pitch_m); F(cbs_plan_desc, pad_lo); F(cbs_plan_desc, pad_hi); F(cbs_plan_desc, tol);
  F(cbs_plan_desc, max_iter); F(cbs_plan_desc, check_every); F(cbs_plan_desc, cuda_stream);
  F(cbs_plan_desc, layer_round_trip); F(cbs_plan_desc, layer_power); F(cbs_plan_desc, layer_corner_max);
  F(cbs_source, pol); F(cbs_source, z_plane); F(cbs_source, r0); F(cbs_source, user_src_dev);
  F(cbs_source, warm_start);
  F(cbs_stats, rel_resid); F(cbs_stats, resid0); F(cbs_stats, seconds); F(cbs_stats, status);
  F(cbs_design_desc, n_lens); F(cbs_design_desc, aperture_um); F(cbs_design_desc, h_max_um);
  F(cbs_design_desc, sigma_um); F(cbs_design_desc, mirror); F(cbs_design_desc, alpha);
  F(cbs_design_desc, beta1); F(cbs_design_desc, beta2); F(cbs_design_desc, adam_eps);
  F(cbs_server_desc, max_active); F(cbs_server_desc, tol); F(cbs_server_desc, max_iter);
  F(cbs_server_desc, check_every);
  F(cbs_request, pitch_m); F(cbs_request, pad_lo); F(cbs_request, layer_round_trip);
  F(cbs_request, layer_power); F(cbs_request, layer_corner_max); F(cbs_request, eps_host); F(cbs_request, eps_dev);
  F(cbs_request, src); F(cbs_request, adjoint); F(cbs_request, r0); F(cbs_request, E_host);
  F(cbs_request, E_dev); F(cbs_request, grad_host); F(cbs_request, grad_dev);
  F(cbs_result, status); F(cbs_result, objective); F(cbs_result, fwd); F(cbs_result, adj);
  F(cbs_result, t_submit); F(cbs_result, t_admit); F(cbs_result, t_done); F(cbs_result, error);
  return 0;
}
''')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    lines = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {}
    for ln in lines:
        if ln:
            t, m, v = ln.split()
            got[(t, m)] = int(v)
    types = {"cbs_plan_desc": L.cbs_plan_desc, "cbs_source": L.cbs_source, "cbs_stats": L.cbs_stats,
             "cbs_design_desc": L.cbs_design_desc, "cbs_server_desc": L.cbs_server_desc,
             "cbs_request": L.cbs_request, "cbs_result": L.cbs_result}
    for (t, m), v in got.items():
        if m == "size":
            assert ctypes.sizeof(types[t]) == v, (t, v)
        else:
            assert getattr(types[t], m).offset == v, (t, m, v)


def test_return_codes_match_header():
    text = open(HEADER).read()
    for name in ("CBS_OK", "CBS_ERR_ARG", "CBS_ERR_OOM", "CBS_ERR_NOT_CONVERGED", "CBS_ERR_DIVERGED",
                 "CBS_ERR_CUDA", "CBS_ERR_STATE", "CBS_ERR_STAGNATED", "CBS_ERR_TIME_LIMIT", "CBS_SRC_PLANE_WAVE", "CBS_SRC_POINT", "CBS_SRC_USER"):
        m = re.search(r"#define\s+%s\s+\(?(-?\d+)\)?" % name, text)
        assert m and int(m.group(1)) == getattr(L, name), name


def test_design_state_calls_reject_null_arguments(built_lib):
    """The checkpoint entry points check their arguments before touching the device."""
    lib = L.load(built_lib)
    t = ctypes.c_int(7)
    assert lib.cbs_design_get_state(None, None, None, ctypes.byref(t)) == L.CBS_ERR_ARG
    assert b"NULL" in lib.cbs_last_error() and t.value == 7
    assert lib.cbs_design_set_state(None, None, None, 0) == L.CBS_ERR_ARG


def test_time_limit_rejects_a_null_plan(built_lib):
    lib = L.load(built_lib)
    assert lib.cbs_set_time_limit(None, 1.0) == L.CBS_ERR_ARG
    assert b"NULL" in lib.cbs_last_error()


def test_plan_rejects_bad_descriptions_before_touching_the_device(built_lib):
    """Sizes outside [1, 1024], lengths with a prime factor above 13, layers that do not fit,
    non-positive physics and solver settings: CBS_ERR_ARG, *out = NULL, no CUDA call."""
    lib = L.load(built_lib)
    lam = 1.064e-6

    def plan(nx=16, ny=16, nz=16, pitch=lam / 8, lo=(2, 2, 2), hi=(2, 2, 2), n_bg=1.0, max_iter=10, check_every=8,
             rt=0.0, power=0.0, corner=0):
        d = L.cbs_plan_desc(nx, ny, nz, pitch, lam, n_bg, (ctypes.c_int * 3)(*lo), (ctypes.c_int * 3)(*hi),
                            1e-4, max_iter, check_every, None, rt, power, corner)
        h = ctypes.c_void_p(1)
        rc = lib.cbs_plan(ctypes.byref(h), ctypes.byref(d))
        return rc, h.value, lib.cbs_last_error().decode()

    for kw, words in [(dict(nx=0), "outside"), (dict(ny=1025), "outside"), (dict(nz=-3), "outside"),
                      (dict(nx=17), "product"), (dict(nz=34), "product"), (dict(lo=(9, 2, 2)), "pads"),
                      (dict(hi=(2, 2, -1)), "pads"), (dict(lo=(8, 2, 2), hi=(8, 2, 2)), "pads"),
                      (dict(pitch=0.0), "positive"), (dict(n_bg=-1.0), "positive"),
                      (dict(max_iter=0), ">= 1"), (dict(check_every=0), ">= 1"),
                      (dict(rt=1.5), "layer"), (dict(rt=-0.1), "layer"), (dict(power=-1.0), "layer"),
                      (dict(corner=2), "layer")]:
        rc, h, msg = plan(**kw)
        assert rc == L.CBS_ERR_ARG and h is None and words in msg, (kw, rc, msg)
    assert lib.cbs_plan(None, None) == L.CBS_ERR_ARG
