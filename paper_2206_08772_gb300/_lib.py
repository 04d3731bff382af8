"""ctypes binding of libotm.so (include/otm.h). Argument marshalling only.

The library must exist (built in-tree by ``build.build()``); there is no fallback: every step of
the OTM update runs in the CUDA kernels behind these entry points.
"""
from __future__ import annotations

import ctypes as C
import os
import re
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libotm.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "otm.h")

OK = 0
ERR_ARG, ERR_CUDA, ERR_WORKSPACE, ERR_LME_NOCONV = -1, -2, -3, -4
ERR_JACOBIAN, ERR_NONFINITE, ERR_RETURNMAP_NOCONV, ERR_CAPACITY = -5, -6, -7, -8
ERR_NAMES = {0: "OK", -1: "ARG", -2: "CUDA", -3: "WORKSPACE", -4: "LME_NOCONV", -5: "JACOBIAN",
             -6: "NONFINITE", -7: "RETURNMAP_NOCONV", -8: "CAPACITY"}

PRECISION_FP64, PRECISION_MIXED = 0, 1

PHASES = ["node_update", "kinematics", "return_map", "grid", "search", "node_major", "lme", "compact"]

FIELD = dict(node_x=0, node_du=1, node_mass=2, node_force=3, mp_x=4, F=5, be=6, sigma=7, vol=8,
             ebar=9, T=10, lam=11, support_count=12, support_ids=13, shape=14, newton_it=15,
             rate=16, dF=17, mp_gid=18, node_gid=19, node_flags=20, kinv=21)


class OTMError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        super().__init__(f"{what}: OTM_ERR_{ERR_NAMES.get(code, code)} ({code})")


class Material(C.Structure):
    _fields_ = [("model", C.c_int32), ("fracture", C.c_int32),
                ("E", C.c_double), ("nu", C.c_double), ("rho0", C.c_double),
                ("sigma_y0", C.c_double), ("H", C.c_double),
                ("A", C.c_double), ("B", C.c_double), ("n", C.c_double), ("C", C.c_double),
                ("m", C.c_double), ("eps_dot0", C.c_double),
                ("T_room", C.c_double), ("T_melt", C.c_double), ("chi", C.c_double), ("cp", C.c_double),
                ("d1", C.c_double), ("d2", C.c_double), ("d3", C.c_double), ("d4", C.c_double),
                ("d5", C.c_double)]


class Params(C.Structure):
    _fields_ = [("h", C.c_double), ("beta", C.c_double), ("rs2", C.c_double),
                ("cell_size", C.c_double), ("dt", C.c_double), ("T0", C.c_double),
                ("newton_tol", C.c_double), ("eps_stab", C.c_double),
                ("max_newton", C.c_int32), ("n_materials", C.c_int32), ("precision", C.c_int32),
                ("wall", C.c_int32), ("tool", C.c_int32), ("allow_erode", C.c_int32),
                ("wall_p", C.c_double * 3), ("wall_n", C.c_double * 3),
                ("tool_x0", C.c_double), ("tool_tip_y", C.c_double), ("tool_rake", C.c_double),
                ("tool_clear", C.c_double), ("tool_v", C.c_double), ("friction", C.c_double),
                ("max_support", C.c_int32), ("max_insert", C.c_int32),
                ("mat", Material * 4)]


class Problem(C.Structure):
    _fields_ = [("n_nodes", C.c_int64), ("n_mps", C.c_int64),
                ("node_x", C.c_void_p), ("node_du0", C.c_void_p), ("node_flags", C.c_void_p),
                ("mp_x", C.c_void_p), ("mp_vol", C.c_void_p), ("mp_mass", C.c_void_p),
                ("mp_material", C.c_void_p)]


_lock = threading.Lock()
_lib = None

_P, _I64, _I32, _D, _SZ = C.c_void_p, C.c_int64, C.c_int32, C.c_double, C.c_size_t
_SIGS = {
    "otm_workspace_bytes": (C.c_int, [_I64, _I64, _P, _P]),
    "otm_init": (C.c_int, [_P, _P, _P, _P, _SZ, _P]),
    "otm_step": (C.c_int, [_P, _I32]),
    "otm_step_async": (C.c_int, [_P, _I32]),
    "otm_counts": (C.c_int, [_P, _P, _P, _P, _P]),
    "otm_state": (C.c_int, [_P, _I32, _P, _SZ]),
    "otm_set_state": (C.c_int, [_P, _I32, _P, _SZ]),
    "otm_state_rows": (C.c_int, [_P, _I32, _P, _I64, _P, _SZ]),
    "otm_refresh": (C.c_int, [_P]),
    "otm_error_detail": (C.c_int, [_P, _P, _P]),
    "otm_kernel_launches": (C.c_int, [_P, _P]),
    "otm_destroy": (None, [_P]),
    "otm_phase_timing": (C.c_int, [_P, _I32]),
    "otm_phase_times": (C.c_int, [_P, _P, _P]),
    "otm_search_scratch_bytes": (C.c_int, [_I64, _P]),
    "otm_support_search": (C.c_int, [_P, _I64, _P, _I64, _D, _D, _I32, _P, _P, _P, _SZ, _P, _P, _P]),
    "otm_lme": (C.c_int, [_P, _P, _I64, _P, _P, _I32, _D, _D, _I32, _P, _P, _P, _P, _P]),
    "otm_return_map": (C.c_int, [_P, _D, _I64, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "otm_exp_selftest": (C.c_int, [_P, _I64, _P, _P, _P]),
    "otm_snapshot_bytes": (C.c_int, [_P, _P]),
    "otm_snapshot_save": (C.c_int, [_P, _P]),
    "otm_snapshot_load": (C.c_int, [_P, _P]),
    "otm_adjoint_bytes": (C.c_int, [_P, _P]),
    "otm_adjoint_begin": (C.c_int, [_P, _P, _SZ, _P]),
    "otm_adjoint_step": (C.c_int, [_P, _P, _P]),
    "otm_freeze_topology": (C.c_int, [_P, C.c_int32]),
    "otm_step_with_supports": (C.c_int, [_P, _P, _P]),
    "otm_adjoint_result": (C.c_int, [_P, _P, _P, _P, _P]),
    "otm_supports_export": (C.c_int, [_P, _P, _P, _I64, _P]),
    "otm_keep_last_good": (C.c_int, [_P, _P, _SZ]),
    "otm_step_with_supports_csr": (C.c_int, [_P, _P, _P, _I64]),
    "otm_grid_cells": (C.c_int, [_P, _P, _P, _P, _P, _I64, _P]),
}


def header_functions() -> list[str]:
    """Names of the entry points declared in include/otm.h."""
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|void)\s+(otm_\w+)\s*\(", txt, re.M)))


def load(path: str = LIB_PATH):
    """Load the CUDA library; raises if it has not been built (no fallback path exists)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise ImportError(f"libotm.so not built ({path}); run __graft_entry__.build()")
            L = C.CDLL(path)
            for name, (res, args) in _SIGS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def check(code: int, what: str = ""):
    if code != OK:
        raise OTMError(code, what)
