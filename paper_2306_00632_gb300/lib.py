"""Thin ctypes binding of the C ABI in include/tpcg.h (argument marshalling only).

Every compute step runs in the CUDA library; this module only builds the C structs, passes device
pointers of torch tensors and raises on non-zero status codes.  If the shared library cannot be loaded
the import fails loudly: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

F64, F32, MIXED = 0, 1, 2
GEOM_CUBE, GEOM_TWIST = 0, 1
MAX_BLOCKS = 128
DESC_BYTES = 8192
STATUS = {0: "OK", 1: "E_INVALID", 2: "E_NOMEM", 3: "E_NOT_CONVERGED", 4: "E_RANK_CAP", 5: "E_TIMEOUT",
          6: "E_CUDA", 7: "E_BREAKDOWN"}
STATUS_CODES = {name: code for code, name in STATUS.items()}

# the exported symbols declared in include/tpcg.h
SYMBOLS = [
    "tpcg_setup", "tpcg_problem_create", "tpcg_problem_get_info", "tpcg_problem_export", "tpcg_problem_export_w",
    "tpcg_problem_destroy",
    "tpcg_ctx_create", "tpcg_ctx_bytes", "tpcg_ctx_destroy", "tucker_set_plain", "tucker_get_ranks",
    "tucker_apply", "tucker_residual", "tucker_axpby", "tucker_dot", "tucker_dot_static", "tucker_round", "fd_precond_apply",
    "tpcg_params_default", "tpcg_solve", "tpcg_ctx_history", "tpcg_solve_batch", "tpcg_ctx_stream", "tpcg_last_error", "tpcg_version",
    "tpcg_profile_enable", "tpcg_profile_reset", "tpcg_profile_get", "tpcg_launch_count", "tpcg_set_option",
    "tpcg_expsum_best", "tpcg_setup_host",
    "tpcg_elast_setup", "tpcg_elast_create", "tpcg_elast_get_info", "tpcg_elast_apply", "tpcg_elast_residual",
    "tpcg_elast_precond", "tpcg_elast_solve", "tpcg_elast_destroy",
]
PROF_KINDS = {"zgemm": 0, "zblk": 1, "gram": 2, "eig": 3, "proj": 4, "qr": 5, "apply": 6, "fd": 7, "dot": 8,
              "round": 9}
OPT_GEMM_CTAS_PER_SM, OPT_EXPSUM_BEST, OPT_EIG, OPT_DST, OPT_TC, OPT_RR, OPT_GRAM_MIN_K, OPT_GEMM_KIND = 1, 2, 3, 4, 5, 6, 7, 8   # tpcg_set_option keys
OPT_ROUND_RULE, OPT_RESOLVED = 9, 10
HIST_COLS = 8   # TPCG_HIST_COLS: columns of a tpcg_ctx_history row
PROF_SWEEPS = 11   # one-CTA Jacobi: (sweeps, Grams) in the (flops, bytes) fields of this kind


class TuckerT(C.Structure):
    _fields_ = [("dtype", C.c_int), ("n", C.c_int), ("cap", C.c_int), ("core_cap", C.c_longlong),
                ("U", C.c_void_p * 3), ("core", C.c_void_p), ("desc", C.c_void_p)]


class Geometry(C.Structure):
    _fields_ = [("kind", C.c_int), ("amp", C.c_double), ("eps_geo", C.c_double), ("eps_prec", C.c_double),
                ("k0", C.c_int), ("k1", C.c_int)]


class ProblemArrays(C.Structure):
    _fields_ = [("n", C.c_int), ("p", C.c_int), ("R", C.c_int), ("dtype", C.c_int),
                ("w", C.POINTER(C.c_double)), ("bands", C.POINTER(C.c_double)),
                ("rf", C.c_int * 3), ("f_core", C.POINTER(C.c_double)), ("f_U", C.POINTER(C.c_double) * 3),
                ("n1", C.c_int), ("n2", C.c_int), ("RP", C.c_int), ("w_nnz", C.c_int),
                ("lam", C.POINTER(C.c_double)), ("mu", C.POINTER(C.c_double)),
                ("w_rowptr", C.POINTER(C.c_int)), ("w_col", C.POINTER(C.c_int)), ("w_val", C.POINTER(C.c_double)),
                ("v2u2", C.POINTER(C.c_double)), ("omega", C.POINTER(C.c_double)),
                ("alpha", C.POINTER(C.c_double)), ("lambda_min", C.c_double), ("k0", C.c_int), ("k1", C.c_int)]


class ProblemInfo(C.Structure):
    _fields_ = [("n", C.c_int), ("p", C.c_int), ("R", C.c_int), ("RP", C.c_int), ("n1", C.c_int),
                ("n2", C.c_int), ("rf", C.c_int * 3), ("dtype", C.c_int), ("lambda_min", C.c_double),
                ("lambda_max", C.c_double), ("MP", C.c_double), ("norm_f", C.c_double), ("w_nnz", C.c_int),
                ("k0", C.c_int), ("k1", C.c_int)]


class Params(C.Structure):
    _fields_ = [("tol", C.c_double), ("eps0", C.c_double), ("eps_min", C.c_double), ("alpha", C.c_double),
                ("delta", C.c_double), ("beta_trunc", C.c_double), ("max_it", C.c_int), ("rank_cap", C.c_int),
                ("inner_tol", C.c_double), ("max_outer", C.c_int), ("refine_keep", C.c_double)]


class Stats(C.Structure):
    _fields_ = [("iters", C.c_int), ("status", C.c_int), ("rel_res", C.c_double), ("rank", C.c_int * 3),
                ("mem_compression", C.c_double), ("dt_trials", C.c_int), ("max_rank_seen", C.c_int),
                ("outer_iters", C.c_int), ("true_rel_res", C.c_double)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load the shared library (building it first when asked); raises if it is unavailable."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing:
        path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"TPCG CUDA library not found at {path}; run paper_2306_00632_gb300.build.build()")
    lib = C.CDLL(path)
    vp, i, d, pd = C.c_void_p, C.c_int, C.c_double, C.POINTER(C.c_double)
    PT = C.POINTER(TuckerT)
    sig = {
        "tpcg_setup": (i, [C.POINTER(Geometry), i, i, i, C.POINTER(vp)]),
        "tpcg_problem_create": (i, [C.POINTER(ProblemArrays), C.POINTER(vp)]),
        "tpcg_problem_get_info": (i, [vp, C.POINTER(ProblemInfo)]),
        "tpcg_problem_export": (i, [vp] + [vp] * 11),
        "tpcg_problem_export_w": (i, [vp, vp, vp, vp]),
        "tpcg_problem_destroy": (None, [vp]),
        "tpcg_ctx_create": (i, [i, i, i, i, C.POINTER(vp)]),
        "tpcg_ctx_bytes": (C.c_size_t, [i, i, i, i]),
        "tpcg_ctx_destroy": (None, [vp]),
        "tucker_set_plain": (i, [PT, i, i, i, vp]),
        "tucker_get_ranks": (i, [PT, C.POINTER(C.c_int), C.POINTER(C.c_int), vp]),
        "tucker_apply": (i, [vp, PT, PT, vp]),
        "tucker_residual": (i, [vp, PT, PT, vp]),
        "tucker_axpby": (i, [d, vp, PT, d, vp, PT, PT, vp]),
        "tucker_dot": (i, [vp, PT, PT, vp, vp]),
        "tucker_dot_static": (i, [PT, PT, vp, vp]),
        "tucker_round": (i, [vp, PT, d, vp, i, vp, vp]),
        "fd_precond_apply": (i, [vp, vp, PT, PT, vp]),
        "tpcg_params_default": (None, [C.POINTER(Params)]),
        "tpcg_solve": (i, [vp, vp, C.POINTER(Params), PT, C.POINTER(Stats), vp]),
        "tpcg_ctx_history": (i, [vp, C.POINTER(d), i, C.POINTER(C.c_int)]),
        "tpcg_ctx_stream": (i, [vp, C.POINTER(vp)]),
        "tpcg_solve_batch": (i, [i, vp, vp, C.POINTER(Params), PT, C.POINTER(Stats), vp, C.POINTER(C.c_int)]),
        "tpcg_last_error": (C.c_char_p, []),
        "tpcg_profile_enable": (i, [i]),
        "tpcg_profile_reset": (i, []),
        "tpcg_profile_get": (i, [i, C.POINTER(d), C.POINTER(C.c_longlong), C.POINTER(d), C.POINTER(d)]),
        "tpcg_launch_count": (C.c_longlong, []),
        "tpcg_set_option": (i, [i, C.c_longlong]),
        "tpcg_expsum_best": (i, [d, d, i, C.POINTER(d), C.POINTER(d), C.POINTER(C.c_int), C.POINTER(d)]),
        "tpcg_setup_host": (i, [C.POINTER(Geometry), i, i, C.POINTER(ProblemInfo)] + [C.POINTER(d)] * 11
                            + [C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(d)]),
        "tpcg_version": (C.c_char_p, []),
        "tpcg_elast_setup": (i, [C.POINTER(Geometry), i, i, d, d, C.POINTER(d), i, C.POINTER(vp)]),
        "tpcg_elast_create": (i, [C.POINTER(ProblemArrays), d, d, C.POINTER(vp)]),
        "tpcg_elast_get_info": (i, [vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(d)]),
        "tpcg_elast_apply": (i, [vp, PT, PT, vp]),
        "tpcg_elast_residual": (i, [vp, PT, PT, vp]),
        "tpcg_elast_precond": (i, [vp, vp, PT, PT, vp]),
        "tpcg_elast_solve": (i, [vp, vp, C.POINTER(Params), PT, C.POINTER(Stats), vp]),
        "tpcg_elast_destroy": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class TpcgError(RuntimeError):
    def __init__(self, code, where):
        msg = load().tpcg_last_error().decode()
        super().__init__(f"{where}: {STATUS.get(code, code)}: {msg}")
        self.code = code


def check(code: int, where: str):
    if code != 0:
        raise TpcgError(code, where)
    return code
