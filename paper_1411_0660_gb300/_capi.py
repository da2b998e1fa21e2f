"""ctypes declarations of libmblsi (include/mblsi.h).  Argument marshalling only."""
from __future__ import annotations

import ctypes
import os

from . import build as _build

c_int, c_int64, c_double, c_void_p, c_size_t, c_uint64 = (
    ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint64)
P = ctypes.POINTER

MBL_OK = 0
MBL_ERR_INVALID = 1
MBL_ERR_OOM = 2
MBL_ERR_SINGULAR = 3
MBL_ERR_NOT_CONVERGED = 4
MBL_ERR_TIMEOUT = 5
MBL_ERR_CUDA = 6
MBL_PENDING = 7
MBL_PREC_FP64 = 0
MBL_PREC_FP32 = 1
MBL_ORDER_BAND = 0
MBL_ORDER_COVER = 1
MBL_ORDER_MODES = 2
MBL_ORDER_AUTO = 3
MBL_ORDER_HYBRID = 4


class Opts(ctypes.Structure):
    _fields_ = [("precision", c_int), ("block", c_int), ("ncv", c_int), ("max_restarts", c_int),
                ("tol", c_double), ("target_tol", c_double), ("refine_tol", c_double), ("max_refine", c_int),
                ("start_seed", c_uint64), ("tensor_cores", c_int), ("refine_mode", c_int),
                ("gmres_restart", c_int), ("solve_dataflow", c_int), ("deflate", c_int),
                ("wait_limit_s", c_double), ("arena_mode", c_int), ("pivot_tiny", c_double)]


class FactorStats(ctypes.Structure):
    _fields_ = [("n", c_int64), ("nnz_l", c_int64), ("n_supernodes", c_int64), ("max_front", c_int64),
                ("tree_levels", c_int64), ("perturbed", c_int64), ("negative", c_int64), ("flops", c_double),
                ("factor_bytes", c_double), ("front_bytes", c_double), ("ms_factor", c_double),
                ("max_abs_l", c_double), ("min_abs_d", c_double), ("tune_choice", c_int * 8),
                ("tune_us_tc", ctypes.c_float * 8), ("tune_us_cc", ctypes.c_float * 8)]


class PlanStats(ctypes.Structure):
    _fields_ = [("n", c_int64), ("nnz_l", c_int64), ("n_supernodes", c_int64), ("max_front", c_int64),
                ("tree_levels", c_int64), ("panel_steps", c_int64), ("solve_steps", c_int64), ("flops", c_double),
                ("ms_analyse", c_double), ("factor_bytes_fp32", c_double), ("factor_bytes_fp64", c_double),
                ("front_bytes_fp32", c_double), ("front_bytes_fp64", c_double),
                ("solve_factor_bytes_fp32", c_double), ("job_peak_bytes_fp32", c_double),
                ("job_peak_bytes_fp64", c_double), ("front_peak_bytes_fp32", c_double),
                ("front_peak_bytes_fp64", c_double), ("ordering", c_int64)]


class SolveStats(ctypes.Structure):
    _fields_ = [("restarts", c_int), ("op_applies", c_int), ("solves", c_int), ("fp64_fallback", c_int),
                ("krylov_dim", c_int), ("max_resid", c_double), ("ms_total", c_double), ("ms_factor", c_double),
                ("shift_moves", c_int), ("refine_escalations", c_int), ("factor_reused", c_int),
                ("static_pivot", c_double)]


class Request(ctypes.Structure):
    _fields_ = [("L", c_int), ("h", c_double), ("seed", c_uint64), ("fields", c_void_p), ("eps", c_double),
                ("nev", c_int), ("precision", c_int), ("want_vectors", c_int), ("nup", c_int)]


class Result(ctypes.Structure):
    _fields_ = [("status", c_int), ("nconv", c_int), ("nev", c_int), ("L", c_int), ("dim", c_int64),
                ("sigma", c_double), ("r_mean", c_double), ("t_submit_ms", c_double), ("t_admit_ms", c_double),
                ("t_end_ms", c_double), ("d_start_ms", c_double), ("d_end_ms", c_double),
                ("reserved_bytes", c_size_t), ("evals", c_void_p), ("resid", c_void_p),
                ("r", c_void_p), ("s1p", c_void_p), ("se", c_void_p), ("evecs", c_void_p),
                ("factor_reused", c_int)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", c_int64), ("completed", c_int64), ("failed", c_int64), ("running", c_int),
                ("queued", c_int), ("slots", c_int), ("budget_bytes", c_size_t), ("reserved_bytes", c_size_t),
                ("peak_reserved_bytes", c_size_t), ("solve_batches", c_int64), ("batched_solves", c_int64),
                ("batch_ms", c_double), ("batch_bytes", c_double), ("cache_hits", c_int64),
                ("cache_bytes", c_size_t), ("batch_busy_ms", c_double)]


# (name, restype, argtypes); every entry point of include/mblsi.h
SIGNATURES = [
    ("mbl_opts_default", None, [P(Opts)]),
    ("mbl_version", ctypes.c_char_p, []),
    ("mbl_last_error", ctypes.c_char_p, [c_void_p]),
    ("mbl_status_string", ctypes.c_char_p, [c_int]),
    ("mbl_launch_count", ctypes.c_longlong, []),
    ("mbl_ctx_set_profiling", c_int, [c_void_p, c_int]),
    ("mbl_ctx_set_ordering", c_int, [c_void_p, c_int]),
    ("mbl_ctx_profile_get", c_int, [c_void_p, ctypes.c_char_p, P(c_int64), P(c_double), P(c_double)]),
    ("mbl_ctx_create", c_int, [c_int, c_size_t, P(c_void_p)]),
    ("mbl_ctx_destroy", None, [c_void_p]),
    ("mbl_ctx_synchronize", c_int, [c_void_p]),
    ("mbl_build_sector", c_int, [c_void_p, c_int, c_double, c_uint64, P(c_void_p)]),
    ("mbl_build_sector_fields", c_int, [c_void_p, c_int, c_void_p, c_double, P(c_void_p)]),
    ("mbl_build_sector_nup", c_int, [c_void_p, c_int, c_int, c_double, c_uint64, P(c_void_p)]),
    ("mbl_build_sector_fields_nup", c_int, [c_void_p, c_int, c_int, c_void_p, c_double, P(c_void_p)]),
    ("mbl_sector_shape", c_int, [c_void_p, P(c_int), P(c_int)]),
    ("mbl_sector_destroy", None, [c_void_p]),
    ("mbl_sector_info", c_int, [c_void_p, P(c_int64), P(c_int64)]),
    ("mbl_sector_copy_basis", c_int, [c_void_p, c_void_p]),
    ("mbl_sector_copy_csr", c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    ("mbl_sector_copy_fields", c_int, [c_void_p, c_void_p]),
    ("mbl_sector_rank", c_int, [c_void_p, c_void_p, c_int64, c_void_p]),
    ("mbl_spmv", c_int, [c_void_p, c_double, c_void_p, c_void_p, c_int]),
    ("mbl_extremal_bounds", c_int, [c_void_p, P(c_double), P(c_double)]),
    ("mbl_factor", c_int, [c_void_p, c_double, P(Opts), P(c_void_p)]),
    ("mbl_factor_stats_get", c_int, [c_void_p, P(FactorStats)]),
    ("mbl_factor_solve", c_int, [c_void_p, c_void_p, c_void_p, c_int, c_int]),
    ("mbl_factor_solve_dev", c_int, [c_void_p, c_void_p, c_void_p, c_int, c_int, c_void_p]),
    ("mbl_factor_destroy", None, [c_void_p]),
    ("mbl_solve_near", c_int, [c_void_p, c_double, c_int, P(Opts), c_void_p, c_void_p, c_void_p, P(c_int),
                               P(c_double), P(SolveStats)]),
    ("mbl_solve_near_dev", c_int, [c_void_p, c_double, c_int, P(Opts), c_void_p, c_void_p, c_void_p, P(c_int),
                                   P(c_double), P(SolveStats), c_void_p]),
    ("mbl_analyse", c_int, [c_void_p, c_int, c_int, P(PlanStats)]),
    ("mbl_factor_trace", c_int, [c_void_p, c_int]),
    ("mbl_factor_trace_get", c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int, P(c_int)]),
    ("mbl_observables", c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                c_void_p]),
    ("mbl_observables_dev", c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                    c_void_p, c_void_p]),
    ("mbl_observables_extra", c_int, [c_void_p, c_int, c_int, c_void_p, c_double, c_void_p, c_void_p, c_void_p,
                                      c_void_p]),
    ("mbl_observables_extra_dev", c_int, [c_void_p, c_int, c_int, c_void_p, c_double, c_void_p, c_void_p,
                                          c_void_p, c_void_p, c_void_p]),
    ("mbl_observables_nup", c_int, [c_void_p, c_int, c_int, c_int, c_void_p, c_void_p, c_void_p, c_void_p,
                                    c_void_p, c_void_p]),
    ("mbl_observables_nup_dev", c_int, [c_void_p, c_int, c_int, c_int, c_void_p, c_void_p, c_void_p, c_void_p,
                                        c_void_p, c_void_p, c_void_p]),
    ("mbl_observables_extra_nup", c_int, [c_void_p, c_int, c_int, c_int, c_void_p, c_double, c_void_p, c_void_p,
                                          c_void_p, c_void_p]),
    ("mbl_observables_extra_nup_dev", c_int, [c_void_p, c_int, c_int, c_int, c_void_p, c_double, c_void_p,
                                              c_void_p, c_void_p, c_void_p, c_void_p]),
    ("mbl_entanglement_noalloc_dev", c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p, c_void_p]),
    ("mbl_server_start", c_int, [c_void_p, c_int, c_size_t]),
    ("mbl_server_batching", c_int, [c_void_p, c_int, c_double, c_int]),
    ("mbl_server_cache", c_int, [c_void_p, c_double]),
    ("mbl_factor_solve_batch_dev", c_int, [c_void_p, c_int, c_void_p, c_void_p, c_int, c_void_p]),
    ("mbl_submit", c_int, [c_void_p, P(Request), P(c_uint64)]),
    ("mbl_poll", c_int, [c_void_p, c_uint64, P(Result)]),
    ("mbl_wait", c_int, [c_void_p, c_uint64, c_double, P(Result)]),
    ("mbl_server_stats_get", c_int, [c_void_p, P(ServerStats)]),
    ("mbl_server_stop", c_int, [c_void_p]),
]

_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load the CUDA library.  There is no CPU fallback: a missing or unbuildable library raises."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise ImportError(f"libmblsi.so not built ({path}); run paper_1411_0660_gb300.build.build()")
        _build.build()
    L = ctypes.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L
