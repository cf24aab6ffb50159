"""ctypes binding of ``libsislice.so`` (the C ABI in include/sislice.h).

Argument marshalling only.  The library is built in-tree by ``build.py``; importing
this module without it raises immediately -- there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libsislice.so")

SS_OK, SS_ERR_ARG, SS_ERR_CUDA, SS_ERR_OOM, SS_ERR_SINGULAR, SS_ERR_NOT_SPD, SS_ERR_NOCONV, \
    SS_ERR_TIMEOUT, SS_ERR_INTERNAL = range(9)
SS_FP64, SS_MIXED, SS_FP64_SOLVE32 = 0, 1, 2
SS_INERTIA_ONLY = 4
SS_MIXED_TC = 3
SS_SOLVE_SWEEP_KERNEL, SS_SOLVE_PER_STEP = 0, 1
SS_SUBSPACE, SS_BLOCK_LANCZOS = 0, 1
SS_PEAK_FP64_FMA, SS_PEAK_FP32_FMA = 0, 1
SS_SCHUR_TENSOR, SS_SCHUR_SIMT = 0, 1
SS_GEMM_TENSOR, SS_GEMM_SIMT = 0, 1
STATUS_NAMES = {0: "SS_OK", 1: "SS_ERR_ARG", 2: "SS_ERR_CUDA", 3: "SS_ERR_OOM", 4: "SS_ERR_SINGULAR",
                5: "SS_ERR_NOT_SPD", 6: "SS_ERR_NOCONV", 7: "SS_ERR_TIMEOUT", 8: "SS_ERR_INTERNAL"}


class ss_options(C.Structure):
    _fields_ = [("nd_leaf", C.c_int32), ("panel", C.c_int32), ("reserved", C.c_int32 * 6)]


class ss_symbolic_info(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("n_supernodes", C.c_int64),
                ("n_levels", C.c_int64), ("n_panels", C.c_int64), ("n_panel_levels", C.c_int64),
                ("max_front", C.c_int64), ("factor_entries", C.c_int64), ("front_entries", C.c_int64),
                ("factor_flops", C.c_double), ("schur_flops", C.c_double), ("panel_flops", C.c_double),
                ("l_offdiag_entries", C.c_int64), ("l_diag_entries", C.c_int64), ("analyze_seconds", C.c_double),
                ("l_storage_entries", C.c_int64), ("workspace_entries", C.c_int64), ("cb_pool_entries", C.c_int64)]


class ss_probe_stats(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("refine_steps", C.c_int32), ("converged", C.c_int32),
                ("reserved", C.c_int32), ("max_resid_in_slice", C.c_double), ("seconds", C.c_double)]


class ss_solve_opts(C.Structure):
    _fields_ = [("driver", C.c_int32), ("max_iter", C.c_int32), ("check_every", C.c_int32),
                ("refine", C.c_int32), ("tol", C.c_double), ("n_expect", C.c_int32),
                ("k_out", C.c_int32), ("refine_from_start", C.c_int32), ("reserved", C.c_int32),
                ("refine_ratio", C.c_double)]


EXPORTS = ["ss_create", "ss_destroy", "ss_last_error", "ss_analyze", "ss_symbolic_info_get",
           "ss_symbolic_perm", "ss_symbolic_destroy", "ss_symbolic_validate", "ss_factor", "ss_factor_segments", "ss_factor_destroy", "ss_inertia", "ss_inertia_segments", "ss_factor_stats", "ss_factor_quality",
           "ss_solve", "ss_solve_noalloc", "ss_slice_solve", "ss_dos_estimate", "ss_dos_lanczos", "ss_band_energy_grad", "ss_spmm", "ss_sync", "ss_launch_count", "ss_profile", "ss_profile_query", "ss_set_solve_mode", "ss_set_sweep_fusion", "ss_selftest_barrier", "ss_measure_peak", "ss_set_schur_mode", "ss_selftest_tc", "ss_set_factor_graph", "ss_autotune_schur", "ss_set_gemm_mode", "ss_dense_gram", "ss_dense_gemm", "ss_profile_query_tensor"]
KERNEL_CLASSES = ["assemble", "extend_add", "diag_bk", "panel", "schur", "fwd_diag", "fwd_update", "bwd_gather",
                  "bwd_diag", "permute", "spmm", "gram", "gemm", "small_dense", "jacobi", "lanczos", "sddmm", "misc",
                  "panel_f32", "schur_f32", "fwd_update_f32", "bwd_gather_f32", "solve", "solve_f32",
                  "schur_tc", "gemm_tc", "spmm_tc"]

_lib = None


def load():
    """Load the library (raises OSError if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise OSError(f"{LIB_PATH} is missing: run paper_1908_06043_gb300/build.py (or __graft_entry__.build())")
    L = C.CDLL(LIB_PATH)
    P, i32, i64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    PP = C.POINTER(C.c_void_p)
    sig = {
        "ss_create": ([PP, i32, P], i32),
        "ss_destroy": ([P], i32),
        "ss_last_error": ([P], C.c_char_p),
        "ss_set_solve_mode": ([P, i32], i32),
        "ss_selftest_barrier": ([P, i32, C.c_int64], i32),
        "ss_measure_peak": ([P, i32, dbl, C.POINTER(dbl)], i32),
        "ss_set_schur_mode": ([P, i32, dbl], i32),
        "ss_selftest_tc": ([P, C.c_uint64, C.POINTER(dbl)], i32),
        "ss_set_factor_graph": ([P, i32], i32),
        "ss_set_gemm_mode": ([P, i32], i32),
        "ss_dense_gram": ([P, P, i64, i64, i32, P, i64, i32, P], i32),
        "ss_profile_query_tensor": ([P, i32, C.POINTER(dbl)], i32),
        "ss_dense_gemm": ([P, P, i64, i64, i32, P, i32, i32, dbl, dbl, P, i64], i32),
        "ss_autotune_schur": ([P, P, P, dbl, C.POINTER(i32)], i32),
        "ss_analyze": ([P, i64, P, P, C.POINTER(ss_options), PP], i32),
        "ss_symbolic_info_get": ([P, C.POINTER(ss_symbolic_info)], i32),
        "ss_symbolic_perm": ([P, P], i32),
        "ss_symbolic_destroy": ([P], i32),
        "ss_symbolic_validate": ([P], i32),
        "ss_factor": ([P, P, P, P, i32, i32, PP], i32),
        "ss_factor_destroy": ([P], i32),
        "ss_inertia": ([P, i32, C.POINTER(i64), C.POINTER(i64), C.POINTER(i64), C.POINTER(i32)], i32),
        "ss_factor_segments": ([P, P, P, P, i32, P, i32, PP], i32),
        "ss_set_sweep_fusion": ([P, i32], i32),
        "ss_inertia_segments": ([P, i32, P, P, P, P], i32),
        "ss_factor_stats": ([P, i32, C.POINTER(dbl), C.POINTER(dbl), C.POINTER(i64)], i32),
        "ss_factor_quality": ([P, i32, C.POINTER(i32), C.POINTER(dbl)], i32),
        "ss_solve": ([P, i32, P, i32, P, i32], i32),
        "ss_solve_noalloc": ([P, i32, P, i32, P], i32),
        "ss_slice_solve": ([P, i32, dbl, dbl, C.POINTER(ss_solve_opts), P, i32, P, P, P, C.POINTER(i32),
                            C.POINTER(ss_probe_stats)], i32),
        "ss_dos_estimate": ([P, P, P, i32, i32, P, P, P, P], i32),
        "ss_dos_lanczos": ([P, P, P, i32, i32, P, P, P, P], i32),
        "ss_band_energy_grad": ([P, P, P, i32, P, P], i32),
        "ss_spmm": ([P, P, P, P, P, P, i32, P], i32),
        "ss_sync": ([P], i32),
        "ss_launch_count": ([], i64),
        "ss_profile": ([P, C.c_uint32], i32),
        "ss_profile_query": ([P, i32, C.POINTER(i64), C.POINTER(dbl), C.POINTER(dbl)], i32),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L
