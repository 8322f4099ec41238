"""ctypes declarations of the C ABI in include/tucker.h (libtucker.so).

Loading fails loudly when the library has not been built: there is no
fallback implementation behind these names.
"""
from __future__ import annotations

import ctypes as C
import os

MAX_ORDER = 8

OK, EINVAL, ENOMEM, ECUDA, ENOTSPD, ERANK, EDRAWLIMIT, EHASHFULL, ECAPACITY, ENOTSUP, EINTERNAL = range(11)
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ECUDA", "ENOTSPD", "ERANK", "EDRAWLIMIT", "EHASHFULL",
                "ECAPACITY", "ENOTSUP", "EINTERNAL"]
F32, F64 = 0, 1
PREC_FP64, PREC_FP32, PREC_TF32, PREC_BF16 = 0, 1, 2, 3
REG_EXACT, REG_AUGMENTED, REG_RIDGE = 0, 1, 2
SOLVER_FP64_CHOLESKY, SOLVER_MIXED, SOLVER_KRON_PCG = 0, 1, 2

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libtucker.so")


class TuckerTensor(C.Structure):
    _fields_ = [("order", C.c_int), ("dims", C.c_int64 * MAX_ORDER), ("dtype", C.c_int),
                ("dense", C.c_void_p), ("nnz", C.c_int64), ("keys", C.c_void_p),
                ("vals", C.c_void_p)]


class TuckerSamples(C.Structure):
    _fields_ = [("capacity", C.c_int64), ("n_unique", C.c_int64), ("n_draws", C.c_int64),
                ("keys", C.c_void_p), ("counts", C.c_void_p), ("prob", C.c_void_p)]


class TuckerStats(C.Structure):
    _fields_ = [("ms_leverage", C.c_double), ("ms_sample", C.c_double), ("ms_dedupe", C.c_double),
                ("ms_gather", C.c_double), ("ms_gram", C.c_double), ("ms_solve", C.c_double),
                ("ms_total", C.c_double), ("n_unique", C.c_int64), ("n_draws", C.c_int64),
                ("n_real", C.c_int64), ("refine_iters", C.c_int), ("refine_rel", C.c_double),
                ("solve_id", C.c_uint64), ("launches", C.c_int64), ("ms_factor", C.c_double),
                ("ms_gram_kernel", C.c_double), ("ms_inner", C.c_double),
                ("inner_iters", C.c_int64), ("gram_prec_used", C.c_int)]


class TuckerMissingBetaInfo(C.Structure):
    _fields_ = [("lambda_max", C.c_double), ("beta_miss", C.c_double), ("c_min", C.c_double),
                ("beta", C.c_double), ("beta_prime", C.c_double), ("s", C.c_double),
                ("nu_est", C.c_double), ("iters", C.c_int), ("certify_tries", C.c_int)]


_P = C.c_void_p
_PP = C.POINTER(C.c_void_p)
_I64P = C.POINTER(C.c_int64)
_IP = C.POINTER(C.c_int)
_DP = C.POINTER(C.c_double)

# name -> (restype, argtypes)
SIGNATURES = {
    "tucker_create": (C.c_int, [C.POINTER(C.c_void_p), _P]),
    "tucker_destroy": (C.c_int, [_P]),
    "tucker_last_error": (C.c_char_p, [_P]),
    "tucker_set_sync": (C.c_int, [_P, C.c_int]),
    "tucker_set_solver": (C.c_int, [_P, C.c_int]),
    "tucker_sync": (C.c_int, [_P]),
    "tucker_leverage_scores": (C.c_int, [_P, C.c_int, _I64P, _IP, C.c_int, _PP, _PP, _PP, _IP]),
    "tucker_sample_rows": (C.c_int, [_P, C.c_int, _I64P, _IP, _PP, C.c_int64, C.c_uint64,
                                     C.c_uint32, C.c_int, C.POINTER(TuckerTensor), C.c_int64,
                                     C.POINTER(TuckerSamples)]),
    "tucker_core_update_sketched": (C.c_int, [_P, C.POINTER(TuckerTensor), _IP, _PP, C.c_double,
                                              C.c_int64, C.c_double, C.c_double, C.c_uint64,
                                              C.c_uint32, C.c_int, C.c_int,
                                              C.POINTER(TuckerSamples), _P,
                                              C.POINTER(TuckerStats)]),
    "tucker_core_update_exact": (C.c_int, [_P, C.POINTER(TuckerTensor), _IP, _PP, C.c_double,
                                           C.c_int, _P]),
    "tucker_als_sweep": (C.c_int, [_P, C.POINTER(TuckerTensor), _IP, _PP, _P, C.c_double, C.c_int,
                                   C.c_int64, C.c_uint64, C.c_uint32, C.c_int, C.c_int, _DP, _DP]),
    "tucker_ridge_loss": (C.c_int, [_P, C.POINTER(TuckerTensor), _IP, _PP, C.c_double, _P, _DP]),
    "tucker_core_solve_adjoint": (C.c_int, [_P, C.POINTER(TuckerTensor), _IP, _PP, C.c_double,
                                            C.c_int, C.c_int, C.POINTER(TuckerSamples),
                                            C.c_uint64, _P, _P, _PP, _P]),
    "tucker_sketched_gram": (C.c_int, [_P, C.POINTER(TuckerTensor), _IP, _PP, C.c_int,
                                       C.POINTER(TuckerSamples), _P, _P]),
    "tucker_ridge_tables": (C.c_int, [_P, C.c_int, _I64P, _IP, C.c_int, _PP, C.c_double, _PP, _P,
                                      _IP, _DP]),
    "tucker_sample_rows_ridge": (C.c_int, [_P, C.c_int, _I64P, _IP, _PP, _P, C.c_int64, C.c_uint64,
                                           C.c_uint32, C.POINTER(TuckerSamples)]),
    "tucker_factor_update_sketched": (C.c_int, [_P, C.POINTER(TuckerTensor), _IP, _PP, _P, C.c_int,
                                                C.c_double, C.c_int64, C.c_uint64, C.c_uint32]),
    "tucker_set_factor_sketch": (C.c_int, [_P, C.c_int64]),
    "tucker_cp_factor_update_sketched": (C.c_int, [_P, C.POINTER(TuckerTensor), C.c_int, _PP,
                                                   C.c_int, C.c_double, C.c_int64, C.c_uint64,
                                                   C.c_uint32]),
    "tucker_cp_als_sweep": (C.c_int, [_P, C.POINTER(TuckerTensor), C.c_int, _PP, C.c_double,
                                      C.c_int64, C.c_uint64, C.c_uint32]),
    "tucker_missing_beta": (C.c_int, [_P, C.POINTER(TuckerTensor), _IP, _PP, C.c_double, C.c_int,
                                      C.c_int, C.c_double, C.c_double,
                                      C.POINTER(TuckerMissingBetaInfo)]),
    "tucker_sample_rows_noalloc": (C.c_int, [_P, C.c_int, _I64P, _IP, _PP, C.c_int64, C.c_uint64,
                                             C.c_uint32, C.c_int, C.POINTER(TuckerSamples),
                                             C.c_char_p, C.c_size_t]),
}

NOALLOC_SCRATCH_BYTES = 16 << 20

_lib = None


def load():
    """Load libtucker.so (built by paper_2107_10654_gb300.build); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "`python -m paper_2107_10654_gb300.build` (needs nvcc)")
    lib = C.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def ptr_array(ptrs):
    arr = (C.c_void_p * MAX_ORDER)()
    for i, p in enumerate(ptrs):
        arr[i] = p
    return arr
