"""ctypes binding of libkkspgemm (include/kkspgemm.h): argument marshalling only.

Every computation runs in the CUDA library; this module only loads it and
declares the C signatures.  Importing fails loudly when the library has not
been built: there is no fallback implementation.
"""

from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libkkspgemm.so")

SPGEMM_R32 = 0
SPGEMM_R64 = 1

STATUS_NAMES = {
    0: "SPGEMM_OK", 1: "SPGEMM_ERR_INVALID_ARG", 2: "SPGEMM_ERR_NOT_READY", 3: "SPGEMM_ERR_OOM",
    4: "SPGEMM_ERR_INDEX_OVERFLOW", 5: "SPGEMM_ERR_DEVICE_LIMIT", 6: "SPGEMM_ERR_CUDA",
    7: "SPGEMM_ERR_PATTERN_MISMATCH", 8: "SPGEMM_ERR_BAD_INDEX",
}


class CsrT(C.Structure):
    _fields_ = [("nrows", C.c_int64), ("ncols", C.c_int64), ("nnz", C.c_int64),
                ("rowptr_is_64", C.c_int32), ("dtype", C.c_int32),
                ("rowptr", C.c_void_p), ("colidx", C.c_void_p), ("values", C.c_void_p)]


class OptionsT(C.Structure):
    _fields_ = [("compression", C.c_int32), ("compress_threshold", C.c_double),
                ("l1_max_occupancy", C.c_double), ("l1_max_log2_slots", C.c_int32),
                ("dense", C.c_int32), ("method", C.c_int32),
                ("workspace_limit_bytes", C.c_int64), ("pool_limit_bytes", C.c_int64),
                ("device", C.c_int32), ("hash_function", C.c_int32), ("verbose", C.c_int32),
                ("slots_per_key_log2", C.c_int32), ("tune", C.c_int32),
                ("numeric_positions", C.c_int32), ("cta_partition", C.c_int32), ("window_positions", C.c_int32),
                ("stage_b", C.c_int32), ("sym_merge", C.c_int32)]


class StatsT(C.Structure):
    _fields_ = [("m", C.c_int64), ("n", C.c_int64), ("k", C.c_int64), ("nnzA", C.c_int64),
                ("nnzB", C.c_int64), ("f_m", C.c_int64), ("maxrf", C.c_int64),
                ("f_m_compressed", C.c_int64), ("maxrf_compressed", C.c_int64),
                ("CF", C.c_double), ("CMRF", C.c_double), ("compressed", C.c_int32),
                ("nbins_symbolic", C.c_int32), ("nbins_numeric", C.c_int32), ("tuned_bins", C.c_int32),
                ("nnzC", C.c_int64), ("maxrs", C.c_int64), ("ars", C.c_double),
                ("workspace_bytes", C.c_int64), ("bin_rows_numeric", C.c_int64 * 8),
                ("rows_positions", C.c_int64)]


# name -> (restype, argtypes); mirrors include/kkspgemm.h
_P = C.c_void_p
SIGNATURES = {
    "spgemm_options_default": (C.c_int, [C.POINTER(OptionsT)]),
    "spgemm_handle_create": (C.c_int, [C.POINTER(_P), C.POINTER(OptionsT)]),
    "spgemm_handle_destroy": (C.c_int, [_P]),
    "spgemm_symbolic": (C.c_int, [_P, C.POINTER(CsrT), C.POINTER(CsrT), _P, C.POINTER(C.c_int64), _P]),
    "spgemm_numeric": (C.c_int, [_P, C.POINTER(CsrT), C.POINTER(CsrT), _P, _P, _P, _P]),
    "spgemm_numeric_reuse": (C.c_int, [_P, C.POINTER(CsrT), C.POINTER(CsrT), _P, _P, _P, _P]),
    "spgemm_handle_sync": (C.c_int, [_P, _P]),
    "spgemm_get_stats": (C.c_int, [_P, C.POINTER(StatsT)]),
    "spgemm_masked": (C.c_int, [_P, C.POINTER(CsrT), C.POINTER(CsrT), _P, _P, C.c_int64, _P, _P, _P, _P]),
    "spgemm_masked_count": (C.c_int, [_P, C.POINTER(CsrT), C.POINTER(CsrT), _P, _P, C.c_int64, _P, _P]),
    "spgemm_rap_symbolic": (C.c_int, [_P, C.POINTER(CsrT), C.POINTER(CsrT), _P, C.POINTER(C.c_int64), _P]),
    "spgemm_rap_numeric": (C.c_int, [_P, C.POINTER(CsrT), C.POINTER(CsrT), _P, _P, _P, _P]),
    "spgemm_transpose": (C.c_int, [_P, C.POINTER(CsrT), _P, _P, _P, _P, _P]),
    "spgemm_gather": (C.c_int, [_P, C.c_int, _P, _P, _P, C.c_int64, _P]),
    "spgemm_transpose_noalloc": (C.c_int, [C.POINTER(CsrT), _P, _P, _P, _P, _P]),
    "spgemm_batch_symbolic": (C.c_int, [_P, C.c_int32, C.POINTER(CsrT), C.POINTER(CsrT),
                                        C.POINTER(_P), C.POINTER(C.c_int64), _P]),
    "spgemm_batch_numeric": (C.c_int, [_P, C.c_int32, C.POINTER(CsrT), C.POINTER(CsrT),
                                       C.POINTER(_P), C.POINTER(_P), C.POINTER(_P), _P]),
    "spgemm_row_flops": (C.c_int, [_P, C.POINTER(CsrT), C.POINTER(CsrT), _P, _P]),
    "spgemm_partition_rows": (C.c_int, [_P, C.c_int64, C.c_int32, _P]),
    "spgemm_status_string": (C.c_char_p, [C.c_int]),
    "spgemm_version": (C.c_int32, []),
    "spgemm_launch_count": (C.c_int64, []),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libkkspgemm.so; raises ImportError when it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError("libkkspgemm.so is not built (expected at %s); run "
                          "`python -c 'import __graft_entry__ as g; g.build()'` first" % path)
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


class SpGEMMError(RuntimeError):
    def __init__(self, status: int, call: str):
        self.status = status
        super().__init__("%s returned %s" % (call, STATUS_NAMES.get(status, str(status))))


def check(status: int, call: str):
    if status != 0:
        raise SpGEMMError(status, call)
