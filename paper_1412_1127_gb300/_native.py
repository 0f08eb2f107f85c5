"""Loader of the in-tree C-ABI library ``libaccr.so`` (see ``include/accr.h``).

There is no fallback: if the library is missing or does not load, every call
raises, so no result can silently come from anywhere but the CUDA kernels.
"""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
# The library: the in-tree release build, or another build of it named by
# ACCR_LIBRARY (the debug build, libaccr_debug.so, for bounds-checked runs).
LIB_PATH = os.environ.get("ACCR_LIBRARY") or os.path.join(_HERE, "libaccr.so")

# status codes of include/accr.h
ACCR_OK = 0
ACCR_EINVAL = -1
ACCR_ETYPE = -2
ACCR_ENOMEM = -3
ACCR_ECUDA = -4
ACCR_EAGAIN = -5
ACCR_EBUDGET = -6
ACCR_ETIMEDOUT = -7

ERROR_NAMES = {ACCR_EINVAL: "EINVAL", ACCR_ETYPE: "ETYPE", ACCR_ENOMEM: "ENOMEM",
               ACCR_ECUDA: "ECUDA", ACCR_EAGAIN: "EAGAIN", ACCR_EBUDGET: "EBUDGET",
               ACCR_ETIMEDOUT: "ETIMEDOUT"}


class AccrError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (ERROR_NAMES.get(code, "?"), code, msg))
        self.code = code


class Clause(ctypes.Structure):
    """``accr_clause``: one reduction(op:var) clause."""
    _fields_ = [("op", ctypes.c_int32), ("acc_type", ctypes.c_int32),
                ("init", ctypes.c_void_p), ("out", ctypes.c_void_p)]


class Region(ctypes.Structure):
    """``accr_region``: one region of a batch."""
    _fields_ = [("in_", ctypes.c_void_p), ("n", ctypes.c_int64), ("in_type", ctypes.c_int32),
                ("nclauses", ctypes.c_int32), ("flags", ctypes.c_uint32), ("reserved", ctypes.c_int32),
                ("clauses", Clause * 4)]


class Result(ctypes.Structure):
    """``accr_result``: one served region's variables and times."""
    _fields_ = [("status", ctypes.c_int32), ("nclauses", ctypes.c_int32),
                ("value", ctypes.c_uint64 * 4), ("submit_ns", ctypes.c_int64),
                ("launch_ns", ctypes.c_int64), ("done_ns", ctypes.c_int64)]


# Every symbol include/accr.h declares, with its ctypes signature.
_vp, _i32, _i64, _u32, _u64 = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64,
                               ctypes.c_uint32, ctypes.c_uint64)
_CP = ctypes.POINTER(Clause)
SIGNATURES = {
    "accr_reduce": (ctypes.c_int, [_vp, _i64, _i32, _CP, _i32, _u32, _vp]),
    "accr_rowreduce": (ctypes.c_int, [_vp, _i64, _i64, _i64, _i32, _CP, _i32, _u32, _vp]),
    "accr_batch_reduce": (ctypes.c_int, [ctypes.POINTER(Region), _i64, _u32, _vp]),
    "accr_segmented_reduce": (ctypes.c_int, [_vp, ctypes.POINTER(_i64), _i64, _i32, _CP, _i32, _u32, _vp]),
    "accr_batch_create": (ctypes.c_int, [ctypes.POINTER(Region), _i64, _u32, ctypes.POINTER(_vp)]),
    "accr_batch_launch": (ctypes.c_int, [_vp, _vp]),
    "accr_batch_destroy": (ctypes.c_int, [_vp]),
    "accr_batch_tiling": (ctypes.c_int, [_i64, _i64, ctypes.POINTER(_i64), ctypes.POINTER(_i64)]),
    "accr_server_create": (ctypes.c_int, [_u64, _i32, _i32, ctypes.POINTER(_vp)]),
    "accr_submit": (ctypes.c_int, [_vp, ctypes.POINTER(Region), ctypes.POINTER(_u64)]),
    "accr_poll": (ctypes.c_int, [_vp, _u64, ctypes.POINTER(Result), _i64]),
    "accr_server_destroy": (ctypes.c_int, [_vp]),
    "accr_server_replay": (ctypes.c_int, [_vp, ctypes.POINTER(Region), ctypes.POINTER(ctypes.c_double), _i64,
                                          _u32, _vp, ctypes.POINTER(Result)]),
    "accr_matmul_nest": (ctypes.c_int, [_vp, _vp, _vp, _i64, _i32, _u32, _vp]),
    "accr_nearest_k": (ctypes.c_int, [_vp, _i64, ctypes.c_float, ctypes.c_float, _i32, _vp, _vp, _u32, _vp]),
    "accr_standardize": (ctypes.c_int, [_vp, _i64, _vp, _vp, _u32, _vp]),
    "accr_grid_bfs": (ctypes.c_int, [_vp, _i64, _i64, _i64, _vp, _i32, ctypes.POINTER(_i64), _vp]),
    "accr_reduce_noalloc": (ctypes.c_int, [_vp, _i64, _i32, _CP, _i32, _u32, _vp]),
    "accr_fault_inject": (ctypes.c_int, [_i32, _i64]),
    "accr_selftest_wait_timeout": (ctypes.c_int, [_u32, _vp]),
    "accr_probe_fma": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int64, _vp, _vp]),
    "accr_probe_fma_packed": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int64, _vp, _vp]),
    "accr_debug_report": (ctypes.c_int, [ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint32),
                                         ctypes.POINTER(ctypes.c_int32), ctypes.c_int32]),
    "accr_last_error": (ctypes.c_char_p, []),
    "accr_launch_count": (_u64, []),
    "accr_version": (_i32, []),
}

_lib = None


def lib():
    """The loaded library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libaccr.so is not built (run `python -c \"import __graft_entry__ as g; "
                               "g.build()\"`); there is no fallback path")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(rc):
    """Raise AccrError for a negative status."""
    if rc != ACCR_OK:
        msg = lib().accr_last_error()
        raise AccrError(rc, msg.decode() if msg else "")
    return rc
