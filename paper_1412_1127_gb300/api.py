"""Python binding of the accr C ABI: argument marshalling only.

Each function has the name of the C entry point it calls (``include/accr.h``)
and takes torch tensors for device arrays.  PyTorch provides device memory and
streams; every step of a region runs in the library's CUDA kernels.
"""
import ctypes

import torch

from . import _native
from ._native import Clause, check, lib

ACCR_I32, ACCR_I64, ACCR_F32, ACCR_F64 = 0, 1, 2, 3
ACCR_ADD, ACCR_MUL, ACCR_MAX, ACCR_MIN, ACCR_BAND, ACCR_BOR, ACCR_BXOR, ACCR_LAND, ACCR_LOR = range(9)
ACCR_COMPENSATED, ACCR_SYNC, ACCR_TWO_LEVEL_HOST = 0x1, 0x2, 0x4
ACCR_MAX_CLAUSES = 4

OPS = {"add": ACCR_ADD, "mul": ACCR_MUL, "max": ACCR_MAX, "min": ACCR_MIN, "band": ACCR_BAND,
       "bor": ACCR_BOR, "bxor": ACCR_BXOR, "land": ACCR_LAND, "lor": ACCR_LOR,
       "+": ACCR_ADD, "*": ACCR_MUL, "&": ACCR_BAND, "|": ACCR_BOR, "^": ACCR_BXOR,
       "&&": ACCR_LAND, "||": ACCR_LOR}
TYPES = {torch.int32: ACCR_I32, torch.int64: ACCR_I64, torch.float32: ACCR_F32,
         torch.float64: ACCR_F64}
_CT = {ACCR_I32: ctypes.c_int32, ACCR_I64: ctypes.c_int64, ACCR_F32: ctypes.c_float,
       ACCR_F64: ctypes.c_double}


def type_of(dtype):
    try:
        return TYPES[dtype]
    except KeyError:
        raise TypeError("accr: unsupported dtype %s" % dtype)


def op_of(op):
    return OPS[op] if isinstance(op, str) else int(op)


class clause:
    """One ``reduction(op:var)`` clause: the variable is `out` (its dtype is the
    variable's type); `init` is its value before the region (None = identity)."""

    def __init__(self, op, out, init=None):
        self.op = op_of(op)
        self.out = out
        self.acc_type = type_of(out.dtype)
        self.init = init

    def _c(self, keep):
        c = Clause()
        c.op = self.op
        c.acc_type = self.acc_type
        if self.init is None:
            c.init = None
        else:
            v = _CT[self.acc_type](self.init)
            keep.append(v)
            c.init = ctypes.cast(ctypes.pointer(v), ctypes.c_void_p)
        c.out = self.out.data_ptr()
        return c


def _clauses(cls):
    keep = []
    arr = (Clause * len(cls))(*[c._c(keep) for c in cls])
    return arr, keep


def _stream(stream):
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def accr_reduce(x, clauses, flags=0, stream=None, n=None):
    """One region: fold the elements of the 1-D CUDA tensor `x` (its first `n`)
    into each clause's variable in a single pass."""
    assert x.is_cuda and x.dim() == 1 and (x.stride(0) == 1 or x.numel() <= 1)
    n = x.numel() if n is None else n
    assert 0 <= n <= x.numel()
    two_level = bool(flags & ACCR_TWO_LEVEL_HOST)
    for c in clauses:
        assert c.out.numel() >= 1 and c.out.is_cuda != two_level
    arr, keep = _clauses(clauses)
    return check(lib().accr_reduce(x.data_ptr() if x.numel() else None, n, type_of(x.dtype), arr,
                                   len(clauses), flags, _stream(stream)))


def accr_reduce_noalloc(x, clauses, flags=0, stream=None, n=None):
    """accr_reduce for callers that cannot allocate device memory: the block
    partials and counter live in a fixed array inside the library.  Calls
    that overlap on the GPU race on that array; serialise them."""
    assert x.is_cuda and x.dim() == 1 and (x.stride(0) == 1 or x.numel() <= 1)
    n = x.numel() if n is None else n
    assert 0 <= n <= x.numel()
    for c in clauses:
        assert c.out.is_cuda and c.out.numel() >= 1
    arr, keep = _clauses(clauses)
    return check(lib().accr_reduce_noalloc(x.data_ptr() if x.numel() else None, n, type_of(x.dtype),
                                           arr, len(clauses), flags, _stream(stream)))


def accr_rowreduce(A, clauses, flags=0, stream=None):
    """Row nest: out[i] = fold of row i of the 2-D CUDA tensor A (rows may be
    padded: A may be a column slice of a wider row-major matrix)."""
    assert A.is_cuda and A.dim() == 2 and (A.stride(1) == 1 or A.shape[1] <= 1)
    rows, cols = A.shape
    ld = A.stride(0) if rows > 1 else cols
    for c in clauses:
        assert c.out.is_cuda and c.out.numel() >= rows
    arr, keep = _clauses(clauses)
    return check(lib().accr_rowreduce(A.data_ptr() if A.numel() else None, rows, cols, max(ld, cols),
                                      type_of(A.dtype), arr, len(clauses), flags, _stream(stream)))


def accr_last_error():
    return lib().accr_last_error().decode()


def accr_launch_count():
    return int(lib().accr_launch_count())


def accr_version():
    return int(lib().accr_version())
