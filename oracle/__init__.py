"""ctypes binding of the serial C oracle (``oracle/oracle.c``).

TEST INFRASTRUCTURE ONLY.  Imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the product package, which
must fail loudly rather than fall back to this code.

Every function is the region's serial program with the OpenACC directives
ignored (IPMACC Sec. 1.3 and Listing 1a; the reduction clause of Stage 3.4
item iii and Stage 3.7), or the exactly rounded truth used for floating-point
tolerances.  Names of types and operators are plain strings:
types ``i32 i64 f32 f64``; operators ``add mul max min band bor bxor land lor``.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_TYPES = {"i32": 0, "i64": 1, "f32": 2, "f64": 3}
_OPS = {"add": 0, "mul": 1, "max": 2, "min": 3, "band": 4, "bor": 5,
        "bxor": 6, "land": 7, "lor": 8}
_NP = {"i32": np.int32, "i64": np.int64, "f32": np.float32, "f64": np.float64}

class OracleLib:
    """Binding of one build of the oracle (the default one, or a test build)."""

    def __init__(self, path):
        L = ctypes.CDLL(path)
        vp, i64, i = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        L.oracle_reduce.argtypes = [vp, i64, i64, i, i, i, vp, vp]
        L.oracle_rowreduce.argtypes = [vp, i64, i64, i64, i, i, i, vp, vp]
        L.oracle_segmented_reduce.argtypes = [vp, vp, i64, i, i, i, vp, vp]
        L.oracle_identity.argtypes = [i, i, vp]
        L.oracle_truth_sum.argtypes = [vp, i64, i64, i]
        L.oracle_truth_sum.restype = ctypes.c_double
        L.oracle_truth_abs_sum.argtypes = [vp, i64, i64, i]
        L.oracle_truth_abs_sum.restype = ctypes.c_double
        L.oracle_matmul_listing1.argtypes = [vp, vp, vp, i64]
        L.oracle_matmul_truth.argtypes = [vp, vp, vp, vp, i64]
        L.oracle_matmul_listing1_at.argtypes = [vp, vp, i64, i64, i64]
        L.oracle_matmul_listing1_at.restype = ctypes.c_float
        L.oracle_matmul_truth_at.argtypes = [vp, vp, i64, i64, i64, vp]
        L.oracle_matmul_truth_at.restype = ctypes.c_double
        L.oracle_matmul_listing1_rows_bt.argtypes = [vp, vp, vp, i64, i64, i64]
        L.oracle_matmul_truth_rows_bt.argtypes = [vp, vp, vp, vp, i64, i64, i64]
        L.oracle_nearest_k.argtypes = [vp, i64, ctypes.c_float, ctypes.c_float, i, vp, vp]
        L.oracle_standardize.argtypes = [vp, i64, vp, vp]
        L.oracle_grid_bfs.argtypes = [vp, i64, i64, i64, vp]
        L.oracle_grid_bfs.restype = i64
        self.L = L
        self.path = path

    def identity(self, op, acc):
        out = np.zeros(1, dtype=_NP[acc])
        if self.L.oracle_identity(_OPS[op], _TYPES[acc], _ptr(out)) != 0:
            raise ValueError("oracle: no identity for %s over %s" % (op, acc))
        return out[0]

    def reduce(self, x, op, acc=None, init=None):
        """var = var (op) x[i], i = 0..n-1 (serial), from init or the identity."""
        x = np.ascontiguousarray(x)
        t = _type_of(x)
        acc = acc or t
        out = np.zeros(1, dtype=_NP[acc])
        keep, ip = _init_buf(init, acc)
        rc = self.L.oracle_reduce(_ptr(x), x.size, 1, _TYPES[t], _OPS[op], _TYPES[acc], ip,
                                  _ptr(out))
        if rc != 0:
            raise ValueError("oracle: %s over %s into %s is not defined" % (op, t, acc))
        return out[0]

    def rowreduce(self, A, op, acc=None, init=None):
        """out[r] = serial fold of row r of the 2-D array A (rows may be padded)."""
        A = np.asarray(A)
        assert A.ndim == 2 and (A.shape[1] <= 1 or A.strides[1] == A.itemsize)
        t = _type_of(A)
        acc = acc or t
        rows, cols = A.shape
        ld = A.strides[0] // A.itemsize if rows > 1 else cols
        base = A if rows > 0 else np.zeros(1, dtype=A.dtype)
        out = np.zeros(rows, dtype=_NP[acc])
        keep, ip = _init_buf(init, acc)
        rc = self.L.oracle_rowreduce(ctypes.c_void_p(base.ctypes.data), rows, cols, ld,
                                     _TYPES[t], _OPS[op], _TYPES[acc], ip, _ptr(out))
        if rc != 0:
            raise ValueError("oracle: invalid row reduction")
        return out

    def segmented_reduce(self, values, offsets, op, acc=None, init=None):
        """out[s] = serial fold of values[offsets[s]:offsets[s+1]]."""
        values = np.ascontiguousarray(values)
        offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        t = _type_of(values)
        acc = acc or t
        nseg = offsets.size - 1
        out = np.zeros(nseg, dtype=_NP[acc])
        keep, ip = _init_buf(init, acc)
        rc = self.L.oracle_segmented_reduce(_ptr(values), _ptr(offsets), nseg, _TYPES[t],
                                            _OPS[op], _TYPES[acc], ip, _ptr(out))
        if rc != 0:
            raise ValueError("oracle: invalid segmented reduction")
        return out

    def truth_sum(self, x):
        """Exact sum of the float/double values, rounded once to double."""
        x = np.ascontiguousarray(x)
        return self.L.oracle_truth_sum(_ptr(x), x.size, 1, _TYPES[_type_of(x)])

    def truth_abs_sum(self, x):
        x = np.ascontiguousarray(x)
        return self.L.oracle_truth_abs_sum(_ptr(x), x.size, 1, _TYPES[_type_of(x)])

    def matmul_listing1(self, a, b):
        """Listing 1a with the directives ignored (float accumulator)."""
        a = np.ascontiguousarray(a, dtype=np.float32)
        b = np.ascontiguousarray(b, dtype=np.float32)
        n = a.shape[0]
        c = np.zeros((n, n), dtype=np.float32)
        self.L.oracle_matmul_listing1(_ptr(a), _ptr(b), _ptr(c), n)
        return c

    def matmul_truth(self, a, b):
        """(c64, absab): double-accumulated product and sum_l |a_il b_lj|."""
        a = np.ascontiguousarray(a, dtype=np.float32)
        b = np.ascontiguousarray(b, dtype=np.float32)
        n = a.shape[0]
        c = np.zeros((n, n), dtype=np.float64)
        s = np.zeros((n, n), dtype=np.float64)
        self.L.oracle_matmul_truth(_ptr(a), _ptr(b), _ptr(c), _ptr(s), n)
        return c, s

    def matmul_listing1_at(self, a, b, i, j):
        assert a.dtype == np.float32 and b.dtype == np.float32
        assert a.flags.c_contiguous and b.flags.c_contiguous
        n = a.shape[0]
        return np.float32(self.L.oracle_matmul_listing1_at(_ptr(a), _ptr(b), n, i, j))

    def matmul_truth_at(self, a, b, i, j):
        assert a.dtype == np.float32 and b.dtype == np.float32
        assert a.flags.c_contiguous and b.flags.c_contiguous
        n = a.shape[0]
        s = np.zeros(1, dtype=np.float64)
        c = self.L.oracle_matmul_truth_at(_ptr(a), _ptr(b), n, i, j, _ptr(s))
        return c, s[0]

    def _row_blocks(self, n, fn, threads):
        import concurrent.futures as cf
        threads = max(1, min(threads or os.cpu_count() or 1, n or 1))
        step = -(-n // threads) if n else 1
        with cf.ThreadPoolExecutor(max_workers=threads) as ex:   # ctypes releases the GIL
            list(ex.map(lambda i0: fn(i0, min(i0 + step, n)), range(0, n, step)))

    def matmul_listing1_threads(self, a, b, threads=None):
        """matmul_listing1 with rows split over host threads (b read through
        its transpose); the same bits, each entry computed as Listing 1a does."""
        a = np.ascontiguousarray(a, dtype=np.float32)
        bt = np.ascontiguousarray(np.asarray(b, dtype=np.float32).T)
        n = a.shape[0]
        c = np.zeros((n, n), dtype=np.float32)
        self._row_blocks(n, lambda i0, i1: self.L.oracle_matmul_listing1_rows_bt(
            _ptr(a), _ptr(bt), _ptr(c), n, i0, i1), threads)
        return c

    def matmul_truth_threads(self, a, b, threads=None):
        """matmul_truth with rows split over host threads."""
        a = np.ascontiguousarray(a, dtype=np.float32)
        bt = np.ascontiguousarray(np.asarray(b, dtype=np.float32).T)
        n = a.shape[0]
        c = np.zeros((n, n), dtype=np.float64)
        s = np.zeros((n, n), dtype=np.float64)
        self._row_blocks(n, lambda i0, i1: self.L.oracle_matmul_truth_rows_bt(
            _ptr(a), _ptr(bt), _ptr(c), _ptr(s), n, i0, i1), threads)
        return c, s


    def nearest_k(self, pts, qx, qy, k):
        """(idx[k], d2[k]): the k points nearest to (qx, qy) by squared distance,
        ties by index; pts is an (n, 2) float32 array."""
        pts = np.ascontiguousarray(pts, dtype=np.float32)
        n = pts.shape[0]
        idx = np.zeros(k, dtype=np.int64)
        d2 = np.zeros(k, dtype=np.float32)
        self.L.oracle_nearest_k(_ptr(pts), n, ctypes.c_float(qx), ctypes.c_float(qy), k, _ptr(idx), _ptr(d2))
        return idx, d2

    def standardize(self, x):
        """(y, (mean, var)): y = (x - mean) / sqrt(var) as the serial program computes it."""
        x = np.ascontiguousarray(x, dtype=np.float32)
        y = np.zeros_like(x)
        st = np.zeros(2, dtype=np.float64)
        self.L.oracle_standardize(_ptr(x), x.size, _ptr(y), _ptr(st))
        return y, (st[0], st[1])

    def grid_bfs(self, open_cells, src):
        """(dist, levels): BFS distances on the grid of open cells (uint8, 2-D)."""
        g = np.ascontiguousarray(open_cells, dtype=np.uint8)
        rows, cols = g.shape
        dist = np.zeros((rows, cols), dtype=np.int32)
        levels = self.L.oracle_grid_bfs(_ptr(g), rows, cols, int(src), _ptr(dist))
        return dist, int(levels)


def _type_of(a):
    for k, v in _NP.items():
        if a.dtype == np.dtype(v):
            return k
    raise TypeError("oracle: unsupported dtype %s" % a.dtype)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _init_buf(init, acc):
    if init is None:
        return None, None
    buf = np.array([init], dtype=_NP[acc])
    return buf, _ptr(buf)


_default = None


def default():
    """The oracle built from ``oracle/oracle.c`` (compiled on first use)."""
    global _default
    if _default is None:
        _default = OracleLib(_build.build())
    return _default


def identity(op, acc):
    return default().identity(op, acc)


def reduce(x, op, acc=None, init=None):
    return default().reduce(x, op, acc, init)


def rowreduce(A, op, acc=None, init=None):
    return default().rowreduce(A, op, acc, init)


def segmented_reduce(values, offsets, op, acc=None, init=None):
    return default().segmented_reduce(values, offsets, op, acc, init)


def truth_sum(x):
    return default().truth_sum(x)


def truth_abs_sum(x):
    return default().truth_abs_sum(x)


def matmul_listing1(a, b):
    return default().matmul_listing1(a, b)


def matmul_truth(a, b):
    return default().matmul_truth(a, b)


def matmul_listing1_threads(a, b, threads=None):
    return default().matmul_listing1_threads(a, b, threads)


def matmul_truth_threads(a, b, threads=None):
    return default().matmul_truth_threads(a, b, threads)


def matmul_listing1_at(a, b, i, j):
    return default().matmul_listing1_at(a, b, i, j)


def matmul_truth_at(a, b, i, j):
    return default().matmul_truth_at(a, b, i, j)


def nearest_k(pts, qx, qy, k):
    return default().nearest_k(pts, qx, qy, k)


def standardize(x):
    return default().standardize(x)


def grid_bfs(open_cells, src):
    return default().grid_bfs(open_cells, src)
