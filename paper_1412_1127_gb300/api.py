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
ACCR_COMPENSATED, ACCR_SYNC, ACCR_TWO_LEVEL_HOST, ACCR_PLAIN, ACCR_UNFUSED = 0x1, 0x2, 0x4, 0x8, 0x10
ACCR_MAX_CLAUSES = 4
ACCR_SMALL_BYTES = 65536   # default split of batched regions (include/accr.h)
ACCR_TILE_BYTES = 2097152

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
        assert c.out.numel() >= 1
        assert (not c.out.is_cuda) if two_level else (c.out.is_cuda or c.out.is_pinned())
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


def _region_desc(x, clauses, flags, keep):
    return _region(x, clauses, flags, keep, need_out=False)


def _region(x, clauses, flags, keep, need_out=True):
    assert x.is_cuda and x.dim() == 1 and (x.stride(0) == 1 or x.numel() <= 1)
    assert 1 <= len(clauses) <= ACCR_MAX_CLAUSES
    g = _native.Region()
    g.in_ = x.data_ptr() if x.numel() else None
    g.n = x.numel()
    g.in_type = type_of(x.dtype)
    g.nclauses = len(clauses)
    g.flags = flags
    g.reserved = 0
    for i, c in enumerate(clauses):
        if need_out:
            assert c.out.is_cuda and c.out.numel() >= 1
        g.clauses[i] = c._c(keep)
    return g


def regions_array(regions, need_out=True):
    """ctypes array of ``accr_region`` from (tensor, [clause...], flags) triples."""
    keep = []
    arr = (_native.Region * max(len(regions), 1))()
    for i, (x, cls, fl) in enumerate(regions):
        arr[i] = _region(x, cls, fl, keep, need_out)
    return arr, keep


def accr_batch_reduce(regions, flags=0, stream=None):
    """Many independent regions in one launch.  `regions` is a list of
    (1-D CUDA tensor, [clause, ...], flags) triples; each clause's `out` is a
    one-element CUDA tensor (or a one-element view into a larger one)."""
    arr, keep = regions_array(regions)
    return check(lib().accr_batch_reduce(arr, len(regions), flags, _stream(stream)))


def accr_segmented_reduce(values, offsets, clauses, flags=0, stream=None):
    """Segments values[offsets[s]:offsets[s+1]] of one CUDA tensor, one
    variable per segment in each clause's `out` array (length nseg).
    `offsets` is a host sequence of nseg + 1 element offsets."""
    import numpy as np
    assert values.is_cuda and values.dim() == 1 and (values.stride(0) == 1 or values.numel() <= 1)
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    nseg = off.size - 1
    assert nseg >= 0 and (nseg == 0 or off[-1] <= values.numel())
    for c in clauses:
        assert c.out.is_cuda and c.out.numel() >= nseg
    arr, keep = _clauses(clauses)
    return check(lib().accr_segmented_reduce(
        values.data_ptr() if values.numel() else None,
        off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), nseg, type_of(values.dtype), arr,
        len(clauses), flags, _stream(stream)))


class Batch:
    """A prepared batch (accr_batch_create): launch() replays its CUDA graph."""

    def __init__(self, regions):
        arr, keep = regions_array(regions)
        h = ctypes.c_void_p()
        check(lib().accr_batch_create(arr, len(regions), 0, ctypes.byref(h)))
        self.handle = h
        self._tensors = [(x, [c.out for c in cls]) for x, cls, _ in regions]

    def launch(self, stream=None):
        return check(lib().accr_batch_launch(self.handle, _stream(stream)))

    def destroy(self):
        if self.handle:
            check(lib().accr_batch_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def accr_batch_create(regions):
    return Batch(regions)


def accr_batch_launch(batch, stream=None):
    return batch.launch(stream)


def accr_batch_destroy(batch):
    return batch.destroy()


def accr_batch_tiling(small_bytes=0, tile_bytes=0):
    """Set the batched-region split (0 keeps a value); returns the old values."""
    os_, ot = ctypes.c_int64(), ctypes.c_int64()
    check(lib().accr_batch_tiling(small_bytes, tile_bytes, ctypes.byref(os_), ctypes.byref(ot)))
    return os_.value, ot.value


class Server:
    """The served request loop (accr_server_create ... accr_server_destroy)."""

    def __init__(self, hbm_budget_bytes, nstreams=4, max_batch=1024):
        h = ctypes.c_void_p()
        check(lib().accr_server_create(int(hbm_budget_bytes), nstreams, max_batch, ctypes.byref(h)))
        self.handle = h
        self._keep = {}

    def submit(self, x, clauses, flags=0):
        """Queue one region over the CUDA tensor x; clauses give (op, variable
        dtype) through `clause(op, out)` where only out's dtype is used."""
        keep = []
        g = _region_desc(x, clauses, flags, keep)
        t = ctypes.c_uint64()
        check(lib().accr_submit(self.handle, ctypes.byref(g), ctypes.byref(t)))
        self._keep[t.value] = (x, keep)
        return t.value

    def poll(self, ticket, timeout_us=60_000_000):
        """(status, [values...], result) of a ticket, waiting at most timeout_us
        (-1: no limit); returns (ACCR_EAGAIN / ACCR_ETIMEDOUT, None, ...) if it
        is not ready."""
        r = _native.Result()
        rc = lib().accr_poll(self.handle, ticket, ctypes.byref(r), int(timeout_us))
        if rc == _native.ACCR_EAGAIN or rc == _native.ACCR_ETIMEDOUT:
            return rc, None, r
        self._keep.pop(ticket, None)
        check(rc)
        return rc, list(r.value[: r.nclauses]), r

    def replay(self, regions, arrival_s, plain=False, stream=None):
        return accr_server_replay(self, regions, arrival_s, plain, stream)

    def destroy(self):
        if self.handle:
            check(lib().accr_server_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def decode(bits, dtype):
    """A variable's value from the 64-bit slot of an accr_result."""
    import numpy as np
    nd = {torch.int32: np.int32, torch.int64: np.int64, torch.float32: np.float32,
          torch.float64: np.float64}[dtype]
    b = np.array([bits], dtype=np.uint64)
    if np.dtype(nd).itemsize == 4:
        return b.astype(np.uint32).view(nd)[0]
    return b.view(nd)[0]


def accr_server_replay(server, regions, arrival_s, plain=False, stream=None):
    """Open-loop client: region i is submitted at arrival_s[i] seconds after
    the call starts; with plain=True each region instead runs as one
    synchronous single-region launch (server may be None).  Returns the ctypes
    array of accr_result (values decode with `decode`)."""
    import numpy as np
    arr, keep = regions_array(regions, need_out=False)
    at = np.ascontiguousarray(np.asarray(arrival_s, dtype=np.float64))
    assert at.size == len(regions)
    res = (_native.Result * max(len(regions), 1))()
    handle = server.handle if server is not None else None
    check(lib().accr_server_replay(handle, arr, at.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                   len(regions), ACCR_PLAIN if plain else 0, _stream(stream), res))
    return res


ACCR_MM_SIMT, ACCR_MM_SIMT_SERIAL, ACCR_MM_BF16X3 = 0, 1, 2
ACCR_MM_REUSE_SPLIT = 0x20
MM_MODES = {"simt": ACCR_MM_SIMT, "serial": ACCR_MM_SIMT_SERIAL, "bf16x3": ACCR_MM_BF16X3}


def accr_matmul_nest(a, b, c, mode="simt", flags=0, stream=None):
    """Listing 1a: c = a @ b for len x len row-major float CUDA tensors."""
    n = a.shape[0]
    for t in (a, b, c):
        assert t.is_cuda and t.dtype == torch.float32 and t.is_contiguous() and tuple(t.shape) == (n, n)
    m = MM_MODES[mode] if isinstance(mode, str) else int(mode)
    return check(lib().accr_matmul_nest(a.data_ptr() if n else None, b.data_ptr() if n else None,
                                        c.data_ptr() if n else None, n, m, flags, _stream(stream)))


ACCR_FAULT_ALLOC, ACCR_FAULT_LAUNCH, ACCR_FAULT_ADMIT = 1, 2, 3


def accr_fault_inject(kind, count):
    """Host-side fault injection for tests (see include/accr.h)."""
    return check(lib().accr_fault_inject(int(kind), int(count)))


def accr_probe_fma(ctas, rounds, sink, stream=None):
    """FP32 peak probe (2 * 16 * 256 * ctas * rounds flop); sink: CUDA float
    tensor of at least 256 * ctas elements."""
    assert sink.is_cuda and sink.dtype == torch.float32 and sink.numel() >= 256 * ctas
    return check(lib().accr_probe_fma(int(ctas), int(rounds), sink.data_ptr(), _stream(stream)))


def accr_probe_fma_packed(ctas, rounds, sink, stream=None):
    """FP32 peak probe with packed pairs (2 * 32 * 256 * ctas * rounds flop)."""
    assert sink.is_cuda and sink.dtype == torch.float32 and sink.numel() >= 256 * ctas
    return check(lib().accr_probe_fma_packed(int(ctas), int(rounds), sink.data_ptr(), _stream(stream)))


def accr_selftest_wait_timeout(tries=1000, stream=None):
    """Runs the bounded-wait self-test; returns its status code (ACCR_ETIMEDOUT expected)."""
    return int(lib().accr_selftest_wait_timeout(int(tries), _stream(stream)))


def accr_nearest_k(pts, qx, qy, k, idx_out, d2_out, flags=0, stream=None):
    """Nearest Neighbor: the k points of pts (CUDA float tensor (n, 2)) nearest
    to (qx, qy); indices into idx_out (int64[k]) and squared distances into
    d2_out (float[k])."""
    assert pts.is_cuda and pts.dtype == torch.float32 and pts.is_contiguous() and pts.dim() == 2
    assert idx_out.dtype == torch.int64 and d2_out.dtype == torch.float32
    assert idx_out.numel() >= k and d2_out.numel() >= k
    return check(lib().accr_nearest_k(pts.data_ptr() if pts.numel() else None, pts.shape[0], float(qx), float(qy),
                                      int(k), idx_out.data_ptr(), d2_out.data_ptr(), flags, _stream(stream)))


def accr_standardize(x, y, stats, flags=0, stream=None):
    """SRAD pattern: stats <- (mean, var) of x; y <- (x - mean) / sqrt(var)."""
    assert x.is_cuda and x.dtype == torch.float32 and x.is_contiguous()
    assert y.is_cuda and y.dtype == torch.float32 and y.numel() == x.numel()
    assert stats.is_cuda and stats.dtype == torch.float64 and stats.numel() >= 2
    return check(lib().accr_standardize(x.data_ptr() if x.numel() else None, x.numel(),
                                        y.data_ptr() if y.numel() else None, stats.data_ptr(), flags,
                                        _stream(stream)))


ACCR_BFS_REDUCE, ACCR_BFS_GUARDED, ACCR_BFS_PERSISTENT = 0, 1, 2
BFS_MODES = {"reduce": 0, "guarded": 1, "persistent": 2}


def accr_grid_bfs(open_cells, src, dist, mode="reduce", stream=None):
    """BFS pattern: distances on a grid of open cells (CUDA uint8 (rows, cols));
    returns the number of levels."""
    assert open_cells.is_cuda and open_cells.dtype == torch.uint8 and open_cells.is_contiguous()
    assert dist.is_cuda and dist.dtype == torch.int32 and dist.shape == open_cells.shape
    rows, cols = open_cells.shape
    lv = ctypes.c_int64()
    m = BFS_MODES[mode] if isinstance(mode, str) else int(mode)
    check(lib().accr_grid_bfs(open_cells.data_ptr(), rows, cols, int(src), dist.data_ptr(), m,
                              ctypes.byref(lv), _stream(stream)))
    return lv.value


def accr_last_error():
    return lib().accr_last_error().decode()


def accr_launch_count():
    return int(lib().accr_launch_count())


def accr_version():
    return int(lib().accr_version())


def accr_debug_report(clear=True):
    """(violations, first failing site, checked) of a debug build's bounds
    checks; checked is False for release builds (see include/accr.h)."""
    v, site, chk = ctypes.c_uint64(), ctypes.c_uint32(), ctypes.c_int32()
    check(lib().accr_debug_report(ctypes.byref(v), ctypes.byref(site), ctypes.byref(chk), int(bool(clear))))
    return int(v.value), int(site.value), bool(chk.value)
