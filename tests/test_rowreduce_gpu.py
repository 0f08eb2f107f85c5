"""accr_rowreduce (gang = row, vector = column) on the GPU against the oracle."""
import math

import numpy as np
import pytest
import torch

import oracle
from guard import guarded
from paper_1412_1127_gb300 import api, inputs
from tolerances import TOL_F32, TOL_F32_COMP, same_bits

pytestmark = pytest.mark.gpu

TD = {"i32": torch.int32, "i64": torch.int64, "f32": torch.float32, "f64": torch.float64}
SHAPES = [(1, 1), (3, 5), (7, 33), (64, 128), (129, 1023), (1000, 4096), (5, 70001), (37, 0)]


def gpu_rows(A_np, op, acc, init=None, flags=0, pad=0, offset=0):
    rows, cols = A_np.shape
    big = np.zeros((rows, cols + pad + offset), dtype=A_np.dtype)
    big[:, offset:offset + cols] = A_np
    t = torch.from_numpy(big).cuda()[:, offset:offset + cols]
    out = guarded((rows,), TD[acc], 9)
    api.accr_rowreduce(t, [api.clause(op, out.t, init)], flags=flags)
    return out.check("row %s into %s, %dx%d" % (op, acc, rows, cols)).cpu().numpy()


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("op", ["add", "mul", "max", "min", "band", "bor", "bxor", "land", "lor"])
def test_int_rows_bit_exact(shape, op):
    g = np.random.default_rng(shape[0] * 7 + shape[1])
    A = g.integers(-(1 << 31), 1 << 31, size=shape, dtype=np.int64).astype(np.int32)
    if op == "land":
        A |= 1
        A[::3, -1:] = 0
    for pad, off in [(0, 0), (3, 1)]:
        assert np.array_equal(gpu_rows(A, op, "i64", pad=pad, offset=off), oracle.rowreduce(A, op, "i64"))
        assert np.array_equal(gpu_rows(A, op, "i32", init=5, pad=pad, offset=off),
                              oracle.rowreduce(A, op, "i32", init=5))


@pytest.mark.parametrize("shape", SHAPES)
def test_fp_rows(shape):
    A = inputs.uniform_matrix(*shape)
    for op in ["max", "min"]:
        for pad, off in [(0, 0), (5, 3)]:
            assert same_bits(gpu_rows(A, op, "f32", pad=pad, offset=off), oracle.rowreduce(A, op))
    rows, cols = shape
    for flags, tol in [(0, TOL_F32), (api.ACCR_COMPENSATED, TOL_F32_COMP)]:
        got = gpu_rows(A, "add", "f32", flags=flags, pad=1)
        for r in range(rows):
            truth = oracle.truth_sum(A[r])
            err = abs(float(got[r]) - truth) / max(abs(truth), 0.1 * math.sqrt(max(cols, 1)) * 0.577)
            assert err <= tol, (r, got[r], truth)
    D = A.astype(np.float64)
    got = gpu_rows(D, "add", "f64")
    for r in range(rows):
        truth = oracle.truth_sum(D[r])
        assert abs(got[r] - truth) <= 1e-12 * max(abs(truth), 0.1 * math.sqrt(max(cols, 1)))


def test_two_clauses_rows_full_size():
    # row sum and row max of a 65536 x 4096 U(-1,1) float matrix in one pass
    A = inputs.uniform_matrix(65536, 4096)
    At = torch.from_numpy(A).cuda()
    gs, gm = guarded((65536,), torch.float32), guarded((65536,), torch.float32)
    api.accr_rowreduce(At, [api.clause("add", gs.t), api.clause("max", gm.t)])
    m_np, s_np = gm.check("row max").cpu().numpy(), gs.check("row sum").cpu().numpy()
    assert same_bits(m_np, oracle.rowreduce(A, "max"))
    # every row's sum against its exact sum (host threads; ctypes releases the GIL)
    import concurrent.futures as cf
    with cf.ThreadPoolExecutor(max_workers=16) as ex:
        truths = np.array(list(ex.map(lambda r: oracle.truth_sum(A[r]), range(65536))))
    err = np.abs(s_np.astype(np.float64) - truths) / np.maximum(np.abs(truths), 0.1 * 64 * 0.577)
    assert float(err.max()) <= TOL_F32, (int(err.argmax()), float(err.max()))


PAIR_CASES = [  # (element type, sum variable, flags) for the fixed-code two-clause kernels
    ("i32", "i32", 0), ("i32", "i64", 0), ("i64", "i64", 0),
    ("f32", "f32", 0), ("f32", "f32", api.ACCR_COMPENSATED), ("f64", "f64", 0)]


@pytest.mark.parametrize("t,acc,flags", PAIR_CASES)
@pytest.mark.parametrize("ext", ["max", "min"])
@pytest.mark.parametrize("sum_first", [True, False])
@pytest.mark.parametrize("shape", [(129, 1023), (300, 4096), (3, 70001)])
def test_sum_and_extreme_pairs(t, acc, flags, ext, sum_first, shape):
    """A sum and a max/min in one pass, in either clause order: each variable
    gets its own row fold (integers bit-exact, float extremes bit-exact, float
    sums within the sum tolerance)."""
    g = np.random.default_rng(shape[0] + shape[1])
    if t in ("i32", "i64"):
        A = g.integers(-(1 << 31), 1 << 31, size=shape, dtype=np.int64).astype(np.int32 if t == "i32" else np.int64)
    else:
        A = inputs.uniform_matrix(*shape)
        A = A.astype(np.float64) if t == "f64" else A
    At = torch.from_numpy(A).cuda()
    rows, cols = shape
    gs, gm = guarded((rows,), TD[acc], 9), guarded((rows,), TD[t], 9)
    cls = [api.clause("add", gs.t), api.clause(ext, gm.t)]
    api.accr_rowreduce(At, cls if sum_first else cls[::-1], flags=flags)
    s_np, m_np = gs.check("row sum").cpu().numpy(), gm.check("row " + ext).cpu().numpy()
    want_m = oracle.rowreduce(A, ext, t) if t in ("i32", "i64") else oracle.rowreduce(A, ext)
    if t in ("i32", "i64"):
        assert np.array_equal(m_np, want_m)
        assert np.array_equal(s_np, oracle.rowreduce(A, "add", acc))
        return
    assert same_bits(m_np, want_m)
    tol = TOL_F32_COMP if flags else (TOL_F32 if t == "f32" else 1e-12)
    for r in range(0, rows, max(1, rows // 40)):
        truth = oracle.truth_sum(A[r])
        assert abs(float(s_np[r]) - truth) / max(abs(truth), 0.1 * math.sqrt(cols) * 0.577) <= tol, (r, t)


def test_generic_two_clause_rows():
    """A pair outside the fixed-code set (product and xor) runs the generic fold."""
    g = np.random.default_rng(5)
    A = g.integers(-(1 << 31), 1 << 31, size=(77, 3000), dtype=np.int64).astype(np.int32)
    At = torch.from_numpy(A).cuda()
    p, x = guarded((77,), torch.int64), guarded((77,), torch.int32)
    api.accr_rowreduce(At, [api.clause("mul", p.t), api.clause("bxor", x.t)])
    assert np.array_equal(p.check("row product").cpu().numpy(), oracle.rowreduce(A, "mul", "i64"))
    assert np.array_equal(x.check("row xor").cpu().numpy(), oracle.rowreduce(A, "bxor", "i32"))


@pytest.mark.slow
@pytest.mark.parametrize("shape", [(4, 1 << 24), (64, 1 << 22)])
def test_long_rows_split_path(shape):
    """A few long rows (the split-row form: each row cut into CTA tiles):
    every row's max bit-exact, every row's sum within the float tolerance of
    its exact sum, the same bits on a repeat, and one row alone gives the
    same bits as inside the matrix (the split depends on the row length only)."""
    import concurrent.futures as cf
    rows, cols = shape
    A = inputs.uniform_matrix(rows, cols, salt=rows)
    At = torch.from_numpy(A).cuda()
    gs, gm = guarded((rows,), torch.float32), guarded((rows,), torch.float32)
    api.accr_rowreduce(At, [api.clause("add", gs.t), api.clause("max", gm.t)])
    s_np, m_np = gs.check("row sum").cpu().numpy(), gm.check("row max").cpu().numpy()
    assert same_bits(m_np, oracle.rowreduce(A, "max"))
    with cf.ThreadPoolExecutor(max_workers=16) as ex:
        truths = list(ex.map(lambda r: oracle.truth_sum(A[r]), range(rows)))
    for r, truth in enumerate(truths):
        assert abs(float(s_np[r]) - truth) / max(abs(truth), 0.1 * math.sqrt(cols) * 0.577) <= TOL_F32, r
    s2 = torch.empty(rows, dtype=torch.float32, device="cuda")
    api.accr_rowreduce(At, [api.clause("add", s2)])
    assert same_bits(s2.cpu().numpy(), s_np)
    one = torch.empty(1, dtype=torch.float32, device="cuda")
    api.accr_rowreduce(At[rows - 1:rows], [api.clause("add", one)])
    assert same_bits(one.cpu().numpy(), s_np[rows - 1:rows])


def test_long_integer_rows_split_path():
    """Integer rows past the split-row threshold, with padded rows (ld not a
    multiple of the vector) and three clauses (two passes over each row)."""
    g = np.random.default_rng(17)
    A = g.integers(-(1 << 40), 1 << 40, size=(3, (1 << 20) + 7), dtype=np.int64)
    for pad, off in [(0, 0), (3, 1)]:
        big = np.zeros((3, A.shape[1] + pad + off), dtype=np.int64)
        big[:, off:off + A.shape[1]] = A
        t = torch.from_numpy(big).cuda()[:, off:off + A.shape[1]]
        outs = [guarded((3,), torch.int64, 5) for _ in range(3)]
        api.accr_rowreduce(t, [api.clause("add", outs[0].t), api.clause("bxor", outs[1].t, init=9),
                               api.clause("min", outs[2].t)])
        for o, (op, init) in zip(outs, [("add", None), ("bxor", 9), ("min", None)]):
            assert np.array_equal(o.check(op).cpu().numpy(), oracle.rowreduce(A, op, "i64", init=init)), (op, pad)


@pytest.mark.parametrize("rows,cols", [(5, (1 << 18) + 13), (300, (1 << 16) + 3)])
@pytest.mark.parametrize("pad,off", [(0, 0), (3, 1)])
def test_split_rows_cross_runs_and_padding(rows, cols, pad, off):
    """4-byte rows past the split-row threshold (one 1024-thread CTA per SM):
    rows whose chunks start off the 16-byte grid (ld not a multiple of the
    vector, an offset base), and CTA runs that end mid-row or cover several
    rows, so one CTA counts into many rows and rows complete in any CTA.
    Integer results bit-exact: a sum into int64 with a max (the fixed-code
    pair), a lone int32 sum, and a float sum within its tolerance."""
    g = np.random.default_rng(rows + pad)
    A = g.integers(-1000, 1000, size=(rows, cols), dtype=np.int32)
    big = np.zeros((rows, cols + pad + off), dtype=np.int32)
    big[:, off:off + cols] = A
    t = torch.from_numpy(big).cuda()[:, off:off + cols]
    s64, mx = guarded((rows,), torch.int64, 5), guarded((rows,), torch.int32, 5)
    api.accr_rowreduce(t, [api.clause("add", s64.t), api.clause("max", mx.t)])
    assert np.array_equal(s64.check("sum").cpu().numpy(), oracle.rowreduce(A, "add", "i64"))
    assert np.array_equal(mx.check("max").cpu().numpy(), oracle.rowreduce(A, "max", "i32"))
    s32 = guarded((rows,), torch.int32, 5)
    api.accr_rowreduce(t, [api.clause("add", s32.t, init=7)])
    assert np.array_equal(s32.check("sum32").cpu().numpy(), oracle.rowreduce(A, "add", "i32", init=7))
    F = (A.astype(np.float32) / np.float32(1000.0)).astype(np.float32)
    fbig = np.zeros((rows, cols + pad + off), dtype=np.float32)
    fbig[:, off:off + cols] = F
    ft = torch.from_numpy(fbig).cuda()[:, off:off + cols]
    fs = guarded((rows,), torch.float32, 5)
    api.accr_rowreduce(ft, [api.clause("add", fs.t)])
    got = fs.check("fsum").cpu().numpy()
    for r in range(0, rows, max(1, rows // 16)):
        truth = oracle.truth_sum(F[r])
        assert abs(float(got[r]) - truth) / max(abs(truth), 0.1 * math.sqrt(cols) * 0.577) <= TOL_F32, r
