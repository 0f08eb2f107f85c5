"""Pins for the serial oracle: facts fixed by mathematics, not by the oracle.

Each ``pin_*`` takes an oracle binding (``oracle.OracleLib``) and raises
AssertionError if the oracle disagrees with

* closed forms (sum of 1..n, constant arrays, the XOR-of-0..n-1 pattern,
  products of -1, identities on empty input),
* brute force on tiny inputs with Python's unbounded integers,
* library routines whose result is the definition (``math.fsum`` is the
  correctly rounded sum; ``numpy.cumsum`` is a sequential float fold; integer
  prefix sums / prefix XORs taken modulo 2^64),
* invariants (permutation, split, x ^ x = 0, bounds of max/min),
* and, for the Listing-1a nest (IPMACC Sec. 1.3), exact small-integer
  products, the identity matrix, and the transpose identity.

``test_oracle.py`` runs them on the oracle; ``test_oracle_mutants.py`` plants
mistakes in a copy of the oracle and checks that some pin catches each one.
"""
import math
from fractions import Fraction

import numpy as np

I32_MIN, I32_MAX = -(1 << 31), (1 << 31) - 1
I64_MIN, I64_MAX = -(1 << 63), (1 << 63) - 1
INT_OPS = ["add", "mul", "max", "min", "band", "bor", "bxor", "land", "lor"]
FP_OPS = ["add", "mul", "max", "min"]


def wrap(v, bits):
    """Two's-complement value of v modulo 2^bits."""
    v %= 1 << bits
    return v - (1 << bits) if v >= 1 << (bits - 1) else v


def py_fold(values, op, bits, init=None):
    """Independent fold over Python integers (unbounded), wrapped at the end."""
    ident = {"add": 0, "mul": 1, "max": -(1 << (bits - 1)), "min": (1 << (bits - 1)) - 1,
             "band": -1, "bor": 0, "bxor": 0, "land": 1, "lor": 0}
    acc = ident[op] if init is None else int(init)
    for v in values:
        v = int(v)
        if op == "add":
            acc = acc + v
        elif op == "mul":
            acc = acc * v
        elif op == "max":
            acc = max(acc, v)
        elif op == "min":
            acc = min(acc, v)
        elif op == "band":
            acc = acc & v
        elif op == "bor":
            acc = acc | v
        elif op == "bxor":
            acc = acc ^ v
        elif op == "land":
            acc = 1 if (acc != 0 and v != 0) else 0
        elif op == "lor":
            acc = 1 if (acc != 0 or v != 0) else 0
        acc = wrap(acc, bits)
    return acc


# --------------------------------------------------------------------------
# integer closed forms
# --------------------------------------------------------------------------
def pin_sum_1_to_n(orc):
    for n in [0, 1, 2, 31, 32, 33, 1000, 65537, 100000]:
        x = np.arange(1, n + 1, dtype=np.int32)
        t = n * (n + 1) // 2
        assert int(orc.reduce(x, "add", "i64")) == t, n
        assert int(orc.reduce(x, "add", "i32")) == wrap(t, 32), n
    x = np.arange(1, 1001, dtype=np.int64)
    assert int(orc.reduce(x, "add", "i64", init=7)) == 500500 + 7


def pin_constant_arrays(orc):
    for c in [-7, 0, 3, I32_MAX, I32_MIN]:
        for n in [1, 2, 5, 64]:
            x = np.full(n, c, dtype=np.int32)
            assert int(orc.reduce(x, "add", "i32")) == wrap(n * c, 32)
            assert int(orc.reduce(x, "add", "i64")) == n * c
            assert int(orc.reduce(x, "mul", "i32")) == wrap(c ** n, 32)
            assert int(orc.reduce(x, "mul", "i64")) == wrap(c ** n, 64)
            for op in ["max", "min", "band", "bor"]:
                assert int(orc.reduce(x, op, "i32")) == c, op
            assert int(orc.reduce(x, "bxor", "i32")) == (c if n % 2 else 0)
            assert int(orc.reduce(x, "land", "i32")) == (1 if c != 0 else 0)
            assert int(orc.reduce(x, "lor", "i64")) == (1 if c != 0 else 0)


def pin_xor_pattern(orc):
    # XOR of 0..m is m, 1, m+1, 0 for m = 0, 1, 2, 3 (mod 4)
    for n in range(0, 70):
        x = np.arange(n, dtype=np.int32)
        m = n - 1
        want = 0 if n == 0 else [m, 1, m + 1, 0][m % 4]
        assert int(orc.reduce(x, "bxor", "i32")) == want, n
        assert int(orc.reduce(x.astype(np.int64), "bxor", "i64")) == want, n


def pin_products(orc):
    for n in range(0, 40):
        x = np.full(n, -1, dtype=np.int32)
        assert int(orc.reduce(x, "mul", "i32")) == (-1) ** n
        y = np.full(n, 2, dtype=np.int32)
        assert int(orc.reduce(y, "mul", "i32")) == wrap(2 ** n, 32)
        assert int(orc.reduce(y, "mul", "i64")) == wrap(2 ** n, 64)


def pin_logical(orc):
    z = np.zeros(10, dtype=np.int32)
    assert int(orc.reduce(z, "land", "i32")) == 0
    assert int(orc.reduce(z, "lor", "i32")) == 0
    nz = np.arange(1, 11, dtype=np.int32) * -3
    assert int(orc.reduce(nz, "land", "i32")) == 1
    assert int(orc.reduce(nz, "lor", "i32")) == 1
    last0 = nz.copy()
    last0[-1] = 0
    assert int(orc.reduce(last0, "land", "i32")) == 0
    assert int(orc.reduce(last0, "lor", "i32")) == 1
    one = np.zeros(1000, dtype=np.int64)
    one[617] = 1 << 40  # nonzero only in the high word
    assert int(orc.reduce(one, "lor", "i64")) == 1
    # the variable's prior value takes part once; C semantics give 0 / 1
    e = np.zeros(0, dtype=np.int32)
    assert int(orc.reduce(e, "land", "i32", init=5)) == 5
    assert int(orc.reduce(np.array([3], np.int32), "land", "i32", init=5)) == 1
    assert int(orc.reduce(np.array([3], np.int32), "land", "i32", init=0)) == 0
    assert int(orc.reduce(np.array([0], np.int32), "lor", "i32", init=-9)) == 1


def pin_identities(orc):
    want = {
        "i32": {"add": 0, "mul": 1, "max": I32_MIN, "min": I32_MAX, "band": -1, "bor": 0,
                "bxor": 0, "land": 1, "lor": 0},
        "i64": {"add": 0, "mul": 1, "max": I64_MIN, "min": I64_MAX, "band": -1, "bor": 0,
                "bxor": 0, "land": 1, "lor": 0},
    }
    for acc, table in want.items():
        e = np.zeros(0, dtype=np.int32 if acc == "i32" else np.int64)
        for op, v in table.items():
            assert int(orc.identity(op, acc)) == v, (acc, op)
            assert int(orc.reduce(e, op, acc)) == v, (acc, op)
            assert int(orc.reduce(e, op, acc, init=123)) == 123
    for acc, dt in [("f32", np.float32), ("f64", np.float64)]:
        e = np.zeros(0, dtype=dt)
        assert orc.reduce(e, "add", acc) == 0.0
        assert orc.reduce(e, "mul", acc) == 1.0
        assert orc.reduce(e, "max", acc) == -np.inf
        assert orc.reduce(e, "min", acc) == np.inf
        assert orc.reduce(e, "add", acc, init=2.5) == 2.5


def pin_bruteforce_small(orc):
    V = [-2, -1, 0, 1, 2, I32_MIN, I32_MAX]
    arrays = [[]] + [[a] for a in V] + [[a, b] for a in V for b in V]
    arrays += [[a, b, c] for a in V for b in V for c in V]
    for vals in arrays:
        x = np.array(vals, dtype=np.int32)
        for op in INT_OPS:
            assert int(orc.reduce(x, op, "i32")) == py_fold(vals, op, 32), (vals, op)
            assert int(orc.reduce(x, op, "i64")) == py_fold(vals, op, 64), (vals, op)
    for vals in arrays[:60]:
        x = np.array(vals, dtype=np.int32)
        for op in INT_OPS:
            assert int(orc.reduce(x, op, "i64", init=-5)) == py_fold(vals, op, 64, -5)
            assert int(orc.reduce(x.astype(np.int64) * 3, op, "i64", init=9)) == \
                py_fold([3 * v for v in vals], op, 64, 9)


# --------------------------------------------------------------------------
# invariants
# --------------------------------------------------------------------------
def pin_invariants(orc):
    g = np.random.default_rng(5)
    for n in [1, 17, 1000]:
        x = g.integers(I32_MIN, I32_MAX + 1, size=n, dtype=np.int64).astype(np.int32)
        p = g.permutation(x)
        for op in INT_OPS:
            r = orc.reduce(x, op, "i32")
            assert orc.reduce(p, op, "i32") == r, op
            k = n // 3
            assert orc.reduce(x[k:], op, "i32", init=orc.reduce(x[:k], op, "i32")) == r, op
        assert int(orc.reduce(np.concatenate([x, p]), "bxor", "i32")) == 0
        mx, mn = int(orc.reduce(x, "max", "i32")), int(orc.reduce(x, "min", "i32"))
        assert mx >= int(x.max()) and mx in set(x.tolist())
        assert mn <= int(x.min()) and mn in set(x.tolist())
        # serial float folds split exactly at any point (same sequence)
        f = g.standard_normal(n).astype(np.float32)
        k = n // 2
        assert orc.reduce(f[k:], "add", "f32", init=orc.reduce(f[:k], "add", "f32")) == \
            orc.reduce(f, "add", "f32")


# --------------------------------------------------------------------------
# floating point
# --------------------------------------------------------------------------
def pin_f32_serial_stall(orc):
    n = (1 << 24) + 10
    x = np.ones(n, dtype=np.float32)
    # a float accumulator stops growing at 2^24 (1 + 2^24 rounds back)
    assert orc.reduce(x, "add", "f32") == np.float32(1 << 24)
    assert orc.reduce(x, "add", "f64") == float(n)
    assert orc.truth_sum(x) == float(n)


def pin_f32_serial_is_sequential(orc):
    g = np.random.default_rng(7)
    for n in [1, 5, 1000, 4097]:
        x = g.standard_normal(n).astype(np.float32)
        assert orc.reduce(x, "add", "f32") == np.cumsum(x, dtype=np.float32)[-1]
        y = np.concatenate([np.float32([1.5]), x])
        assert orc.reduce(x, "add", "f32", init=1.5) == np.cumsum(y, dtype=np.float32)[-1]
        assert orc.reduce(x, "add", "f64") == np.cumsum(x.astype(np.float64))[-1]
        d = g.standard_normal(n)
        assert orc.reduce(d, "add", "f64") == np.cumsum(d)[-1]
        m = (1.0 + g.random(n) * 1e-3).astype(np.float32)
        assert orc.reduce(m, "mul", "f32") == np.cumprod(m, dtype=np.float32)[-1]


def _fsum_cases():
    g = np.random.default_rng(11)
    yield g.standard_normal(100000)
    yield g.standard_normal(5000).astype(np.float32)
    e = g.integers(-1000, 1000, size=3000)
    yield np.ldexp(g.standard_normal(3000), e)
    a = g.standard_normal(2000) * 1e16
    yield g.permutation(np.concatenate([a, -a, g.standard_normal(10)]))
    yield np.array([1e308, 1e308, -1e308, -1e308, 1.0])
    yield np.array([5e-324] * 7 + [-5e-324, 2.2250738585072014e-308])
    yield np.array([1.0, 2.0 ** -53, 2.0 ** -53])           # ties-to-even needs sticky
    yield np.array([1.0, 2.0 ** -53])                        # exact tie: rounds to even
    yield np.array([1.0, 2.0 ** -53, 2.0 ** -105])           # just above the tie
    yield np.array([-1.0, -(2.0 ** -53), -(2.0 ** -53)])
    yield np.array([2.0 ** 1023, 2.0 ** 1023 * (1 - 2 ** -52), -(2.0 ** 1023)])
    yield (g.random(4096).astype(np.float32) * 2 - 1)
    yield np.array([], dtype=np.float64)


def _exact_sum(vals):
    """Correctly rounded sum: math.fsum, or exact rationals where fsum's
    intermediate overflows (int/int true division rounds correctly)."""
    try:
        return math.fsum(vals)
    except OverflowError:
        return _rational_sum(vals)


def _rational_sum(vals):
    f = sum((Fraction(v) for v in vals), Fraction(0))
    try:
        return float(f)
    except OverflowError:  # beyond the largest double: rounds to infinity
        return math.inf if f > 0 else -math.inf


def pin_truth_is_correctly_rounded(orc):
    for x in _fsum_cases():
        want = _exact_sum(x.tolist())
        if x.size <= 5000:
            assert want == _rational_sum(x.tolist())
        got = orc.truth_sum(x)
        assert got == want and math.copysign(1, got) == math.copysign(1, want) or \
            (got == 0 and want == 0), (x[:4], got, want)
        assert orc.truth_abs_sum(x) == _exact_sum([abs(v) for v in x.tolist()])


def pin_fp_minmax(orc):
    g = np.random.default_rng(13)
    for dt, acc in [(np.float32, "f32"), (np.float64, "f64")]:
        x = g.standard_normal(5001).astype(dt)
        assert orc.reduce(x, "max", acc) == x.max()
        assert orc.reduce(x, "min", acc) == x.min()
        assert orc.reduce(x, "max", acc, init=100.0) == 100.0
        for zs in ([-0.0, 0.0], [0.0, -0.0], [-0.0, -0.0, 0.0, -0.0]):
            z = np.array(zs, dtype=dt)
            assert not np.signbit(orc.reduce(z, "max", acc))
            assert np.signbit(orc.reduce(z, "min", acc))
        assert orc.reduce(np.array([-np.inf], dt), "max", acc) == -np.inf
    x = g.standard_normal(100).astype(np.float32)
    assert orc.reduce(x, "max", "f64") == float(x.max())


# --------------------------------------------------------------------------
# row nest and many regions
# --------------------------------------------------------------------------
def pin_rowreduce(orc):
    g = np.random.default_rng(17)
    A = g.integers(I32_MIN, I32_MAX + 1, size=(37, 53), dtype=np.int64).astype(np.int32)
    assert np.array_equal(orc.rowreduce(A, "add", "i64"), A.astype(np.int64).sum(axis=1))
    assert np.array_equal(orc.rowreduce(A, "max"), A.max(axis=1))
    assert np.array_equal(orc.rowreduce(A, "min"), A.min(axis=1))
    assert np.array_equal(orc.rowreduce(A, "bxor"), np.bitwise_xor.reduce(A, axis=1))
    big = g.integers(-100, 100, size=(9, 40), dtype=np.int64).astype(np.int32)
    view = big[:, 3:21]  # padded rows: leading dimension 40, 18 columns used
    assert np.array_equal(orc.rowreduce(view, "add", "i64"), view.astype(np.int64).sum(axis=1))
    F = g.standard_normal((11, 300)).astype(np.float32)
    assert np.array_equal(orc.rowreduce(F, "add"), np.cumsum(F, axis=1, dtype=np.float32)[:, -1])
    assert np.array_equal(orc.rowreduce(F, "max"), F.max(axis=1))
    E = np.zeros((4, 0), dtype=np.float32)
    assert np.all(orc.rowreduce(E, "max") == -np.inf)


def pin_segmented(orc):
    g = np.random.default_rng(19)
    lens = g.integers(0, 50, size=200)
    lens[::7] = 0
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    v = g.integers(-(1 << 62), 1 << 62, size=int(off[-1]), dtype=np.int64)
    # segment sums as prefix differences modulo 2^64 (numpy int64 wraps)
    with np.errstate(over="ignore"):
        cs = np.concatenate([[0], np.cumsum(v)]).astype(np.int64)
        want = cs[off[1:]] - cs[off[:-1]]
    assert np.array_equal(orc.segmented_reduce(v, off, "add"), want)
    px = np.concatenate([[0], np.bitwise_xor.accumulate(v)]).astype(np.int64)
    assert np.array_equal(orc.segmented_reduce(v, off, "bxor"), px[off[1:]] ^ px[off[:-1]])
    mx = orc.segmented_reduce(v, off, "max")
    for s in range(len(lens)):
        seg = v[off[s]:off[s + 1]]
        assert mx[s] == (seg.max() if seg.size else I64_MIN)


# --------------------------------------------------------------------------
# Listing-1a nest
# --------------------------------------------------------------------------
def pin_matmul_small_int(orc):
    g = np.random.default_rng(23)
    for n in [1, 2, 7, 16, 33]:
        a = g.integers(-16, 17, size=(n, n)).astype(np.float32)
        b = g.integers(-16, 17, size=(n, n)).astype(np.float32)
        exact = (a.astype(np.int64) @ b.astype(np.int64)).astype(np.float32)
        assert np.array_equal(orc.matmul_listing1(a, b), exact), n
        c64, s = orc.matmul_truth(a, b)
        assert np.array_equal(c64, exact.astype(np.float64))
        assert np.array_equal(s, np.abs(a).astype(np.int64) @ np.abs(b).astype(np.int64))


def pin_matmul_identity_and_transpose(orc):
    g = np.random.default_rng(29)
    n = 24
    a = (g.random((n, n)) * 2 - 1).astype(np.float32)
    b = (g.random((n, n)) * 2 - 1).astype(np.float32)
    eye = np.eye(n, dtype=np.float32)
    assert np.array_equal(orc.matmul_listing1(a, eye), a)
    assert np.array_equal(orc.matmul_listing1(eye, b), b)
    c = orc.matmul_listing1(a, b)
    # (AB)^T = B^T A^T with the same products summed in the same order
    assert np.array_equal(orc.matmul_listing1(b.T.copy(), a.T.copy()), c.T)
    for i, j in [(0, 0), (3, 17), (n - 1, n - 1)]:
        prods = (a[i, :] * b[:, j]).astype(np.float32)
        assert c[i, j] == np.cumsum(prods, dtype=np.float32)[-1]
        assert orc.matmul_listing1_at(a, b, i, j) == c[i, j]
    c64, s = orc.matmul_truth(a, b)
    ref = a.astype(np.float64) @ b.astype(np.float64)
    assert np.all(np.abs(c64 - ref) <= 1e-13 * s)
    assert np.allclose(s, np.abs(a).astype(np.float64) @ np.abs(b).astype(np.float64), rtol=1e-13)
    t, ts = orc.matmul_truth_at(a, b, 5, 6)
    assert t == c64[5, 6] and ts == s[5, 6]



def pin_matmul_row_blocks(orc):
    """The threaded row-block form (b read through its transpose): every entry
    is the sequential float sum of its products (numpy's float32 cumsum adds
    in index order, rounding each step), ragged row blocks included; the truth
    form agrees with a float64 product and exact small-integer sums."""
    g = np.random.default_rng(31)
    n = 37
    a = (g.random((n, n)) * 2 - 1).astype(np.float32)
    b = (g.random((n, n)) * 2 - 1).astype(np.float32)
    for threads in [1, 3, 8, 64]:
        c = orc.matmul_listing1_threads(a, b, threads)
        for i in range(n):
            prods = (a[i, :][:, None] * b).astype(np.float32)       # prods[l, j]
            assert np.array_equal(c[i], np.cumsum(prods, axis=0, dtype=np.float32)[-1]), (threads, i)
        c64, s = orc.matmul_truth_threads(a, b, threads)
        ref = a.astype(np.float64) @ b.astype(np.float64)
        assert np.all(np.abs(c64 - ref) <= 1e-13 * s)
        assert np.allclose(s, np.abs(a).astype(np.float64) @ np.abs(b).astype(np.float64), rtol=1e-13)
    ai = g.integers(-16, 17, size=(n, n)).astype(np.float32)
    bi = g.integers(-16, 17, size=(n, n)).astype(np.float32)
    exact = ai.astype(np.int64) @ bi.astype(np.int64)
    assert np.array_equal(orc.matmul_listing1_threads(ai, bi, 5), exact.astype(np.float32))
    c64, s = orc.matmul_truth_threads(ai, bi, 5)
    assert np.array_equal(c64, exact.astype(np.float64))
    assert np.array_equal(s, np.abs(ai).astype(np.int64) @ np.abs(bi).astype(np.int64))

# --------------------------------------------------------------------------
# application patterns (Sec. 4.2): Nearest Neighbor, SRAD, BFS
# --------------------------------------------------------------------------
def _np_nearest(pts, qx, qy, k):
    d = (pts[:, 0] - np.float32(qx)) * (pts[:, 0] - np.float32(qx)) + \
        (pts[:, 1] - np.float32(qy)) * (pts[:, 1] - np.float32(qy))
    order = np.lexsort((np.arange(len(d)), d))[:k]
    return order, d[order]


def pin_nearest_k(orc):
    g = np.random.default_rng(31)
    for n, k in [(1, 1), (5, 5), (7, 3), (1000, 5), (4097, 8), (3, 5), (0, 2)]:
        pts = g.random((n, 2), dtype=np.float32) * 10
        qx, qy = 3.25, 7.5
        idx, d2 = orc.nearest_k(pts, qx, qy, k)
        want_i, want_d = _np_nearest(pts, qx, qy, k)
        m = min(n, k)
        assert np.array_equal(idx[:m], want_i) and np.array_equal(d2[:m], want_d), (n, k)
        assert np.all(idx[m:] == -1) and np.all(np.isinf(d2[m:]))
    # ties: duplicate points are ordered by index
    pts = np.array([[1, 1], [0, 0], [1, 1], [2, 2], [0, 0]], dtype=np.float32)
    idx, d2 = orc.nearest_k(pts, 0.0, 0.0, 4)
    assert idx.tolist() == [1, 4, 0, 2]


def pin_standardize(orc):
    g = np.random.default_rng(37)
    x = (g.standard_normal(100001) * 3 + 5).astype(np.float32)
    y, (mean, var) = orc.standardize(x)
    xd = x.astype(np.float64)
    assert abs(mean - xd.mean()) <= 1e-12 * abs(xd.mean())
    assert abs(var - xd.var()) <= 1e-9 * xd.var()
    assert abs(float(y.astype(np.float64).mean())) < 1e-5
    assert abs(float(y.astype(np.float64).var()) - 1.0) < 1e-5
    # affine invariance (positive scale) up to float rounding
    y2, _ = orc.standardize((x * 2 + 1).astype(np.float32))
    assert np.max(np.abs(y2 - y)) < 1e-5
    c = np.full(10, 4.0, dtype=np.float32)
    yc, (mc, vc) = orc.standardize(c)
    assert mc == 4.0 and vc == 0.0 and np.all(yc == 0)


def pin_grid_bfs(orc):
    rows, cols = 13, 17
    open_all = np.ones((rows, cols), dtype=np.uint8)
    src = 5 * cols + 3
    dist, levels = orc.grid_bfs(open_all, src)
    rr, cc = np.indices((rows, cols))
    assert np.array_equal(dist, np.abs(rr - 5) + np.abs(cc - 3))          # Manhattan distance
    assert levels == int(dist.max()) + 1
    import networkx as nx
    g = np.random.default_rng(41)
    for p_open in [0.9, 0.65]:
        grid = (g.random((rows, cols)) < p_open).astype(np.uint8)
        grid.flat[src] = 1
        G = nx.grid_2d_graph(rows, cols)
        G.remove_nodes_from([(r, c) for r in range(rows) for c in range(cols) if not grid[r, c]])
        sp = nx.single_source_shortest_path_length(G, (5, 3))
        want = np.full((rows, cols), -1, dtype=np.int32)
        for (r, c), d in sp.items():
            want[r, c] = d
        dist, levels = orc.grid_bfs(grid, src)
        assert np.array_equal(dist, want)
    closed = open_all.copy()
    closed.flat[src] = 0
    dist, levels = orc.grid_bfs(closed, src)
    assert levels == 0 and np.all(dist == -1)


ALL_PINS = [v for k, v in sorted(globals().items()) if k.startswith("pin_")]
