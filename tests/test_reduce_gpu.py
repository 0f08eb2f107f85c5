"""accr_reduce on the GPU against the serial oracle (one region, one pass)."""
import numpy as np
import pytest
import torch

import oracle
from guard import guarded
from paper_1412_1127_gb300 import api, inputs
from tolerances import (TOL_F32, TOL_F32_COMP, TOL_F64, assert_sum_close, same_bits)

pytestmark = pytest.mark.gpu

INT_OPS = ["add", "mul", "max", "min", "band", "bor", "bxor", "land", "lor"]
TD = {"i32": torch.int32, "i64": torch.int64, "f32": torch.float32, "f64": torch.float64}
ND = {"i32": np.int32, "i64": np.int64, "f32": np.float32, "f64": np.float64}
# sizes spanning several CTAs, vector tails of every length and the empty region
SIZES = [0, 1, 2, 3, 4, 5, 7, 31, 32, 33, 1000, 4095, 65536 + 7, (1 << 20) + 3]


def to_dev(x, offset=0):
    """Upload x so that the device view starts `offset` elements past a
    256-byte boundary (unaligned heads)."""
    pad = np.zeros(offset, dtype=x.dtype)
    t = torch.from_numpy(np.concatenate([pad, x])).cuda()
    return t[offset:]


def gpu_reduce(x, op, acc, init=None, flags=0, offset=0):
    xt = to_dev(x, offset)
    out = guarded((1,), TD[acc], 7)
    api.accr_reduce(xt, [api.clause(op, out.t, init)], flags=flags)
    return out.check("%s into %s" % (op, acc)).cpu().numpy()[0]


def int_input(op, n, t, salt):
    if op in ("mul", "band", "land", "lor") and n > 0:
        x = inputs.adversarial_i32(n, op, salt=salt)
    else:
        x = inputs.full_range_i32(n, salt=salt)
    if t == "i64":
        hi = inputs.full_range_i32(n, salt=salt + 99).astype(np.int64) << 32
        x = x.astype(np.int64)
        if op not in ("mul", "band", "land", "lor"):
            x = x ^ hi
        elif op == "mul":
            x = x * 3 + 2 * (x & 1)  # still odd: wrap keeps the product odd
    return x


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("op", INT_OPS)
@pytest.mark.parametrize("t,acc", [("i32", "i32"), ("i32", "i64"), ("i64", "i64")])
def test_int_ops_bit_exact(n, op, t, acc):
    x = int_input(op, n, t, salt=n % 97)
    for off in ([0, 1, 3] if n in (5, 4095, 65543) else [0]):
        got = gpu_reduce(x, op, acc, offset=off)
        want = oracle.reduce(x, op, acc)
        assert got == want, (op, t, acc, n, off, got, want)


@pytest.mark.parametrize("op", INT_OPS)
def test_int_ops_with_prior_value(op):
    x = int_input(op, 100003, "i32", salt=5)
    for init in [0, 1, -1, 5, 2 ** 31 - 1, -(2 ** 31)]:
        assert gpu_reduce(x, op, "i32", init=init) == oracle.reduce(x, op, "i32", init=init)
        assert gpu_reduce(x, op, "i64", init=init * 3) == oracle.reduce(x, op, "i64", init=init * 3)
    e = np.zeros(0, dtype=np.int32)
    assert gpu_reduce(e, op, "i32", init=5) == 5          # n = 0 leaves the variable


def test_logical_ops_planted():
    n = (1 << 20) + 17
    for pos in [0, 1, 4, 12345, n - 1]:
        x = np.full(n, 3, dtype=np.int32)
        x[pos] = 0
        assert gpu_reduce(x, "land", "i32") == 0
        z = np.zeros(n, dtype=np.int32)
        z[pos] = -8
        assert gpu_reduce(z, "lor", "i32") == 1
        z64 = np.zeros(n, dtype=np.int64)
        z64[pos] = 1 << 40
        assert gpu_reduce(z64, "lor", "i64") == 1


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("t,acc", [("f32", "f32"), ("f32", "f64"), ("f64", "f64")])
def test_fp_minmax_bit_exact(n, t, acc):
    x = inputs.normal(n, ND[t], salt=n % 89)
    for op in ["max", "min"]:
        for off in ([0, 1] if n in (5, 4095) else [0]):
            got = gpu_reduce(x, op, acc, offset=off)
            want = oracle.reduce(x, op, acc)
            assert same_bits(np.asarray(got), np.asarray(want)), (op, n, got, want)


def test_fp_minmax_signed_zero_and_init():
    for dt, acc in [(np.float32, "f32"), (np.float64, "f64")]:
        z = np.array([-0.0] * 37 + [0.0] + [-0.0] * 50, dtype=dt)
        assert not np.signbit(gpu_reduce(z, "max", acc))
        mixed = np.array([0.0, 0.0, -0.0, 0.0] * 9, dtype=dt)
        assert np.signbit(gpu_reduce(mixed, "min", acc))
        assert not np.signbit(gpu_reduce(-mixed, "max", acc))
        x = inputs.normal(5000, dt)
        assert gpu_reduce(x, "max", acc, init=100.0) == 100.0
        assert gpu_reduce(x, "min", acc, init=-100.0) == -100.0


@pytest.mark.parametrize("n", [1, 3, 33, 4095, 65543, (1 << 20) + 3, 1 << 22])
def test_fp_sums_within_tolerance(n):
    x32 = inputs.normal(n, np.float32, salt=3)
    x64 = inputs.normal(n, np.float64, salt=4)
    assert_sum_close(gpu_reduce(x32, "add", "f32"), x32, TOL_F32)
    assert_sum_close(gpu_reduce(x32, "add", "f32", flags=api.ACCR_COMPENSATED), x32, TOL_F32_COMP)
    assert_sum_close(gpu_reduce(x32, "add", "f64"), x32, TOL_F64)
    assert_sum_close(gpu_reduce(x64, "add", "f64"), x64, TOL_F64)
    assert_sum_close(gpu_reduce(x32, "add", "f32", init=2.5), x32, TOL_F32, init=2.5)
    assert_sum_close(gpu_reduce(x64, "add", "f64", offset=1), x64, TOL_F64)


def test_fp_sum_constant_ones_exact():
    # 2^25 ones: a float accumulator running serially stalls at 2^24, a tree
    # of small partials and the compensated sum are exact
    n = 1 << 25
    x = np.ones(n, dtype=np.float32)
    assert oracle.reduce(x[: (1 << 24) + 8], "add", "f32") == 2.0 ** 24
    assert gpu_reduce(x, "add", "f32") == float(n)
    assert gpu_reduce(x, "add", "f32", flags=api.ACCR_COMPENSATED) == float(n)


def test_fp_products():
    g = np.random.default_rng(3)
    for n in [1, 7, 4099]:
        x = (1.0 + (g.random(n) - 0.5) * 1e-3).astype(np.float32)
        ref = float(oracle.reduce(x, "mul", "f64"))  # double product: reference
        got = float(gpu_reduce(x, "mul", "f32"))
        assert abs(got - ref) <= 2 * n * 2.0 ** -24 * abs(ref)
        assert abs(float(gpu_reduce(x, "mul", "f64")) - ref) <= 2 * n * 2.0 ** -53 * abs(ref)


def test_empty_fp_regions_keep_prior_value():
    for t in ["f32", "f64"]:
        e = np.zeros(0, dtype=ND[t])
        assert same_bits(np.asarray(gpu_reduce(e, "add", t, init=-0.0)), np.asarray(ND[t](-0.0)))
        assert gpu_reduce(e, "add", t) == 0.0
        assert gpu_reduce(e, "max", t) == -np.inf
        assert gpu_reduce(e, "mul", t) == 1.0


def test_two_clauses_one_pass_sum_and_max():
    # reduction(+:s) reduction(max:m) over 2^20 int32 in [-1000, 1000]
    x = inputs.scalar_i32_small()
    xt = torch.from_numpy(x).cuda()
    s = torch.empty(1, dtype=torch.int64, device="cuda")
    m = torch.empty(1, dtype=torch.int32, device="cuda")
    before = api.accr_launch_count()
    api.accr_reduce(xt, [api.clause("add", s), api.clause("max", m)])
    assert api.accr_launch_count() - before == 1
    assert int(s.item()) == int(oracle.reduce(x, "add", "i64"))
    assert int(m.item()) == int(oracle.reduce(x, "max", "i32"))


def test_four_clauses_mixed():
    x = inputs.full_range_i32((1 << 18) + 5, salt=8)
    xt = torch.from_numpy(x).cuda()
    outs = [torch.empty(1, dtype=torch.int64, device="cuda"),
            torch.empty(1, dtype=torch.int32, device="cuda"),
            torch.empty(1, dtype=torch.int32, device="cuda"),
            torch.empty(1, dtype=torch.int64, device="cuda")]
    ops = ["add", "bxor", "min", "max"]
    api.accr_reduce(xt, [api.clause(o, t, init=3) for o, t in zip(ops, outs)])
    for o, t in zip(ops, outs):
        acc = "i64" if t.dtype == torch.int64 else "i32"
        assert int(t.item()) == int(oracle.reduce(x, o, acc, init=3)), o
    f = inputs.normal((1 << 18) + 1, np.float32)
    ft = torch.from_numpy(f).cuda()
    fo = [torch.empty(1, dtype=torch.float32, device="cuda") for _ in range(3)]
    api.accr_reduce(ft, [api.clause("add", fo[0]), api.clause("max", fo[1]),
                         api.clause("min", fo[2])], flags=api.ACCR_COMPENSATED)
    assert_sum_close(fo[0].item(), f, TOL_F32_COMP)
    assert fo[1].item() == float(oracle.reduce(f, "max"))
    assert fo[2].item() == float(oracle.reduce(f, "min"))


def test_deterministic_repeats():
    x = inputs.normal((1 << 22) + 3, np.float32)
    r = [gpu_reduce(x, "add", "f32") for _ in range(3)]
    assert same_bits(np.asarray(r[0]), np.asarray(r[1])) and same_bits(np.asarray(r[0]), np.asarray(r[2]))


def test_streams_overlap_use_separate_scratch():
    xs = [inputs.full_range_i32((1 << 22) + i, salt=i) for i in range(4)]
    ts = [torch.from_numpy(x).cuda() for x in xs]
    outs = [torch.empty(1, dtype=torch.int64, device="cuda") for _ in xs]
    streams = [torch.cuda.Stream() for _ in xs]
    torch.cuda.synchronize()
    for _ in range(3):
        for t, o, s in zip(ts, outs, streams):
            api.accr_reduce(t, [api.clause("add", o)], stream=s)
    torch.cuda.synchronize()
    for x, o in zip(xs, outs):
        assert int(o.item()) == int(oracle.reduce(x, "add", "i64"))


def test_two_level_host_form_matches():
    x = inputs.full_range_i32((1 << 21) + 9, salt=2)
    xt = torch.from_numpy(x).cuda()
    for op, acc in [("add", "i64"), ("bxor", "i32"), ("max", "i32"), ("land", "i32")]:
        out = torch.zeros(1, dtype=TD[acc])      # host variable
        api.accr_reduce(xt, [api.clause(op, out)], flags=api.ACCR_TWO_LEVEL_HOST)
        assert out.item() == oracle.reduce(x, op, acc), op
    f = inputs.normal((1 << 21) + 1, np.float32)
    out = torch.zeros(1, dtype=torch.float32)
    api.accr_reduce(torch.from_numpy(f).cuda(), [api.clause("add", out)],
                    flags=api.ACCR_TWO_LEVEL_HOST | api.ACCR_COMPENSATED)
    assert_sum_close(out.item(), f, TOL_F32_COMP)


def test_errors_are_reported_not_fatal():
    x = torch.zeros(8, dtype=torch.float32, device="cuda")
    o = torch.empty(1, dtype=torch.float32, device="cuda")
    with pytest.raises(api._native.AccrError) as e:
        api.accr_reduce(x, [api.clause("bxor", o)])
    assert e.value.code == api._native.ACCR_ETYPE
    api.accr_reduce(x, [api.clause("add", o)], flags=api.ACCR_SYNC)  # context still fine
    assert o.item() == 0.0


def test_variable_in_pinned_host_memory():
    x = inputs.full_range_i32((1 << 22) + 5, salt=12)
    xt = torch.from_numpy(x).cuda()
    s = torch.zeros(1, dtype=torch.int64).pin_memory()
    m = torch.zeros(1, dtype=torch.int32).pin_memory()
    api.accr_reduce(xt, [api.clause("add", s), api.clause("max", m)], flags=api.ACCR_SYNC)
    assert int(s.item()) == int(oracle.reduce(x, "add", "i64"))
    assert int(m.item()) == int(oracle.reduce(x, "max", "i32"))


def test_f64_sum_wide_dynamic_range():
    g = np.random.default_rng(77)
    for n in [8, 9, 17, 4096, (1 << 20) + 3]:
        x = np.ldexp(g.standard_normal(n), g.integers(-300, 300, size=n))
        x[:: 97] = 0.0
        got = gpu_reduce(x, "add", "f64")
        truth = oracle.truth_sum(x)
        assert abs(float(got) - truth) <= 1e-14 * oracle.truth_abs_sum(x), n
        tiny = np.ldexp(g.standard_normal(n), -1040)          # subnormal range
        assert abs(float(gpu_reduce(tiny, "add", "f64")) - oracle.truth_sum(tiny)) <= \
            1e-14 * oracle.truth_abs_sum(tiny) + 5e-324 * n


@pytest.mark.slow
def test_full_size_all_operators():
    """The all-operator workload at n = 2^28, the inputs bench.py times."""
    n = 1 << 28
    xi = inputs.full_range_i32(n, salt=0)
    xf = inputs.normal(n, np.float32, salt=1000)
    xd = inputs.normal(n, np.float64, salt=2000)
    ti = torch.from_numpy(xi).cuda()
    for op, acc in [("add", "i64"), ("mul", "i32"), ("max", "i32"), ("min", "i32"), ("band", "i32"),
                    ("bor", "i32"), ("bxor", "i32"), ("land", "i32"), ("lor", "i32")]:
        out = torch.empty(1, dtype=TD[acc], device="cuda")
        api.accr_reduce(ti, [api.clause(op, out)])
        assert out.item() == oracle.reduce(xi, op, acc), op
    # the adversarial variants keep *, &, && and || informative at full size
    for op in ["mul", "band", "land", "lor", "max", "min"]:
        xa = inputs.adversarial_i32(n, op)
        out = torch.empty(1, dtype=torch.int32, device="cuda")
        api.accr_reduce(torch.from_numpy(xa).cuda(), [api.clause(op, out)])
        assert out.item() == oracle.reduce(xa, op, "i32"), op
    del ti
    tf = torch.from_numpy(xf).cuda()
    for op in ["max", "min"]:
        out = torch.empty(1, dtype=torch.float32, device="cuda")
        api.accr_reduce(tf, [api.clause(op, out)])
        assert out.item() == float(oracle.reduce(xf, op)), op
    for flags, tol in [(0, TOL_F32), (api.ACCR_COMPENSATED, TOL_F32_COMP)]:
        out = torch.empty(1, dtype=torch.float32, device="cuda")
        api.accr_reduce(tf, [api.clause("add", out)], flags=flags)
        assert_sum_close(out.item(), xf, tol)
    del tf
    td = torch.from_numpy(xd).cuda()
    for op in ["max", "min"]:
        out = torch.empty(1, dtype=torch.float64, device="cuda")
        api.accr_reduce(td, [api.clause(op, out)])
        assert out.item() == float(oracle.reduce(xd, op)), op
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    api.accr_reduce(td, [api.clause("add", out)])
    assert_sum_close(out.item(), xd, TOL_F64)


REDUCE_PAIRS = [  # (element type, sum variable, flags) of the fixed-code two-clause kernels
    ("i32", "i32", 0), ("i32", "i64", 0), ("i64", "i64", 0), ("f32", "f32", 0),
    ("f32", "f32", api.ACCR_COMPENSATED), ("f32", "f64", 0), ("f64", "f64", 0)]


@pytest.mark.parametrize("t,acc,flags", REDUCE_PAIRS)
@pytest.mark.parametrize("ext", ["max", "min"])
@pytest.mark.parametrize("sum_first", [True, False])
@pytest.mark.parametrize("n", [0, 1, 33, 65536 + 7, (1 << 20) + 3])
@pytest.mark.parametrize("two_level", [False, True])
def test_sum_and_extreme_pairs(t, acc, flags, ext, sum_first, n, two_level):
    """reduction(+:s) reduction(max|min:m) in one pass, in either clause order,
    through the fixed-code kernels (and the generic one in the two-level
    form): each variable gets its own fold (integers and extremes bit-exact,
    float sums within the sum tolerance)."""
    if t in ("i32", "i64"):
        x = int_input("add", n, t, salt=n % 89)
    else:
        x = inputs.normal(n, ND[t], salt=n % 89)
    xt = to_dev(x)
    where = "cpu" if two_level else "cuda"  # the two-level form merges into host variables
    s = torch.full((1,), 7, dtype=TD[acc], device=where)
    m = torch.full((1,), 7, dtype=TD[t], device=where)
    cls = [api.clause("add", s, 3 if t in ("i32", "i64") else None), api.clause(ext, m)]
    fl = flags | (api.ACCR_TWO_LEVEL_HOST if two_level else 0)
    api.accr_reduce(xt, cls if sum_first else cls[::-1], flags=fl)
    got_s, got_m = s.cpu().numpy()[0], m.cpu().numpy()[0]
    want_m = oracle.reduce(x, ext, t)
    if t in ("i32", "i64"):
        assert got_m == want_m
        assert got_s == oracle.reduce(x, "add", acc, init=3)
        return
    assert same_bits(np.array([got_m]), np.array([want_m]))
    tol = TOL_F32_COMP if flags else (TOL_F64 if acc == "f64" else TOL_F32)
    assert_sum_close(float(got_s), x, tol)


@pytest.mark.slow
def test_region_beyond_2_31_elements():
    """One region of 2^31 + 77 int32 (8.6 GB): 64-bit index arithmetic all the
    way to the last element (the extremes are planted past 2^31)."""
    n = (1 << 31) + 77
    x = inputs.full_range_i32(n, salt=31)
    x[n - 1] = np.int32(2 ** 31 - 1)
    x[(1 << 31) + 5] = np.int32(-(2 ** 31))
    xt = torch.from_numpy(x).cuda()
    s = torch.empty(1, dtype=torch.int64, device="cuda")
    m = torch.empty(1, dtype=torch.int32, device="cuda")
    lo = torch.empty(1, dtype=torch.int32, device="cuda")
    xo = torch.empty(1, dtype=torch.int32, device="cuda")
    api.accr_reduce(xt, [api.clause("add", s), api.clause("max", m)])   # fixed-code pair
    api.accr_reduce(xt, [api.clause("min", lo), api.clause("bxor", xo)])  # generic pair
    assert s.item() == oracle.reduce(x, "add", "i64")
    assert m.item() == 2 ** 31 - 1 and lo.item() == -(2 ** 31)
    assert xo.item() == oracle.reduce(x, "bxor", "i32")
