"""accr_reduce_noalloc: the reduction entry point for callers that cannot call
cudaMalloc (processes whose device memory all belongs to their own pool or
arena, loops that cannot take the synchronisation cudaMalloc/cudaFree cause).
Its block partials live in a fixed array inside the library instead of
library-allocated scratch.

Checked through the C ABI against accr_reduce on the same inputs, over
calls in a row that alternate between two inputs of different lengths (so the
grid, the number of partials and their values differ from one call to the
next): the array keeps the previous call's contents, and a call that read any
of them, or found a counter left over, would give a different result.  The file name sorts last so that a run that
stops at the first failure has already run every other test; it also passes
alone in a fresh process."""
import numpy as np
import pytest
import torch

import oracle
from paper_1412_1127_gb300 import api, inputs
from paper_1412_1127_gb300._native import ACCR_EINVAL
from tolerances import TOL_F32, TOL_F32_COMP, TOL_F64, assert_sum_close

pytestmark = pytest.mark.gpu

TD = {"i32": torch.int32, "i64": torch.int64, "f32": torch.float32, "f64": torch.float64}
ND = {"i32": np.int32, "i64": np.int64, "f32": np.float32, "f64": np.float64}
TOL = {("f32", 0): TOL_F32, ("f32", 1): TOL_F32_COMP, ("f64", 0): TOL_F64}

# (element type, clauses as (op, variable type), flags)
CASES = [
    ("i32", [("add", "i64"), ("max", "i32")], 0),
    ("i32", [("bxor", "i32"), ("mul", "i32"), ("land", "i32"), ("min", "i32")], 0),
    ("i64", [("add", "i64"), ("bor", "i64")], 0),
    ("f32", [("add", "f32")], api.ACCR_COMPENSATED),
    ("f32", [("add", "f32"), ("max", "f32"), ("min", "f32")], 0),
    ("f64", [("add", "f64"), ("max", "f64")], 0),
]


def make(t, n, salt):
    if t == "i32":
        return inputs.full_range_i32(n, salt=salt)
    if t == "i64":
        return inputs.uniform_i64(n, -(1 << 40), 1 << 40, salt=salt)
    return inputs.normal(n, ND[t], salt=salt)


def run(fn, xt, clauses, flags):
    outs = [torch.full((1,), 3, dtype=TD[acc], device="cuda") for _, acc in clauses]
    fn(xt, [api.clause(op, o) for (op, _), o in zip(clauses, outs)], flags=flags)
    torch.cuda.synchronize()
    return [o.item() for o in outs]


@pytest.mark.parametrize("t,clauses,flags", CASES)
@pytest.mark.parametrize("n", [0, 5, (1 << 22) + 3])
def test_noalloc_matches_reduce(t, clauses, flags, n):
    other = 70001 if n != 70001 else 5          # a second input, another grid
    xs = [make(t, n, salt=n % 13), make(t, other, salt=7)]
    xts = [torch.from_numpy(x).cuda() for x in xs]
    wants = [run(api.accr_reduce, xt, clauses, flags) for xt in xts]
    for call in range(4):  # calls in a row share the fixed array, alternating inputs
        x, xt, want = xs[call % 2], xts[call % 2], wants[call % 2]
        got = run(api.accr_reduce_noalloc, xt, clauses, flags)
        for (op, acc), g, w in zip(clauses, got, want):
            if acc in ("i32", "i64") or op in ("max", "min") or x.size == 0:
                assert g == w, (call, op, acc, g, w)
            else:
                tol = TOL[(t if acc == t else "f64", 1 if flags else 0)]
                assert_sum_close(g, x, tol)
                assert abs(g - w) <= tol * max(abs(w), 0.1 * max(x.size, 1) ** 0.5)
        if x.size > 0 and t == "i32":
            assert got[0] == int(oracle.reduce(x, clauses[0][0], clauses[0][1]))


def test_noalloc_allocates_nothing_and_rejects_host_form():
    x = inputs.full_range_i32((1 << 20) + 1)
    xt = torch.from_numpy(x).cuda()
    s = torch.empty(1, dtype=torch.int64, device="cuda")
    y = inputs.full_range_i32(3001, salt=4)
    yt = torch.from_numpy(y).cuda()
    s2 = torch.empty(1, dtype=torch.int64, device="cuda")
    fresh = torch.cuda.Stream()
    api.accr_reduce_noalloc(xt, [api.clause("add", s)], stream=fresh)   # first call: set-up
    torch.cuda.synchronize()
    s.fill_(-12345)                     # the measured calls must write the results
    s2.fill_(-12345)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    st = torch.cuda.Stream()            # one stream: the calls must not overlap
    api.accr_reduce_noalloc(xt, [api.clause("add", s)], stream=st)
    api.accr_reduce_noalloc(yt, [api.clause("add", s2)], stream=st)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert int(s.item()) == int(oracle.reduce(x, "add", "i64"))
    assert int(s2.item()) == int(oracle.reduce(y, "add", "i64"))
    arr, keep = api._clauses([api.clause("add", s)])
    rc = api.lib().accr_reduce_noalloc(xt.data_ptr(), xt.numel(), api.ACCR_I32, arr, 1,
                                       api.ACCR_TWO_LEVEL_HOST, None)
    assert rc == ACCR_EINVAL and "two-level" in api.accr_last_error()
