"""The CUDA path against the stored expected values in tests/golden/."""
import numpy as np
import pytest
import torch

import golden_data as G
from paper_1412_1127_gb300 import api
from tolerances import TOL_F32, TOL_F64, assert_sum_close

pytestmark = pytest.mark.gpu

TD = {"i32": torch.int32, "i64": torch.int64, "f32": torch.float32, "f64": torch.float64}


def test_reductions_match_stored_values():
    for t, x, op, acc, init, bits, val in G.reduce_cases():
        out = torch.full((1,), 3, dtype=TD[acc], device="cuda")
        api.accr_reduce(torch.from_numpy(x).cuda(), [api.clause(op, out, init)])
        got = out.cpu().numpy()[0]
        if t in ("i32", "i64") or op in ("max", "min"):
            assert G.bits_of(got, acc) == bits, (t, op, acc, init)    # exact
        elif op == "add":  # another summation order: against the exact sum
            assert_sum_close(float(got), x, TOL_F64 if acc == "f64" else TOL_F32, init)
        else:  # a product in another order: relative to the stored serial product
            rel = 1e-12 if acc == "f64" else 1e-5
            assert abs(float(got) - float(val)) <= rel * abs(float(val)), (t, op, got, val)


@pytest.mark.parametrize("mode", ["simt", "serial", "bf16x3"])
def test_listing1_matches_closed_form(mode):
    c = G.listing1()
    n = c.shape[0]
    a = torch.tensor([[i + 2 * l - 3 for l in range(n)] for i in range(n)], dtype=torch.float32, device="cuda")
    b = torch.tensor([[l * j - 2 for j in range(n)] for l in range(n)], dtype=torch.float32, device="cuda")
    out = torch.empty_like(a)
    api.accr_matmul_nest(a, b, out, mode=mode)
    assert np.array_equal(out.cpu().numpy(), c)


def test_nearest_matches_stored_values():
    pts, qx, qy, idx, d = G.nearest()
    i = torch.empty(5, dtype=torch.int64, device="cuda")
    dd = torch.empty(5, dtype=torch.float32, device="cuda")
    api.accr_nearest_k(torch.from_numpy(pts).cuda(), float(qx), float(qy), 5, i, dd, flags=api.ACCR_SYNC)
    assert np.array_equal(i.cpu().numpy(), idx)
    assert np.array_equal(dd.cpu().numpy(), d)


@pytest.mark.parametrize("mode", ["reduce", "guarded", "persistent"])
def test_bfs_matches_stored_values(mode):
    grid, src, dist, levels = G.bfs()
    out = torch.empty(grid.shape, dtype=torch.int32, device="cuda")
    assert api.accr_grid_bfs(torch.from_numpy(grid).cuda(), src, out, mode=mode) == levels
    assert np.array_equal(out.cpu().numpy(), dist)
