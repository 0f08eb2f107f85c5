"""Application patterns of the paper (Sec. 4.2) on the GPU against the oracle:
Nearest Neighbor (k smallest distances), SRAD (a reduction feeding an
elementwise region), BFS (a convergence loop with an || flag)."""
import numpy as np
import pytest
import torch

import oracle
from guard import guarded
from paper_1412_1127_gb300 import api, inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [0, 1, 2, 3, 7, 100, 1001, 65537, (1 << 20) + 3])
@pytest.mark.parametrize("k", [1, 5, 8, 16])
def test_nearest_k_exact(n, k):
    g = inputs.rng(21, n)
    pts = (g.random((n, 2), dtype=np.float32) * 100).astype(np.float32)
    if n > 10:
        pts[n // 2] = pts[n // 3]          # an exact tie, broken by index
    qx, qy = 41.5, 58.25
    for off in ([0, 1] if n in (7, 1001) else [0]):
        big = np.zeros((n + off, 2), dtype=np.float32)
        big[off:] = pts
        pt = torch.from_numpy(big).cuda()[off:]
        gi, gd = guarded((k,), torch.int64, -7), guarded((k,), torch.float32, -7)
        api.accr_nearest_k(pt, qx, qy, k, gi.t, gd.t, flags=api.ACCR_SYNC)
        wi, wd = oracle.nearest_k(pts, qx, qy, k)
        assert np.array_equal(gi.check("idx").cpu().numpy(), wi), (n, k, off)
        assert np.array_equal(gd.check("d2").cpu().numpy(), wd), (n, k, off)


@pytest.mark.parametrize("order", ["random", "far_first", "near_first", "all_equal"])
@pytest.mark.parametrize("k", [1, 8, 16])
def test_nearest_k_sampled_bound(order, k):
    """Inputs large enough for the sampled distance bound: exact whatever the
    order of the points (a sample of far points gives a loose bound, one of
    near points a tight one, equal points put every point on the bound)."""
    n = (1 << 22) + 5
    g = inputs.rng(22, k)
    pts = (g.random((n, 2), dtype=np.float32) * 100).astype(np.float32)
    qx, qy = 50.0, 50.0
    if order == "all_equal":
        pts[:] = np.float32(12.5)
    elif order != "random":
        d = (pts[:, 0] - qx) ** 2 + (pts[:, 1] - qy) ** 2
        pts = pts[np.argsort(-d if order == "far_first" else d, kind="stable")].copy()
    pts[n - 1] = pts[n // 2]                  # an exact tie, broken by index
    for off in [0, 1]:
        big = np.zeros((n + off, 2), dtype=np.float32)
        big[off:] = pts
        pt = torch.from_numpy(big).cuda()[off:]
        gi, gd = guarded((k,), torch.int64, -7), guarded((k,), torch.float32, -7)
        api.accr_nearest_k(pt, qx, qy, k, gi.t, gd.t, flags=api.ACCR_SYNC)
        wi, wd = oracle.nearest_k(pts, qx, qy, k)
        assert np.array_equal(gi.check("idx").cpu().numpy(), wi), (order, k, off)
        assert np.array_equal(gd.check("d2").cpu().numpy(), wd), (order, k, off)


def test_nearest_k_rejects_bad_k():
    pts = torch.zeros((4, 2), device="cuda")
    i = torch.empty(32, dtype=torch.int64, device="cuda")
    d = torch.empty(32, device="cuda")
    with pytest.raises(api._native.AccrError):
        api.accr_nearest_k(pts, 0, 0, 17, i, d)


@pytest.mark.parametrize("n", [1, 5, 1000, 4 * 1024 * 1024 + 3, 1 << 26])
@pytest.mark.parametrize("form", ["fused", "unfused", "host"])
def test_standardize(n, form):
    x = (inputs.normal(n, np.float32, salt=n % 7) * 3 + 5).astype(np.float32)
    xt = torch.from_numpy(x).cuda()
    gy, gst = guarded((n,), torch.float32, float("nan")), guarded((2,), torch.float64, float("nan"))
    y, st = gy.t, gst.t
    flags = {"fused": 0, "unfused": api.ACCR_UNFUSED, "host": api.ACCR_TWO_LEVEL_HOST}[form] | api.ACCR_SYNC
    api.accr_standardize(xt, y, st, flags=flags)
    gy.check("y"), gst.check("stats")
    wy, (wm, wv) = oracle.standardize(x)
    mean, var = st.cpu().numpy()
    assert abs(mean - wm) <= 1e-9 * max(abs(wm), 1.0)
    assert abs(var - wv) <= 1e-9 * max(abs(wv), 1e-30) or n == 1
    got = y.cpu().numpy()
    # (x - mean_f) * rstd_f: the float statistics may differ in their last bit
    assert np.max(np.abs(got - wy) / np.maximum(np.abs(wy), 1.0)) <= 4e-6


def test_standardize_in_place_and_repeat():
    x = inputs.normal(1 << 20, np.float32, salt=3)
    xt = torch.from_numpy(x.copy()).cuda()
    st = torch.empty(2, dtype=torch.float64, device="cuda")
    api.accr_standardize(xt, xt, st, flags=api.ACCR_SYNC)       # y aliases x
    wy, _ = oracle.standardize(x)
    assert np.max(np.abs(xt.cpu().numpy() - wy)) <= 4e-6 * max(1.0, float(np.abs(wy).max()))
    for _ in range(3):                                            # the grid wait re-arms
        y = torch.empty_like(xt)
        api.accr_standardize(torch.from_numpy(x).cuda(), y, st, flags=api.ACCR_SYNC)


def grid_case(rows, cols, p_open, seed):
    g = inputs.rng(23, seed)
    grid = (g.random((rows, cols)) < p_open).astype(np.uint8)
    src = int(g.integers(0, rows * cols))
    grid.flat[src] = 1
    return grid, src


@pytest.mark.parametrize("mode", ["reduce", "guarded", "persistent"])
@pytest.mark.parametrize("shape,p", [((1, 1), 1.0), ((1, 50), 1.0), ((13, 17), 0.7), ((64, 64), 0.6),
                                     ((300, 200), 0.65), ((1024, 1024), 0.62)])
def test_grid_bfs_exact(mode, shape, p):
    grid, src = grid_case(*shape, p, seed=shape[0] * 31 + shape[1])
    want, wl = oracle.grid_bfs(grid, src)
    gt = torch.from_numpy(grid).cuda()
    dist = guarded(shape, torch.int32, 12345)
    levels = api.accr_grid_bfs(gt, src, dist.t, mode=mode)
    assert np.array_equal(dist.check("dist").cpu().numpy(), want)
    assert levels == wl


def test_grid_bfs_closed_source():
    grid = np.ones((8, 8), dtype=np.uint8)
    grid.flat[9] = 0
    gt = torch.from_numpy(grid).cuda()
    dist = torch.empty((8, 8), dtype=torch.int32, device="cuda")
    for mode in ["reduce", "guarded", "persistent"]:
        assert api.accr_grid_bfs(gt, 9, dist, mode=mode) == 0
        assert bool((dist == -1).all())


def test_grid_bfs_serpentine_many_levels():
    """A one-cell-wide winding corridor: thousands of levels, each adding one
    cell, so every level's flag slot is reused many times; repeated calls
    re-arm the grid barrier."""
    rows, cols = 41, 96
    grid = np.zeros((rows, cols), dtype=np.uint8)
    grid[0::2, :] = 1                      # open corridors on even rows
    for r in range(1, rows, 2):            # one opening per wall row, alternating ends
        grid[r, cols - 1 if (r // 2) % 2 == 0 else 0] = 1
    src = 0
    want, wl = oracle.grid_bfs(grid, src)
    assert wl > 2000
    gt = torch.from_numpy(grid).cuda()
    for mode in ["persistent", "persistent", "guarded", "persistent"]:
        dist = guarded((rows, cols), torch.int32, 12345)
        assert api.accr_grid_bfs(gt, src, dist.t, mode=mode) == wl
        assert np.array_equal(dist.check("dist").cpu().numpy(), want)


@pytest.mark.slow
def test_nearest_k_full_size():
    """k = 5 nearest of the 2^26 points bench.py times (same generator)."""
    n = 1 << 26
    pts = (inputs.rng(21, 5).random((n, 2), dtype=np.float32) * 100).astype(np.float32)
    pt = torch.from_numpy(pts).cuda()
    gi, gd = guarded((5,), torch.int64, -7), guarded((5,), torch.float32, -7)
    api.accr_nearest_k(pt, 41.5, 58.25, 5, gi.t, gd.t, flags=api.ACCR_SYNC)
    wi, wd = oracle.nearest_k(pts, 41.5, 58.25, 5)
    assert np.array_equal(gi.check("idx").cpu().numpy(), wi)
    assert np.array_equal(gd.check("d2").cpu().numpy(), wd)


@pytest.mark.parametrize("k", [5, 8])
def test_nearest_k_fewer_real_points_than_k(k):
    """All but three points have NaN coordinates (a NaN distance never enters
    a list, in the oracle as here): the three real points come first and the
    rest of the k are empty (-1, inf), with every CTA list but three holding
    placeholders only."""
    n = (1 << 22) + 5
    pts = np.full((n, 2), np.nan, dtype=np.float32)
    for i, v in [(17, 1.0), (n // 2, 3.0), (n - 1, 2.0)]:
        pts[i] = (v, v)
    pt = torch.from_numpy(pts).cuda()
    gi, gd = guarded((k,), torch.int64, -7), guarded((k,), torch.float32, -7)
    api.accr_nearest_k(pt, 0.0, 0.0, k, gi.t, gd.t, flags=api.ACCR_SYNC)
    wi, wd = oracle.nearest_k(pts, 0.0, 0.0, k)
    assert list(wi[:3]) == [17, n - 1, n // 2] and all(wi[3:] == -1)
    assert np.array_equal(gi.check("idx").cpu().numpy(), wi)
    assert np.array_equal(gd.check("d2").cpu().numpy(), wd)
