"""accr_matmul_nest (Listing 1a) on the GPU against the serial oracle."""
import numpy as np
import pytest
import torch

import oracle
from guard import guarded
from tolerances import BF16X3_CAP, bf16x3_tol
from paper_1412_1127_gb300 import api, inputs

pytestmark = pytest.mark.gpu

SIZES = [1, 2, 7, 33, 64, 100, 128, 129, 200, 256, 257, 300, 513]
U = 2.0 ** -24


def gpu_mm(a, b, mode):
    at, bt = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    c = guarded(at.shape, torch.float32, float("nan"))
    api.accr_matmul_nest(at, bt, c.t, mode=mode, flags=api.ACCR_SYNC)
    return c.check("c (%s, len %d)" % (mode, a.shape[0])).cpu().numpy()


@pytest.mark.parametrize("n", SIZES)
def test_serial_mode_is_the_serial_program(n):
    a = inputs.uniform_matrix(n, n, salt=n)
    b = inputs.uniform_matrix(n, n, salt=n + 1)
    assert np.array_equal(gpu_mm(a, b, "serial"), oracle.matmul_listing1(a, b))


@pytest.mark.parametrize("n", SIZES)
def test_fma_mode_error_bound(n):
    a = inputs.uniform_matrix(n, n, salt=2 * n)
    b = inputs.uniform_matrix(n, n, salt=2 * n + 1)
    c = gpu_mm(a, b, "simt").astype(np.float64)
    t, s = oracle.matmul_truth(a, b)
    assert np.all(np.abs(c - t) <= (n + 2) * U * s + 1e-30)


@pytest.mark.parametrize("n", SIZES)
def test_bf16x3_error_bound(n):
    a = inputs.uniform_matrix(n, n, salt=3 * n)
    b = inputs.uniform_matrix(n, n, salt=3 * n + 1)
    c = gpu_mm(a, b, "bf16x3").astype(np.float64)
    assert not np.isnan(c).any()
    t, s = oracle.matmul_truth(a, b)
    assert np.all(np.abs(c - t) <= bf16x3_tol(a, b, s))


@pytest.mark.parametrize("n", [1, 16, 64, 130, 256])
def test_small_integers_exact_in_every_mode(n):
    a = inputs.small_int_matrix(n, n, salt=n)
    b = inputs.small_int_matrix(n, n, salt=n + 5)
    exact = (a.astype(np.int64) @ b.astype(np.int64)).astype(np.float32)
    for mode in ["serial", "simt", "bf16x3"]:
        assert np.array_equal(gpu_mm(a, b, mode), exact), mode


def test_identity():
    n = 200
    a = inputs.uniform_matrix(n, n, salt=9)
    eye = np.eye(n, dtype=np.float32)
    assert np.array_equal(gpu_mm(a, eye, "serial"), a)
    assert np.array_equal(gpu_mm(a, eye, "simt"), a)
    c = gpu_mm(a, eye, "bf16x3")
    assert np.all(np.abs(c - a) <= 2.0 ** -16 * np.abs(a))


def test_full_size_sampled():
    """LEN = 4096, U(-1,1): sampled entries against the oracle."""
    n = 4096
    a = inputs.uniform_matrix(n, n, salt=41)
    b = inputs.uniform_matrix(n, n, salt=42)
    at, bt = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    out = {}
    for mode in ["serial", "simt", "bf16x3"]:
        ct = torch.empty_like(at)
        api.accr_matmul_nest(at, bt, ct, mode=mode, flags=api.ACCR_SYNC)
        out[mode] = ct.cpu().numpy()
    g = np.random.default_rng(0)
    for i, j in zip(g.integers(0, n, 48), g.integers(0, n, 48)):
        assert out["serial"][i, j] == oracle.matmul_listing1_at(a, b, i, j)
        t, s = oracle.matmul_truth_at(a, b, i, j)
        assert abs(float(out["simt"][i, j]) - t) <= (n + 2) * U * s
        assert abs(float(out["bf16x3"][i, j]) - t) <= BF16X3_CAP * s


@pytest.mark.slow
def test_every_cta_owns_several_tiles():
    """LEN = 3072, U(-1,1), every entry of every mode against the oracle.  The
    BF16x3 kernel's 128 x 224 tiles number 24 x 14 = 336 here, so each of the
    persistent CTAs takes two or three tiles: both tensor-memory accumulators,
    their full/empty handshake and the operand ring carried across tiles all
    run.  SERIAL is bit-exact with Listing 1a, the fused SIMT form within
    (n + 2) 2^-24 sum|ab|, BF16x3 within the bound derived in
    tolerances.bf16x3_tol (below 2e-5 sum|ab| at this size)."""
    n = 3072
    a = inputs.uniform_matrix(n, n, salt=61)
    b = inputs.uniform_matrix(n, n, salt=62)
    serial = oracle.matmul_listing1_threads(a, b)
    t, s = oracle.matmul_truth_threads(a, b)
    tol = bf16x3_tol(a, b, s)
    assert float(np.max(tol / s)) <= BF16X3_CAP
    out = {m: gpu_mm(a, b, m) for m in ["serial", "simt", "bf16x3"]}
    assert np.array_equal(out["serial"], serial)
    assert np.all(np.abs(out["simt"].astype(np.float64) - t) <= (n + 2) * U * s)
    err = np.abs(out["bf16x3"].astype(np.float64) - t)
    assert np.all(err <= tol), float(np.max(err / s))
    # a repeat gives the same bits (the tile-to-CTA order does not change sums)
    assert np.array_equal(gpu_mm(a, b, "bf16x3"), out["bf16x3"])


def test_rejects_bad_arguments():
    x = torch.zeros(4, 4, device="cuda")
    with pytest.raises(api._native.AccrError):
        api.accr_matmul_nest(x, x, x, mode=7)
    assert api.lib().accr_matmul_nest(None, None, None, -1, 0, 0, None) == api._native.ACCR_EINVAL


def test_reuse_split_flag():
    n = 300
    a = inputs.uniform_matrix(n, n, salt=51)
    b = inputs.uniform_matrix(n, n, salt=52)
    at, bt = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    c1, c2 = torch.empty_like(at), torch.empty_like(at)
    api.accr_matmul_nest(at, bt, c1, mode="bf16x3", flags=api.ACCR_SYNC)
    api.accr_matmul_nest(at, bt, c2, mode="bf16x3", flags=api.ACCR_SYNC | api.ACCR_MM_REUSE_SPLIT)
    assert torch.equal(c1, c2)
    # different operands: the flag does not reuse a stale split
    b2 = inputs.uniform_matrix(n, n, salt=53)
    bt2 = torch.from_numpy(b2).cuda()
    api.accr_matmul_nest(at, bt2, c2, mode="bf16x3", flags=api.ACCR_SYNC | api.ACCR_MM_REUSE_SPLIT)
    t, s = oracle.matmul_truth(a, b2)
    assert np.all(np.abs(c2.cpu().numpy() - t) <= bf16x3_tol(a, b2, s))


def test_fma_probe():
    """The FP32 peak probe runs its chains to the fixed point 1.0 and rejects
    bad arguments on the host."""
    sink = torch.zeros(256 * 8, dtype=torch.float32, device="cuda")
    api.accr_probe_fma(8, 20000, sink)
    s = sink.cpu().numpy()
    assert np.all(np.abs(s - 1.0) < 1e-3), (s.min(), s.max())
    with pytest.raises(api._native.AccrError):
        api.accr_probe_fma(0, 10, sink)
    sink.zero_()
    api.accr_probe_fma_packed(8, 20000, sink)
    s = sink.cpu().numpy()
    assert np.all(np.abs(s - 1.0) < 1e-3), (s.min(), s.max())
    with pytest.raises(api._native.AccrError):
        api.accr_probe_fma_packed(8, 0, sink)
