"""Batched regions (accr_batch_reduce, accr_segmented_reduce, prepared
batches) on the GPU against the serial oracle, and the same bits for a region
alone and inside a batch."""
import math

import numpy as np
import pytest
import torch

import oracle
from guard import guarded
from paper_1412_1127_gb300 import api, inputs
from tolerances import TOL_F32, TOL_F32_COMP, TOL_F64, same_bits

pytestmark = pytest.mark.gpu

TD = {"i32": torch.int32, "i64": torch.int64, "f32": torch.float32, "f64": torch.float64}
ND = {"i32": np.int32, "i64": np.int64, "f32": np.float32, "f64": np.float64}
INT_OPS = ["add", "mul", "max", "min", "band", "bor", "bxor", "land", "lor"]


def seg_lengths(t):
    """Lengths around every boundary of the split: empty, tiny, the warp/tile
    threshold, tile multiples and ragged multi-tile regions."""
    eb = 4 if t in ("i32", "f32") else 8
    small = api.ACCR_SMALL_BYTES // eb
    tile = api.ACCR_TILE_BYTES // eb if hasattr(api, "ACCR_TILE_BYTES") else 131072 // eb
    L = [0, 1, 2, 3, 5, 31, 32, 33, 100, 1000, small - 1, small, small + 1, tile, tile + 1,
         2 * tile, 3 * tile + 7, 17 * tile + 5, 0, 4]
    g = np.random.default_rng(eb)
    L += list(g.integers(0, 5000, size=40)) + list(g.integers(small, 6 * tile, size=10))
    return np.array(L, dtype=np.int64)


def values_for(t, n, op, salt=0):
    if t in ("f32", "f64"):
        return inputs.normal(n, ND[t], salt=salt)
    if op == "mul":
        x = inputs.full_range_i32(n, salt=salt) | 1
    elif op == "land":
        x = inputs.full_range_i32(n, salt=salt) | 1
        if n > 10:
            x[n // 3] = 0
    elif op == "band":
        x = np.full(n, -1, dtype=np.int32)
        x[:: 9973] = ~np.int32(5)
    elif op == "lor":
        x = np.zeros(n, dtype=np.int32)
        x[:: 7919] = 3
    else:
        x = inputs.full_range_i32(n, salt=salt)
    return x.astype(ND[t]) if t == "i64" else x


@pytest.mark.parametrize("op", INT_OPS)
@pytest.mark.parametrize("t,acc", [("i32", "i32"), ("i32", "i64"), ("i64", "i64")])
def test_segmented_int_bit_exact(op, t, acc):
    L = seg_lengths(t)
    off = inputs.offsets_from_lengths(L)
    v = values_for(t, int(off[-1]), op, salt=len(op))
    vt = torch.from_numpy(v).cuda()
    out = guarded((len(L),), TD[acc], 5)
    api.accr_segmented_reduce(vt, off, [api.clause(op, out.t, init=3)])
    want = oracle.segmented_reduce(v, off, op, acc, init=3)
    assert np.array_equal(out.check("segmented %s" % op).cpu().numpy(), want)


@pytest.mark.parametrize("t,acc", [("f32", "f32"), ("f32", "f64"), ("f64", "f64")])
def test_segmented_fp(t, acc):
    L = seg_lengths(t)
    off = inputs.offsets_from_lengths(L)
    v = values_for(t, int(off[-1]), "add", salt=9)
    vt = torch.from_numpy(v).cuda()
    mx, mn, s = (guarded((len(L),), TD[acc]) for _ in range(3))
    flags = api.ACCR_COMPENSATED if (t, acc) == ("f32", "f32") else 0
    api.accr_segmented_reduce(vt, off, [api.clause("max", mx.t), api.clause("min", mn.t),
                                        api.clause("add", s.t)], flags=flags)
    assert same_bits(mx.check("max").cpu().numpy(), oracle.segmented_reduce(v, off, "max", acc))
    assert same_bits(mn.check("min").cpu().numpy(), oracle.segmented_reduce(v, off, "min", acc))
    tol = TOL_F32_COMP if flags else TOL_F64 if acc == "f64" else TOL_F32
    s_np = s.check("sum").cpu().numpy()
    for k in range(len(L)):
        seg = v[off[k]:off[k + 1]]
        truth = oracle.truth_sum(seg)
        assert abs(float(s_np[k]) - truth) <= tol * max(abs(truth), 0.1 * math.sqrt(max(seg.size, 1))), k


def _mixed_regions(seed=0):
    """A heterogeneous batch: every element type, one to four clauses."""
    g = np.random.default_rng(seed)
    specs = []
    for k in range(300):
        t = ["i32", "i64", "f32", "f64"][k % 4]
        n = int(np.exp(g.uniform(0, np.log(400000))))
        if k % 17 == 0:
            n = 0
        if t == "i32":
            cls = [("add", "i64"), ("max", "i32"), ("bxor", "i32"), ("lor", "i32")][: 1 + k % 4]
        elif t == "i64":
            cls = [("add", "i64"), ("bxor", "i64")]
        elif t == "f32":
            cls = [("add", "f32"), ("max", "f32")] if k % 3 else [("add", "f64")]
        else:
            cls = [("min", "f64"), ("add", "f64")]
        specs.append((t, n, cls, api.ACCR_COMPENSATED if (t == "f32" and k % 2) else 0))
    return specs


SLOT_GAP = 3   # untouched elements between neighbouring variables


def _run_mixed(specs, subset=None, salt=0):
    """Runs a batch whose variables are one-element views into one guarded
    array per variable type, SLOT_GAP elements apart: a store to the wrong
    slot, or past the last one, changes a sentinel."""
    data, regions, outs = [], [], []
    arrays = {a: guarded((SLOT_GAP * 4 * len(specs) + SLOT_GAP,), TD[a], 7) for a in TD}
    used = {a: 0 for a in TD}
    for k, (t, n, cls, fl) in enumerate(specs):
        x = values_for(t, n, "add", salt=salt + k)
        xt = torch.from_numpy(x).cuda()
        os_ = []
        for _, a in cls:
            used[a] += SLOT_GAP
            os_.append(arrays[a].t[used[a]:used[a] + 1])
        data.append(x)
        outs.append(os_)
        regions.append((xt, [api.clause(op, o, init=1) for (op, _), o in zip(cls, os_)], fl))
    idx = range(len(specs)) if subset is None else subset
    api.accr_batch_reduce([regions[i] for i in idx])
    torch.cuda.synchronize()
    written = {a: set() for a in TD}
    for i in idx:
        for (_, a), o in zip(specs[i][2], outs[i]):
            written[a].add((o.data_ptr() - arrays[a].t.data_ptr()) // o.element_size())
    for a, g in arrays.items():
        vals = g.check("batch variables (%s)" % a).cpu().numpy()
        others = np.array([j for j in range(vals.size) if j not in written[a]], dtype=np.int64)
        assert np.all(vals[others] == 7), "a store landed outside its variable (%s)" % a
    return data, {i: [o.cpu().numpy()[0] for o in outs[i]] for i in idx}, regions


def test_mixed_batch_against_oracle():
    specs = _mixed_regions()
    data, res, _ = _run_mixed(specs)
    for k, (t, n, cls, fl) in enumerate(specs):
        x = data[k]
        for (op, acc), got in zip(cls, res[k]):
            if op == "add" and acc in ("f32", "f64"):
                tol = TOL_F64 if acc == "f64" else (TOL_F32_COMP if fl else TOL_F32)
                truth = oracle.truth_sum(np.concatenate([np.array([1], dtype=x.dtype), x]))
                assert abs(float(got) - truth) <= tol * max(abs(truth), 0.1 * math.sqrt(max(n, 1))), (k, op)
            else:
                want = oracle.reduce(x, op, acc, init=1)
                assert same_bits(np.asarray(got), np.asarray(want)), (k, op, acc, got, want)


def test_region_alone_equals_region_in_batch():
    specs = _mixed_regions(seed=3)
    _, res_all, _ = _run_mixed(specs, salt=100)
    for k in [0, 1, 2, 3, 5, 8, 13, 21, 34, 55, 89, 144, 233]:
        _, res_one, _ = _run_mixed(specs, subset=[k], salt=100)
        for a, b in zip(res_all[k], res_one[k]):
            assert same_bits(np.asarray(a), np.asarray(b)), k


def test_prepared_batch_replays():
    specs = _mixed_regions(seed=5)[:120]
    data, res, regions = _run_mixed(specs, salt=200)
    b = api.Batch(regions)
    for rep in range(3):
        for _, cls, _ in regions:
            for c in cls:
                c.out.fill_(99)
        before = api.accr_launch_count()
        b.launch()
        torch.cuda.synchronize()
        assert api.accr_launch_count() - before == 1
        for k, (_, cls, _) in enumerate(regions):
            for c, want in zip(cls, res[k]):
                assert same_bits(c.out.cpu().numpy()[0:1], np.asarray([want])), (rep, k)
    b.destroy()


def test_tiling_changes_keep_results_correct():
    L = seg_lengths("i64")
    off = inputs.offsets_from_lengths(L)
    v = values_for("i64", int(off[-1]), "add", salt=4)
    vt = torch.from_numpy(v).cuda()
    want = oracle.segmented_reduce(v, off, "add", "i64")
    old = api.accr_batch_tiling(16, 4096)
    try:
        for small, tile in [(16, 4096), (0, 65536), (1 << 20, 1 << 20), (65536, 131072)]:
            api.accr_batch_tiling(small or 16, tile)
            out = guarded((len(L),), torch.int64)
            api.accr_segmented_reduce(vt, off, [api.clause("add", out.t)])
            assert np.array_equal(out.check("tiling %d/%d" % (small, tile)).cpu().numpy(), want), (small, tile)
    finally:
        api.accr_batch_tiling(*old)


def test_batch_rejects_bad_regions():
    x = torch.zeros(10, dtype=torch.float32, device="cuda")
    o = torch.empty(1, dtype=torch.float32, device="cuda")
    with pytest.raises(api._native.AccrError) as e:
        api.accr_batch_reduce([(x, [api.clause("band", o)], 0)])
    assert e.value.code == api._native.ACCR_ETYPE
    with pytest.raises(api._native.AccrError):
        api.accr_segmented_reduce(x, [0, 5, 3], [api.clause("add", torch.empty(2, device="cuda"))])


def test_many_regions_full_size():
    """20,000 regions, lengths log-uniform on [1, 2^20]: even ones float
    N(0,1) with compensated +, odd ones int64 with + and ^, in one launch."""
    lengths, pf, off_f, pi, off_i = inputs.batched_regions()
    tf, ti = torch.from_numpy(pf).cuda(), torch.from_numpy(pi).cuda()
    nf, ni = len(off_f) - 1, len(off_i) - 1
    gf, gi, gx = guarded((nf,), torch.float32), guarded((ni,), torch.int64), guarded((ni,), torch.int64)
    sf, si, xi = gf.t, gi.t, gx.t
    regions = []
    for k in range(len(lengths)):
        if k % 2 == 0:
            j = k // 2
            regions.append((tf[off_f[j]:off_f[j + 1]], [api.clause("add", sf[j:j + 1])], api.ACCR_COMPENSATED))
        else:
            j = k // 2
            regions.append((ti[off_i[j]:off_i[j + 1]], [api.clause("add", si[j:j + 1]),
                                                        api.clause("bxor", xi[j:j + 1])], 0))
    before = api.accr_launch_count()
    api.accr_batch_reduce(regions)
    torch.cuda.synchronize()
    assert api.accr_launch_count() - before == 1
    gf.check("float sums"), gi.check("int sums"), gx.check("xors")
    assert np.array_equal(si.cpu().numpy(), oracle.segmented_reduce(pi, off_i, "add", "i64"))
    assert np.array_equal(xi.cpu().numpy(), oracle.segmented_reduce(pi, off_i, "bxor", "i64"))
    s_np = sf.cpu().numpy()
    # every float region against its exact sum (host threads)
    import concurrent.futures as cf
    with cf.ThreadPoolExecutor(max_workers=16) as ex:
        truths = list(ex.map(lambda j: oracle.truth_sum(pf[off_f[j]:off_f[j + 1]]), range(nf)))
    for j, truth in enumerate(truths):
        n = int(off_f[j + 1] - off_f[j])
        assert abs(float(s_np[j]) - truth) <= TOL_F32_COMP * max(abs(truth), 0.1 * math.sqrt(max(n, 1))), j


def test_plain_form_matches_batched():
    specs = [s for s in _mixed_regions(seed=7) if s[0] in ("i32", "i64")][:80]
    data, res, regions = _run_mixed(specs, salt=300)
    for _, cls, _ in regions:
        for c in cls:
            c.out.fill_(-1)
    before = api.accr_launch_count()
    api.accr_batch_reduce(regions, flags=api.ACCR_PLAIN | api.ACCR_SYNC)
    assert api.accr_launch_count() - before == len(regions)
    for k, (_, cls, _) in enumerate(regions):
        for c, want in zip(cls, res[k]):
            assert c.out.cpu().numpy()[0] == want


def test_segmented_many_segments_three_clauses():
    """More than 4,096 segments (the plan is built in chunks on the planner
    threads) with three clauses (two descriptors per segment): every segment
    against the oracle."""
    g = np.random.default_rng(31)
    L = np.exp(g.uniform(0, np.log(200000), size=7000)).astype(np.int64)
    L[::97] = 0
    off = inputs.offsets_from_lengths(L)
    v = inputs.uniform_i64(int(off[-1]), -(1 << 40), 1 << 40, salt=12)
    vt = torch.from_numpy(v).cuda()
    outs = [guarded((len(L),), torch.int64, 3) for _ in range(3)]
    ops = ["add", "bxor", "max"]
    api.accr_segmented_reduce(vt, off, [api.clause(op, o.t) for op, o in zip(ops, outs)])
    for op, o in zip(ops, outs):
        assert np.array_equal(o.check(op).cpu().numpy(), oracle.segmented_reduce(v, off, op, "i64")), op


def test_concurrent_one_shot_batches_from_two_threads():
    """Two host threads plan and launch large one-shot batches at the same time
    on their own streams (plans of 4,096 regions or more share the planner
    threads): every result against the oracle, three rounds each."""
    import threading
    g = np.random.default_rng(41)
    L = np.exp(g.uniform(0, np.log(50000), size=5000)).astype(np.int64)
    off = inputs.offsets_from_lengths(L)
    v = inputs.uniform_i64(int(off[-1]), -(1 << 40), 1 << 40, salt=13)
    vt = torch.from_numpy(v).cuda()
    want = {"add": oracle.segmented_reduce(v, off, "add", "i64"), "bxor": oracle.segmented_reduce(v, off, "bxor", "i64")}
    errors = []

    def worker(op, seed):
        try:
            s = torch.cuda.Stream()
            out = torch.empty(len(L), dtype=torch.int64, device="cuda")
            regions = [(vt[off[k]:off[k + 1]], [api.clause(op, out[k:k + 1])], 0) for k in range(len(L))]
            for _ in range(3):
                out.fill_(-1)
                torch.cuda.synchronize()
                api.accr_batch_reduce(regions, flags=api.ACCR_SYNC, stream=s)
                if not np.array_equal(out.cpu().numpy(), want[op]):
                    errors.append(op)
        except Exception as e:  # reported below
            errors.append(repr(e))

    ts = [threading.Thread(target=worker, args=(op, i)) for i, op in enumerate(["add", "bxor"])]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    assert not errors, errors
