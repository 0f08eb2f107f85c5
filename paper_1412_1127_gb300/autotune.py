"""Autotuner of the streaming kernels: the batched-region split (warp-region
threshold, tile size) and the vector widths (16-byte vectors in flight per
thread) of the batched-region, single-region and row kernels.

`tune(regions)` times every candidate (small_bytes, tile_bytes) pair on a
representative batch with CUDA events and returns the fastest; `apply()`
installs a pair process-wide through ``accr_batch_tiling``.  The split is a
function of each region's own type and length under a fixed pair, so once a
pair is chosen every region keeps giving the same bits alone and in any batch;
changing the pair changes the evaluation order of float sums.

`tune_widths(kind)` builds a kernel with each candidate vector width (they
are compile-time constants of the unrolled loops) -- the batched-region
kernel (tile and warp-region widths), the single-region kernel, the row
kernel -- times each build in a process of its own on that kernel's
workloads, and returns the fastest by the geometric mean; `save_widths()`
records it, and the build compiles the recorded widths in.  Changing a width
also changes the evaluation order of float sums.

The chosen values for GB300 are stored in ``tuning.json`` next to this file:
``load()`` applies the split, ``build.py`` reads the widths.

    python -m paper_1412_1127_gb300.autotune [--batch] [--reduce] [--rows] [--all] [--save]
"""
import json
import math
import os
import subprocess
import sys

import torch

from . import api

HERE = os.path.dirname(os.path.abspath(__file__))
TABLE = os.path.join(HERE, "tuning.json")

SMALL_CANDIDATES = [4096, 16384, 32768, 65536, 131072]
TILE_CANDIDATES = [262144, 524288, 1048576, 2097152, 4194304]


def time_batch(regions, small, tile, reps=5, stream=None):
    """Milliseconds per launch of a prepared batch under the given split."""
    old = api.accr_batch_tiling(small, tile)
    try:
        b = api.Batch(regions)
        s = stream or torch.cuda.current_stream()
        for _ in range(2):
            b.launch(s)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(reps):
            b.launch(s)
        e1.record(s)
        torch.cuda.synchronize()
        b.destroy()
        return e0.elapsed_time(e1) / reps
    finally:
        api.accr_batch_tiling(*old)


def tune(regions, smalls=SMALL_CANDIDATES, tiles=TILE_CANDIDATES, reps=5):
    """Times every candidate pair; returns (best_pair, {pair: ms})."""
    res = {}
    for s in smalls:
        for t in tiles:
            res[(s, t)] = time_batch(regions, s, t, reps)
    best = min(res, key=res.get)
    return best, res


def apply(small_bytes, tile_bytes):
    return api.accr_batch_tiling(int(small_bytes), int(tile_bytes))


def load(path=TABLE):
    """Install the stored split if the table exists; returns it (or None)."""
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    apply(d["small_bytes"], d["tile_bytes"])
    return d


def save(small_bytes, tile_bytes, timings, path=TABLE, note=""):
    """Records the chosen split and its timings; other entries of the table
    (the vector widths) are kept."""
    d = {}
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
    d.update({"small_bytes": int(small_bytes), "tile_bytes": int(tile_bytes), "note": note,
              "timings_ms": {"%d,%d" % k: round(v, 4) for k, v in sorted(timings.items())}})
    with open(path, "w") as f:
        json.dump(d, f, indent=1)
    return d


# Vector-width candidates per kernel: (source file, its macros, candidates).
# batch: (tile vectors per thread, warp-region vectors per lane, CTAs per SM
# the registers are budgeted for); reduce: vectors per thread; rows: vectors
# per lane.
WIDTHS = {
    "batch": ("batch.cu", ("ACCR_BATCH_BU", "ACCR_BATCH_SU", "ACCR_BATCH_MINB"),
              [(4, 8, 4), (4, 4, 4), (8, 8, 4), (2, 8, 4), (4, 16, 3), (8, 16, 3)]),
    "reduce": ("reduce.cu", ("ACCR_REDUCE_RU",), [(2,), (4,), (8,)]),
    "rows": ("rowreduce.cu", ("ACCR_ROW_RU",), [(4,), (8,), (16,)]),
}
VECTOR_CANDIDATES = WIDTHS["batch"][2]
VECTOR_MIXES = (1 << 17, 1 << 20)


def _workload(dev, hi, count=20000):
    """The many-regions workload (lengths log-uniform on [1, hi]) on the device."""
    from . import inputs
    lengths, pf, off_f, pi, off_i = inputs.batched_regions(count, hi=hi)
    tf, ti = torch.from_numpy(pf).to(dev), torch.from_numpy(pi).to(dev)
    sf = torch.empty(len(off_f) - 1, dtype=torch.float32, device=dev)
    si = torch.empty(len(off_i) - 1, dtype=torch.int64, device=dev)
    xi = torch.empty(len(off_i) - 1, dtype=torch.int64, device=dev)
    regions = []
    for k in range(len(lengths)):
        j = k // 2
        if k % 2 == 0:
            regions.append((tf[off_f[j]:off_f[j + 1]], [api.clause("add", sf[j:j + 1])], api.ACCR_COMPENSATED))
        else:
            regions.append((ti[off_i[j]:off_i[j + 1]], [api.clause("add", si[j:j + 1]),
                                                        api.clause("bxor", xi[j:j + 1])], 0))
    return regions, (tf, ti, sf, si, xi)


def _events_ms(fn, reps):
    s = torch.cuda.current_stream()
    for _ in range(3):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(reps):
        fn()
    e1.record(s)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def _time_this_library(kind, reps):
    """{workload: ms} of the kernel `kind` in the library this process loaded
    (the candidate's): batch -- a prepared batch of each length mix with the
    table's split; reduce -- one region of 2^27 int32 (+ into int64), float
    (compensated +) and double (+); rows -- row sum + row max of 65536 x 4096
    and 64 x 2^22 floats."""
    from . import inputs
    load()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    out = {}
    if kind == "batch":
        for hi in VECTOR_MIXES:
            regions, keep = _workload(dev, hi)
            d = load() or {"small_bytes": api.ACCR_SMALL_BYTES, "tile_bytes": api.ACCR_TILE_BYTES}
            out[str(hi)] = min(time_batch(regions, d["small_bytes"], d["tile_bytes"], reps) for _ in range(2))
            del regions, keep
            torch.cuda.empty_cache()
    elif kind == "reduce":
        n = 1 << 27
        cases = [("i32", torch.from_numpy(inputs.full_range_i32(n)).to(dev), torch.int64, 0),
                 ("f32", torch.from_numpy(inputs.normal(n)).to(dev), torch.float32, api.ACCR_COMPENSATED),
                 ("f64", torch.from_numpy(inputs.normal(n, dtype="float64")).to(dev), torch.float64, 0)]
        for name, x, acc, fl in cases:
            o = torch.empty(1, dtype=acc, device=dev)
            cl = [api.clause("add", o)]
            out[name] = _events_ms(lambda: api.accr_reduce(x, cl, flags=fl), reps)
    else:
        for rows, cols in [(65536, 4096), (64, 1 << 22)]:
            A = torch.from_numpy(inputs.uniform_matrix(rows, cols)).to(dev)
            s_ = torch.empty(rows, device=dev)
            m_ = torch.empty(rows, device=dev)
            cl = [api.clause("add", s_), api.clause("max", m_)]
            out["%dx%d" % (rows, cols)] = _events_ms(lambda: api.accr_rowreduce(A, cl), reps)
            del A
            torch.cuda.empty_cache()
    return out


def tune_widths(kind="batch", candidates=None, reps=10):
    """Builds the kernel `kind` with every candidate width, times each build in
    a process of its own, and returns (best, {candidate: {workload: ms}}): the
    best by the geometric mean over the workloads."""
    from . import build
    source, macros, default = WIDTHS[kind]
    res = {}
    for cand in candidates or default:
        out_dir = os.path.join(build.BUILD, "widths_%s_%s" % (kind, "_".join(map(str, cand))))
        lib = build.build_variant(source, ["-D%s=%d" % (m, v) for m, v in zip(macros, cand)], out_dir)
        code = ("import json, sys; sys.path.insert(0, %r)\n"
                "from paper_1412_1127_gb300 import _native\n"
                "_native.LIB_PATH = %r\n"
                "from paper_1412_1127_gb300 import autotune\n"
                "print(json.dumps(autotune._time_this_library(%r, %d)))\n") % (
                    os.path.dirname(build.PKG), lib, kind, reps)
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("timing candidate %s of %s failed:\n%s" % (cand, kind, r.stderr[-2000:]))
        res[tuple(cand)] = json.loads(r.stdout.strip().splitlines()[-1])
    score = {c: math.exp(sum(math.log(v) for v in t.values()) / len(t)) for c, t in res.items()}
    return min(score, key=score.get), res


def tune_vectors(candidates=VECTOR_CANDIDATES, reps=10):
    """The batched-region kernel's widths (see tune_widths)."""
    best, res = tune_widths("batch", candidates, reps)
    return best, {c: {int(k): v for k, v in t.items()} for c, t in res.items()}


# table keys of each kind's widths, and of its timings
_KEYS = {"batch": (("tile_vectors", "warp_vectors", "min_ctas_per_sm"), "timings_ms"),
         "reduce": (("reduce_vectors",), "reduce_timings_ms"),
         "rows": (("row_vectors",), "row_timings_ms")}


def save_widths(kind, best, timings, path=TABLE, note=None):
    """Records a kind's chosen widths (and every candidate's timings) in the
    table's "vectors" entry, keeping the rest of the table."""
    with open(path) as f:
        d = json.load(f)
    v = d.get("vectors") or {}
    keys, tkey = _KEYS[kind]
    for k, b in zip(keys, best):
        v[k] = int(b)
    v[tkey] = {",".join(map(str, c)): {w: round(ms, 4) for w, ms in sorted(t.items())}
               for c, t in sorted(timings.items())}
    if note is not None:
        v["note"] = note
    d["vectors"] = v
    with open(path, "w") as f:
        json.dump(d, f, indent=1)
    return d


def save_vectors(best, timings, path=TABLE, note=""):
    """Records the batched-region kernel's widths (see save_widths)."""
    t = {c: {"2^%d" % (int(k).bit_length() - 1): ms for k, ms in tt.items()} for c, tt in timings.items()}
    return save_widths("batch", best, t, path, note)


NOTE = ("GB300 (152 SMs); batch: ms per prepared-batch launch of the 20,000-region workload, both length mixes, "
        "split from this table; reduce: ms per region of 2^27 int32 (+ into int64), float (compensated +), double "
        "(+); rows: ms per row nest (sum + max) of 65536 x 4096 and 64 x 2^22 floats; each kind's best by the "
        "geometric mean over its workloads")


if __name__ == "__main__":
    kinds = [k for k in ("batch", "reduce", "rows") if "--" + k in sys.argv or "--all" in sys.argv]
    if "--vectors" in sys.argv:
        kinds.append("batch")
    for kind in kinds:
        best, res = tune_widths(kind)
        print(json.dumps({"kind": kind, "best": best, "timings_ms": {",".join(map(str, c)): t for c, t in res.items()}}))
        if "--save" in sys.argv:
            save_widths(kind, best, res, note=NOTE)
