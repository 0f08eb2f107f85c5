"""Autotuner of the batched-region kernel: its split (warp-region threshold,
tile size) and its vector widths (16-byte vectors in flight per thread).

`tune(regions)` times every candidate (small_bytes, tile_bytes) pair on a
representative batch with CUDA events and returns the fastest; `apply()`
installs a pair process-wide through ``accr_batch_tiling``.  The split is a
function of each region's own type and length under a fixed pair, so once a
pair is chosen every region keeps giving the same bits alone and in any batch;
changing the pair changes the evaluation order of float sums.

`tune_vectors()` builds the kernel with each candidate pair of vector widths
(they are compile-time constants of the unrolled loops), times each build in a
process of its own on the 20,000-region workload of both length mixes, and
returns the fastest by the geometric mean; `save_vectors()` records it, and
the build compiles the recorded widths in.  Changing the widths also changes
the evaluation order of float sums.

The chosen values for GB300 are stored in ``tuning.json`` next to this file:
``load()`` applies the split, ``build.py`` reads the widths.

    python -m paper_1412_1127_gb300.autotune --vectors [--save]
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


# (tile vectors per thread, warp-region vectors per lane, CTAs per SM the
# registers are budgeted for)
VECTOR_CANDIDATES = [(4, 8, 4), (4, 4, 4), (8, 8, 4), (2, 8, 4), (4, 16, 3), (8, 16, 3)]
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


def _time_this_library(mixes, reps):
    """ms per prepared-batch launch of each length mix, with the split from
    the table (runs in the process that loaded the candidate library)."""
    load()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    out = {}
    for hi in mixes:
        regions, keep = _workload(dev, hi)
        d = load() or {"small_bytes": api.ACCR_SMALL_BYTES, "tile_bytes": api.ACCR_TILE_BYTES}
        out[str(hi)] = min(time_batch(regions, d["small_bytes"], d["tile_bytes"], reps) for _ in range(2))
        del regions, keep
        torch.cuda.empty_cache()
    return out


def tune_vectors(candidates=VECTOR_CANDIDATES, mixes=VECTOR_MIXES, reps=10):
    """Builds and times every candidate; returns (best, {candidate: {mix: ms}})."""
    from . import build
    res = {}
    for cand in candidates:
        bu, su, mb = cand
        out_dir = os.path.join(build.BUILD, "vectors_%d_%d_%d" % cand)
        lib = build.build_batch_variant(["-DACCR_BATCH_BU=%d" % bu, "-DACCR_BATCH_SU=%d" % su,
                                         "-DACCR_BATCH_MINB=%d" % mb], out_dir)
        code = ("import json, sys; sys.path.insert(0, %r)\n"
                "from paper_1412_1127_gb300 import _native\n"
                "_native.LIB_PATH = %r\n"
                "from paper_1412_1127_gb300 import autotune\n"
                "print(json.dumps(autotune._time_this_library(%r, %d)))\n") % (
                    os.path.dirname(build.PKG), lib, list(mixes), reps)
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("timing candidate %s failed:\n%s" % (cand, r.stderr[-2000:]))
        res[cand] = {int(k): v for k, v in json.loads(r.stdout.strip().splitlines()[-1]).items()}
    score = {c: math.exp(sum(math.log(v) for v in t.values()) / len(t)) for c, t in res.items()}
    return min(score, key=score.get), res


def save_vectors(best, timings, path=TABLE, note=""):
    """Records the chosen widths (and every candidate's timings) in the table."""
    with open(path) as f:
        d = json.load(f)
    d["vectors"] = {"tile_vectors": int(best[0]), "warp_vectors": int(best[1]), "min_ctas_per_sm": int(best[2]),
                    "note": note,
                    "timings_ms": {"%d,%d,%d" % c: {"2^%d" % (int(k).bit_length() - 1): round(v, 4)
                                                   for k, v in sorted(t.items())}
                                   for c, t in sorted(timings.items())}}
    with open(path, "w") as f:
        json.dump(d, f, indent=1)
    return d


if __name__ == "__main__":
    if "--vectors" in sys.argv:
        best, res = tune_vectors()
        print(json.dumps({"best": best, "timings_ms": {"%d,%d,%d" % c: t for c, t in res.items()}}))
        if "--save" in sys.argv:
            save_vectors(best, res, note="GB300 (152 SMs); ms per prepared-batch launch of the 20,000-region "
                                         "workload, both length mixes, split from this table; best by the "
                                         "geometric mean")
