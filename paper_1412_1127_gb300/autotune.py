"""Autotuner of the batched-region split (warp-region threshold, tile size).

`tune(regions)` times every candidate (small_bytes, tile_bytes) pair on a
representative batch with CUDA events and returns the fastest; `apply()`
installs a pair process-wide through ``accr_batch_tiling``.  The split is a
function of each region's own type and length under a fixed pair, so once a
pair is chosen every region keeps giving the same bits alone and in any batch;
changing the pair changes the evaluation order of float sums.

The chosen pair for GB300 is stored in ``tuning.json`` next to this file and
applied by ``load()``.
"""
import json
import os

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
    d = {"small_bytes": int(small_bytes), "tile_bytes": int(tile_bytes), "note": note,
         "timings_ms": {"%d,%d" % k: round(v, 4) for k, v in sorted(timings.items())}}
    with open(path, "w") as f:
        json.dump(d, f, indent=1)
    return d
