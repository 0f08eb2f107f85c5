"""Host-side logic that needs no GPU: the bench's traffic record and source
hash, the autotuner's table, and the library's process-wide batch tiling."""
import json
import os
import shutil

import pytest

import bench
from paper_1412_1127_gb300 import api, autotune

REDUCE_SOURCES = ["paper_1412_1127_gb300/csrc/reduce.cu", "paper_1412_1127_gb300/csrc/fold.cuh"]


def test_committed_traffic_record_matches_the_current_kernel():
    """profiles/traffic.txt carries the hash of the reduce kernel it was taken
    on; it must be the current one (else bench.py reports traffic as null)."""
    assert bench.ncu_traffic("reduce_kernel", "scalar_2^28", REDUCE_SOURCES) is not None


def test_traffic_record_is_dropped_when_the_kernel_changes(tmp_path, monkeypatch):
    root = tmp_path / "repo"
    for f in REDUCE_SOURCES:
        os.makedirs(root / os.path.dirname(f), exist_ok=True)
        shutil.copy(os.path.join(bench.ROOT, f), root / f)
    os.makedirs(root / "profiles")
    shutil.copy(os.path.join(bench.ROOT, "profiles", "traffic.txt"), root / "profiles" / "traffic.txt")
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.ncu_traffic("reduce_kernel", "scalar_2^28", REDUCE_SOURCES) is not None
    # a change before the first kernel (host-side) keeps the hash ...
    src = root / REDUCE_SOURCES[0]
    text = src.read_text()
    src.write_text("// host-side note\n" + text)
    assert bench.ncu_traffic("reduce_kernel", "scalar_2^28", REDUCE_SOURCES) is not None
    # ... a change inside the device code drops the record
    i = text.index("__global__") + len("__global__")
    src.write_text(text[:i] + " /* changed */" + text[i:])
    assert bench.ncu_traffic("reduce_kernel", "scalar_2^28", REDUCE_SOURCES) is None
    assert bench.ncu_traffic("no_such_kernel", "scalar_2^28", REDUCE_SOURCES) is None
    # ... and so does another autotuned width compiled into the same source
    src.write_text(text)
    assert bench.ncu_traffic("reduce_kernel", "scalar_2^28", REDUCE_SOURCES) is not None
    from paper_1412_1127_gb300 import build
    real = build.tuned_defines
    monkeypatch.setattr(build, "tuned_defines",
                        lambda table=None, source="batch.cu": real(table, source) + (["-DACCR_REDUCE_RU=2"]
                                                                                  if source == "reduce.cu" else []))
    assert bench.ncu_traffic("reduce_kernel", "scalar_2^28", REDUCE_SOURCES) is None


def test_whole_job_rate_counts_every_rank():
    assert bench.whole_job_rate(10.0, 4, 2.0) == pytest.approx(20.0)


def test_autotune_table_roundtrip_and_apply(tmp_path):
    old = api.accr_batch_tiling()
    try:
        p = str(tmp_path / "t.json")
        d = autotune.save(32768, 1048576, {(32768, 1048576): 1.25, (65536, 2097152): 1.5}, path=p, note="x")
        assert json.load(open(p)) == d
        got = autotune.load(p)
        assert (got["small_bytes"], got["tile_bytes"]) == (32768, 1048576)
        assert tuple(api.accr_batch_tiling()) == (32768, 1048576)
        assert autotune.load(str(tmp_path / "missing.json")) is None
    finally:
        api.accr_batch_tiling(*old)


def test_committed_tuning_table_is_consistent():
    d = json.load(open(autotune.TABLE))
    assert d["small_bytes"] % 16 == 0 and d["tile_bytes"] % 16 == 0 and d["tile_bytes"] >= 4096
    assert "%d,%d" % (d["small_bytes"], d["tile_bytes"]) in d["timings_ms"]


def test_vector_widths_reach_the_build(tmp_path):
    """The widths the vector autotuner records become compile-time definitions
    of the batched-region kernel; the split tuner's save keeps them."""
    from paper_1412_1127_gb300 import build
    table = tmp_path / "tuning.json"
    with open(autotune.TABLE) as f:
        d = json.load(f)
    d.pop("vectors", None)
    table.write_text(json.dumps(d))
    assert build.tuned_defines(str(table)) == []
    timings = {(4, 8, 4): {1 << 17: 0.25, 1 << 20: 1.35}, (8, 16, 3): {1 << 17: 0.29, 1 << 20: 1.38}}
    autotune.save_vectors((4, 8, 4), timings, path=str(table))
    assert build.tuned_defines(str(table)) == ["-DACCR_BATCH_BU=4", "-DACCR_BATCH_SU=8", "-DACCR_BATCH_MINB=4"]
    autotune.save(65536, 2097152, {(65536, 2097152): 1.33}, path=str(table))
    got = json.loads(table.read_text())
    assert got["vectors"]["tile_vectors"] == 4 and got["vectors"]["timings_ms"]["8,16,3"]["2^20"] == 1.38
    assert got["small_bytes"] == 65536


def test_each_kernels_widths_reach_its_own_source(tmp_path):
    """The single-region and row kernels' widths go to their own sources only."""
    from paper_1412_1127_gb300 import build
    table = tmp_path / "tuning.json"
    table.write_text(json.dumps({"small_bytes": 65536, "tile_bytes": 2097152}))
    autotune.save_widths("reduce", (8,), {(2,): {"i32": 0.3}, (8,): {"i32": 0.2}}, path=str(table))
    autotune.save_widths("rows", (16,), {(16,): {"65536x4096": 0.15}}, path=str(table))
    assert build.tuned_defines(str(table), "reduce.cu") == ["-DACCR_REDUCE_RU=8"]
    assert build.tuned_defines(str(table), "rowreduce.cu") == ["-DACCR_ROW_RU=16"]
    assert build.tuned_defines(str(table), "batch.cu") == []
    assert build.tuned_defines(str(table), "server.cu") == []
    assert json.loads(table.read_text())["vectors"]["reduce_timings_ms"]["2"]["i32"] == 0.3
