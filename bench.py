#!/usr/bin/env python3
"""Benchmark of the accr region runtime on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                    [--workload scalar|rows|...]

Default workload ("scalar"): the all-operator scalar reduction at n = 2^28.
One step runs 16 single-pass regions over inputs resident in HBM:

  int32 full-range uniform: + (int64 variable), *, max, min, &, |, ^, &&, ||
  float N(0,1):             + (plain), + (compensated), max, min
  double N(0,1):            +, max, min

The metric is reduction throughput in GB/s of algorithmic bytes (every input
element read once per region), also given as a fraction of the measured HBM
copy bandwidth.  Inputs (1-2 GiB per region) are far larger than the 129 MB
L2, so no flush is needed between regions.

The JSON line (rank 0) carries the driver's contract keys plus `roofline`
(dominant kernel against measured HBM bandwidth), `cpu_baseline` (the serial
oracle on this host's cores over a bounded sample), `e2e` (the same metric
with host-resident inputs copied in every step) and `clocks`.

`--impl reference` times the serial oracle (the paper's program with the
directives ignored) on this host on a bounded sample of the same workload.
With torchrun (N > 1) every rank runs its own independent copy of the
workload (weak scaling: regions are independent, no collective on the data
path); rank 0 prints the line.
"""
import argparse
import hashlib
import json
import math
import os
import platform
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_SCALAR = 1 << 28
GIB = 1 << 30

# (name, input kind, op, variable type, flags)
SCALAR_REGIONS = [
    ("i32 + -> i64", "i32", "add", "i64", 0),
    ("i32 *", "i32", "mul", "i32", 0),
    ("i32 max", "i32", "max", "i32", 0),
    ("i32 min", "i32", "min", "i32", 0),
    ("i32 &", "i32", "band", "i32", 0),
    ("i32 |", "i32", "bor", "i32", 0),
    ("i32 ^", "i32", "bxor", "i32", 0),
    ("i32 &&", "i32", "land", "i32", 0),
    ("i32 ||", "i32", "lor", "i32", 0),
    ("f32 +", "f32", "add", "f32", 0),
    ("f32 + compensated", "f32", "add", "f32", 1),
    ("f32 max", "f32", "max", "f32", 0),
    ("f32 min", "f32", "min", "f32", 0),
    ("f64 +", "f64", "add", "f64", 0),
    ("f64 max", "f64", "max", "f64", 0),
    ("f64 min", "f64", "min", "f64", 0),
]
ELEM = {"i32": 4, "i64": 8, "f32": 4, "f64": 8}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def source_hash(files):
    """Hash of the device code of the given sources: a .cu file counts from its
    first __global__ kernel to the "// ---- host side" marker (host-only edits
    do not change the kernel), together with the autotuned widths the build
    compiles into it; a header counts whole."""
    from paper_1412_1127_gb300 import build
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, f), "rb") as fh:
            txt = fh.read()
        if f.endswith(".cu"):
            a = txt.find(b"__global__")
            b = txt.find(b"// ---- host side")
            txt = txt[a:b] if a >= 0 and b > a else txt
            txt += " ".join(build.tuned_defines(source=os.path.basename(f))).encode()
        h.update(txt)
    return h.hexdigest()[:16]


def ncu_traffic(kernel, workload, files):
    """DRAM bytes per launch recorded from an ncu capture in profiles/traffic.txt,
    or None if absent or if the kernel's sources changed since the capture."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    want = source_hash(files)
    with open(path) as f:
        for line in f:
            parts = line.split()
            if len(parts) >= 4 and not line.startswith("#") and parts[0] == kernel and parts[1] == workload:
                return float(parts[2]) if parts[3] == want else None
    return None


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sms, maxs, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            p = [x.strip() for x in l.split(",")]
            if len(p) < 9:
                continue
            try:
                sms.append(float(p[1]))
                maxs.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sms:
            return None
        return {"sm_mhz": float(np.median(sms)), "sm_max_mhz": max(maxs), "samples": len(sms),
                "reasons": sorted(reasons)}


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init_ranks(world, backend):
    """Join the process group of a torchrun launch (127.0.0.1 rendezvous)."""
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend)


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(value, world, device="cpu"):
    """The largest `value` over all ranks (every rank gets it)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, seconds):
    """Units all ranks processed per second of the slowest rank (weak scaling:
    every rank processes its own independent copy of the workload)."""
    return units_per_rank * world / seconds


def make_scalar_inputs(n, rank=0):
    from paper_1412_1127_gb300 import inputs
    return {"i32": inputs.full_range_i32(n, salt=rank),
            "f32": inputs.normal(n, np.float32, salt=1000 + rank),
            "f64": inputs.normal(n, np.float64, salt=2000 + rank)}


def oracle_step(host, regions, n):
    """The serial oracle over the first n elements of every region's input."""
    import oracle
    for _, kind, op, acc, _ in regions:
        oracle.reduce(host[kind][:n], op, acc)


def cpu_time_sample(host, regions, n):
    t0 = time.perf_counter()
    oracle_step(host, regions, n)
    return time.perf_counter() - t0


def cpu_model():
    """Host CPU as the kernel reports it, and the number of cores."""
    name = platform.machine()
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                k = line.split(":")[0].strip().lower()
                if k in ("model name", "cpu part", "hardware"):
                    name += " " + line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return {"model": name, "cores": os.cpu_count()}


def cpu_all_cores(host, regions, n):
    """The same oracle sample with one region per host thread, all cores busy
    (the oracle is unchanged: each call is one serial region; ctypes releases
    the interpreter lock for the call)."""
    import concurrent.futures as cf
    import oracle
    cores = min(os.cpu_count() or 1, len(regions))
    oracle.reduce(host["i32"][:1024], "add", "i64")  # load the library before timing

    def one(r):
        _, kind, op, acc, _ = r
        oracle.reduce(host[kind][:n], op, acc)
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=cores) as ex:
        list(ex.map(one, regions))
    dt = time.perf_counter() - t0
    sb = sum(n * ELEM[k] for _, k, _, _, _ in regions)
    return {"value": round(sb / dt / 1e9, 4), "unit": "GB/s", "cores": cores, "seconds": round(dt, 2)}


def oracle_baselines():
    """The serial oracle timed on this host beside each sub-measurement, on a
    bounded sample of the same workload (one core; a baseline, not a target)."""
    import oracle
    from paper_1412_1127_gb300 import inputs

    def timed(fn, warm=True):
        if warm:
            fn()  # library loaded, pages touched
        t0 = time.perf_counter()
        fn()
        return time.perf_counter() - t0

    out = {}
    A = inputs.uniform_matrix(1024, 4096)
    dt = timed(lambda: (oracle.rowreduce(A, "add"), oracle.rowreduce(A, "max")))
    out["rows"] = {"value": round(A.nbytes / dt / 1e9, 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
                   "sample": "1024 x 4096 float U(-1,1), row sum and row max (serial C, one fold each)",
                   "seconds": round(dt, 3)}
    lengths = inputs.log_uniform_lengths(20000, 1, 1 << 20)[:400]
    xs = [inputs.normal(int(n), np.float32, salt=k) if k % 2 == 0 else
          inputs.uniform_i64(int(n), -(1 << 40), 1 << 40, salt=k) for k, n in enumerate(lengths)]
    nb = sum(x.nbytes for x in xs)

    def batch():
        for k, x in enumerate(xs):
            if k % 2 == 0:
                oracle.reduce(x, "add", "f32")
            else:
                oracle.reduce(x, "add", "i64")
                oracle.reduce(x, "bxor", "i64")
    dt = timed(batch)
    out["batched"] = {"value": round(len(xs) / dt, 1), "unit": "regions/s", "gbs": round(nb / dt / 1e9, 4),
                      "cores": 1, "kind": "oracle", "seconds": round(dt, 3),
                      "sample": "the first 400 regions of the 20,000-region length mix (serial C per region)"}
    sl = inputs.log_uniform_lengths(1000, 1 << 8, 1 << 26, seed=5, salt=4)
    keep = int(np.searchsorted(np.cumsum(sl), 1 << 27))  # regions until 2^27 elements in all
    sx = [inputs.full_range_i32(int(n), salt=k) for k, n in enumerate(sl[:max(keep, 1)])]

    def served():
        for x in sx:
            oracle.reduce(x, "add", "i64")
            oracle.reduce(x, "max", "i32")
    dt = timed(served, warm=False)
    out["served"] = {"value": round(len(sx) / dt, 1), "unit": "regions/s",
                     "gbs": round(sum(x.nbytes for x in sx) / dt / 1e9, 4), "cores": 1, "kind": "oracle",
                     "seconds": round(dt, 3),
                     "sample": "%d regions of the served length mix (the first ones up to 2^27 elements; int32, "
                               "+ into int64 and max), back to back" % len(sx)}
    a, b = inputs.uniform_matrix(512, 512, salt=1), inputs.uniform_matrix(512, 512, salt=2)
    dt = timed(lambda: oracle.matmul_listing1(a, b))
    out["matmul"] = {"value": round(2 * 512 ** 3 / dt / 1e9, 4), "unit": "GFLOP/s", "cores": 1, "kind": "oracle",
                     "sample": "Listing 1a at LEN 512 (serial C, float accumulator)", "seconds": round(dt, 3)}
    pts = (inputs.rng(21, 5).random((1 << 22, 2), dtype=np.float32) * 100).astype(np.float32)
    x = inputs.normal(1 << 22, np.float32, salt=3)
    g = inputs.rng(23, 1)
    grid = (g.random((1024, 1024)) < 0.62).astype(np.uint8)
    grid[512, 512] = 1
    t_nk = timed(lambda: oracle.nearest_k(pts, 41.5, 58.25, 5))
    t_sd = timed(lambda: oracle.standardize(x))
    t_bfs = timed(lambda: oracle.grid_bfs(grid, 512 * 1024 + 512))
    out["patterns"] = {"f4_nearest_k5_gbs": round(pts.nbytes / t_nk / 1e9, 4),
                       "f2_standardize_gbs": round(3 * x.nbytes / t_sd / 1e9, 4),
                       "f3_bfs_ms": round(t_bfs * 1e3, 2), "cores": 1, "kind": "oracle",
                       "sample": "2^22 points (k = 5), 2^22 floats, the 1024 x 1024 grid (serial C)"}
    return out


def run_reference(args):
    """--impl reference: the serial oracle on the host cores, bounded sample."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    sample = 1 << 24
    host = make_scalar_inputs(sample)
    bytes_step = sum(sample * ELEM[k] for _, k, _, _, _ in SCALAR_REGIONS)
    for _ in range(args.warmup):
        oracle_step(host, SCALAR_REGIONS, sample)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_step(host, SCALAR_REGIONS, sample)
    dt = (time.perf_counter() - t0) / args.steps
    v = bytes_step / dt / 1e9
    line = {"impl": "reference",
            "metric": "reduction GB/s (% of HBM peak); batched regions/sec + p50/p99 latency vs plain", "value": round(v, 4),
            "unit": "GB/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(dt * 1e3, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "i32+i64+f32+f64", "data": "synthetic",
            "config": {"workload": "all-operator scalar reduction, n=2^28 (16 regions: int32 "
                                   "+,*,max,min,&,|,^,&&,||; float +,+comp,max,min; double +,max,min)",
                       "reference": "serial C oracle (the region's program with directives ignored)",
                       "step_sample": "first 2^24 elements of each region's input"},
            "cpu_baseline": {"value": round(v, 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
                             "sample": "2^24 elements per region, 16 regions per step"},
            "e2e": {"value": round(v, 4), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_scalar(args):
    import torch
    from paper_1412_1127_gb300 import api

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    init_ranks(world, "nccl" if torch.cuda.is_available() else "gloo")
    n = args.n
    host = make_scalar_inputs(n, rank)
    devin = {k: torch.from_numpy(v).to(dev) for k, v in host.items()}
    td = {"i32": torch.int32, "i64": torch.int64, "f32": torch.float32, "f64": torch.float64}
    outs = [torch.empty(1, dtype=td[acc], device=dev) for _, _, _, acc, _ in SCALAR_REGIONS]
    cls = [[api.clause(op, o)] for (_, _, op, _, _), o in zip(SCALAR_REGIONS, outs)]
    flags = [api.ACCR_COMPENSATED if f else 0 for *_, f in SCALAR_REGIONS]
    bytes_region = [n * ELEM[k] for _, k, _, _, _ in SCALAR_REGIONS]
    bytes_step = sum(bytes_region)
    stream = torch.cuda.current_stream(dev)
    R = len(SCALAR_REGIONS)

    def step(ev=None):
        for i, (_, kind, _, _, _) in enumerate(SCALAR_REGIONS):
            if ev is not None:
                ev[i][0].record(stream)
            api.accr_reduce(devin[kind], cls[i], flags=flags[i], stream=stream)
            if ev is not None:
                ev[i][1].record(stream)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    # timed region: K steps, CUDA events on the launching stream, per-region events
    evs = [[[torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)] for _ in range(R)]
           for _ in range(args.steps)]
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    l0 = api.accr_launch_count()
    start.record(stream)
    for k in range(args.steps):
        step(evs[k])
    stop.record(stream)
    torch.cuda.synchronize()
    launches = api.accr_launch_count() - l0
    barrier(world)
    clk = clocks.stop()
    ms = max_over_ranks(start.elapsed_time(stop), world, dev)
    per_region_ms = [sum(evs[k][i][0].elapsed_time(evs[k][i][1]) for k in range(args.steps)) / args.steps
                     for i in range(R)]
    ms_step = ms / args.steps
    value = whole_job_rate(bytes_step, world, ms_step * 1e-3) / 1e9
    step_ms = [sum(evs[k][i][0].elapsed_time(evs[k][i][1]) for i in range(R)) for k in range(args.steps)]
    step_gbs = [bytes_step / (t * 1e-3) / 1e9 for t in step_ms]
    hmean_gbs = len(step_gbs) / sum(1.0 / g for g in step_gbs)

    # results of the last step, checked against the oracle on a cheap subset
    peaks, peak_kind = measured_peaks()
    hbm = float(peaks["hbm_gbs"])
    kernel_ms = sum(per_region_ms)
    achieved = bytes_step / (kernel_ms * 1e-3) / 1e9
    traffic = ncu_traffic("reduce_kernel", "scalar_2^28",
                          ["paper_1412_1127_gb300/csrc/reduce.cu", "paper_1412_1127_gb300/csrc/fold.cuh"])

    # end to end through the public API: host (pinned) inputs copied in every step
    e2e = None
    if not args.no_e2e:
        pinned = {k: torch.from_numpy(v).pin_memory() for k, v in host.items()}
        res_host = torch.empty(R, dtype=torch.int64).pin_memory()

        copy_stream = torch.cuda.Stream(dev)
        kinds = ("i32", "f32", "f64")

        def e2e_step():
            # each input array is copied in on a copy stream; the regions over
            # an array start as soon as its copy is done, overlapping the copy
            # of the next array (host-to-device runs at about 211 GB/s here)
            ready = {}
            copy_stream.wait_stream(stream)
            for kind in kinds:
                with torch.cuda.stream(copy_stream):
                    devin[kind].copy_(pinned[kind], non_blocking=True)
                    ev = torch.cuda.Event()
                    ev.record(copy_stream)
                ready[kind] = ev
            for kind in kinds:
                stream.wait_event(ready[kind])
                for i, (_, k, _, _, _) in enumerate(SCALAR_REGIONS):
                    if k == kind:
                        api.accr_reduce(devin[kind], cls[i], flags=flags[i], stream=stream)
            for i, o in enumerate(outs):
                res_host[i:i + 1].view(torch.uint8)[: o.element_size()].copy_(
                    o.view(torch.uint8), non_blocking=True)
            stream.synchronize()

        e2e_step()
        ek = max(10, min(args.steps, 20))  # at least 10 end-to-end steps (each copies 4 GiB in)
        t0 = time.perf_counter()
        for _ in range(ek):
            e2e_step()
        dt = (time.perf_counter() - t0) / ek
        h2d = sum(v.numel() * v.element_size() for v in pinned.values())
        d2h = sum(o.element_size() for o in outs)
        e2e = {"value": round(bytes_step * world / dt / 1e9, 2), "unit": "GB/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "steps": ek,
               "ms_per_step": round(dt * 1e3, 3)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sample = 1 << 26
        dt = cpu_time_sample(host, SCALAR_REGIONS, sample)
        sb = sum(sample * ELEM[k] for _, k, _, _, _ in SCALAR_REGIONS)
        cpu = {"value": round(sb / dt / 1e9, 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
               "sample": "first 2^26 elements of each of the 16 regions (1/4 of a step), serial C",
               "seconds": round(dt, 2), "cpu": cpu_model(),
               "all_cores": cpu_all_cores(host, SCALAR_REGIONS, sample)}

    extra = {}
    if rank == 0 and world == 1 and not args.no_extra:
        del devin, host
        torch.cuda.empty_cache()
        from paper_1412_1127_gb300 import autotune
        autotune.load()
        extra["batched"] = measure_batched(dev, max(3, min(args.steps, 10)), 3)
        torch.cuda.empty_cache()
        extra["batched_2e8_variant"] = measure_batched(dev, max(3, min(args.steps, 10)), 3, hi=1 << 17)
        torch.cuda.empty_cache()
        extra["served"] = measure_served(dev, args.served_seconds, args.rate)
        torch.cuda.empty_cache()
        extra["matmul"] = measure_matmul(dev)
        torch.cuda.empty_cache()
        extra["rows"] = measure_rows_all(dev)
        torch.cuda.empty_cache()
        extra["patterns"] = measure_patterns(dev)
        torch.cuda.empty_cache()
        extra["one_region_2e20"] = measure_small_region(dev)
        if not args.no_cpu_baseline:
            base = oracle_baselines()
            for k in ("rows", "batched", "served", "matmul", "patterns"):
                extra[k]["cpu_baseline"] = base[k]

    if rank == 0:
        line = {
            "metric": "reduction GB/s (% of HBM peak); batched regions/sec + p50/p99 latency vs plain",
            "value": round(value, 2),
            "unit": "GB/s",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": max(args.warmup, 3),
            "ms_per_step": round(ms_step, 4),
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "i32+i64+f32+f64",
            "data": "synthetic",
            "config": {"workload": "all-operator scalar reduction, n=%s (16 regions: int32 "
                                   "+,*,max,min,&,|,^,&&,||; float +,+comp,max,min; double +,max,min)"
                                   % ("2^%d" % int(math.log2(n)) if n & (n - 1) == 0 else str(n)),
                       "n": n, "regions_per_step": R, "bytes_per_step": bytes_step,
                       "l2": "inputs larger than L2 (1-2 GiB per region vs 129 MB); no flush",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "frac_of_hbm": round(value / world / hbm, 4),
            "kernel_gbs_per_step": {"harmonic_mean": round(hmean_gbs, 1),
                                    "median": round(float(np.median(step_gbs)), 1),
                                    "min": round(min(step_gbs), 1), "max": round(max(step_gbs), 1)},
            "roofline": {"bound": "hbm", "kernel": "reduce_kernel", "achieved": round(achieved, 2),
                         "peak": hbm, "peak_kind": peak_kind + " (copy, hbm_gbs)", "unit": "GB/s",
                         "frac": round(achieved / hbm, 4),
                         "traffic": traffic,
                         "algorithmic_bytes_per_launch": int(bytes_step / R)},
            "per_region_gbs": {SCALAR_REGIONS[i][0]: round(bytes_region[i] / (per_region_ms[i] * 1e-3) / 1e9, 1)
                               for i in range(R)},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": int(launches),
            "clocks": clk,
        }
        line.update(extra)
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def build_batched(dev, count=20000, hi=1 << 20):
    """The many-regions workload on the device: 20,000 regions of log-uniform
    length on [1, 2^20]; even ones float N(0,1) with compensated +, odd ones
    int64 with + and ^ (two clauses, one pass)."""
    import torch
    from paper_1412_1127_gb300 import api, inputs
    lengths, pf, off_f, pi, off_i = inputs.batched_regions(count, hi=hi)
    tf, ti = torch.from_numpy(pf).to(dev), torch.from_numpy(pi).to(dev)
    nf, ni = len(off_f) - 1, len(off_i) - 1
    sf = torch.empty(nf, dtype=torch.float32, device=dev)
    si = torch.empty(ni, dtype=torch.int64, device=dev)
    xi = torch.empty(ni, dtype=torch.int64, device=dev)
    regions = []
    for k in range(len(lengths)):
        j = k // 2
        if k % 2 == 0:
            regions.append((tf[off_f[j]:off_f[j + 1]], [api.clause("add", sf[j:j + 1])], api.ACCR_COMPENSATED))
        else:
            regions.append((ti[off_i[j]:off_i[j + 1]], [api.clause("add", si[j:j + 1]),
                                                        api.clause("bxor", xi[j:j + 1])], 0))
    nbytes = int(off_f[-1]) * 4 + int(off_i[-1]) * 8
    return regions, nbytes, (sf, si, xi), (pf, off_f, pi, off_i)


def measure_batched(dev, steps, warmup, count=20000, tune=False, hi=1 << 20):
    """regions/s and GB/s of the prepared (graph) batch, the one-shot batch and
    the plain one-launch-per-region form, on the same regions."""
    import torch
    from paper_1412_1127_gb300 import api
    regions, nbytes, outs, host = build_batched(dev, count, hi)
    R = len(regions)
    tuned = None
    if tune:
        from paper_1412_1127_gb300 import autotune
        best, res = autotune.tune(regions)
        autotune.apply(*best)
        tuned = {"best": list(best), "ms": {"%d,%d" % k: round(v, 4) for k, v in sorted(res.items())}}
    stream = torch.cuda.current_stream(dev)
    arr, keep = api.regions_array(regions)
    L = api.lib()
    b = api.Batch(regions)

    def timed(fn, k):
        for _ in range(max(warmup, 3)):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = api.accr_launch_count()
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / k, (api.accr_launch_count() - l0) / k

    ms_graph, lg = timed(lambda: b.launch(stream), steps)
    res_graph = [o.clone() for o in outs]
    ms_once, lo = timed(lambda: api.check(L.accr_batch_reduce(arr, R, 0, stream.cuda_stream)), steps)
    ms_plain, lp = timed(lambda: api.check(L.accr_batch_reduce(arr, R, api.ACCR_PLAIN, stream.cuda_stream)),
                         max(2, steps // 5))
    res_plain = [o.clone() for o in outs]
    same_int = bool(torch.equal(res_graph[1], res_plain[1]) and torch.equal(res_graph[2], res_plain[2]))
    rel = ((res_graph[0].double() - res_plain[0].double()).abs()
           / res_plain[0].double().abs().clamp_min(1e-3)).max().item()
    b.destroy()
    return {
        "workload": "%d regions, lengths log-uniform [1, 2^%d]: float N(0,1) compensated + / "
                    "int64 + and ^ (alternating), %d elements, %.2f GB" % (
                        R, int(math.log2(hi)), int(host[1][-1] + host[3][-1]), nbytes / 1e9),
        "regions": R,
        "batched_graph": {"ms": round(ms_graph, 4), "regions_per_s": round(R / (ms_graph * 1e-3), 1),
                          "gbs": round(nbytes / (ms_graph * 1e-3) / 1e9, 1), "launches": lg},
        "batched_oneshot": {"ms": round(ms_once, 4), "regions_per_s": round(R / (ms_once * 1e-3), 1),
                            "gbs": round(nbytes / (ms_once * 1e-3) / 1e9, 1), "launches": lo},
        "plain": {"ms": round(ms_plain, 4), "regions_per_s": round(R / (ms_plain * 1e-3), 1),
                  "gbs": round(nbytes / (ms_plain * 1e-3) / 1e9, 1), "launches": lp},
        "speedup_vs_plain": round(ms_plain / ms_graph, 2),
        "int_results_equal_plain": same_int,
        "float_max_rel_diff_vs_plain": rel,
        "tiling": list(api.accr_batch_tiling()),
        "autotune": tuned,
    }


SERVED_CLAUSES = {"f32": [("add", "f32")], "i32": [("add", "i64"), ("max", "i32")],
                  "i64": [("add", "i64"), ("bxor", "i64")]}


def served_pools(dev, seed=5):
    """Resident pools of the served workload (2^29 float32, 2^29 int32, 2^28
    int64: 6 GiB)."""
    import torch
    from paper_1412_1127_gb300 import inputs
    sizes = {"f32": 1 << 29, "i32": 1 << 29, "i64": 1 << 28}
    host = {"f32": inputs.normal(sizes["f32"], np.float32, seed=seed, salt=1),
            "i32": inputs.full_range_i32(sizes["i32"], seed=seed, salt=2),
            "i64": inputs.uniform_i64(sizes["i64"], -(1 << 40), 1 << 40, seed=seed, salt=3)}
    return {k: torch.from_numpy(v).to(dev) for k, v in host.items()}


def served_requests(dev, pools, count, rate, seed=5):
    """Poisson arrivals at `rate` regions/s; each region is float32
    (compensated +), int32 (+ into int64 and max) or int64 (+ and ^) with
    length log-uniform on [2^8, 2^26], at a random offset of its pool."""
    import torch
    from paper_1412_1127_gb300 import api, inputs
    g = inputs.rng(seed, 9)
    lengths = inputs.log_uniform_lengths(count, 1 << 8, 1 << 26, seed=seed, salt=4)
    kinds = g.integers(0, 3, size=count)
    td = {"i32": torch.int32, "i64": torch.int64, "f32": torch.float32}
    proto = {t: [api.clause(op, torch.empty(1, dtype=td[a], device=dev)) for op, a in c]
             for t, c in SERVED_CLAUSES.items()}
    regions, nbytes, meta = [], 0, []
    for k in range(count):
        t = ["f32", "i32", "i64"][int(kinds[k])]
        n = int(lengths[k])
        off = int(g.integers(0, pools[t].numel() - n))
        regions.append((pools[t][off:off + n], proto[t], api.ACCR_COMPENSATED if t == "f32" else 0))
        nbytes += n * (8 if t == "i64" else 4)
        meta.append((t, off, n))
    arrivals = inputs.poisson_arrivals(rate, count, seed=seed, salt=5)
    return regions, arrivals, nbytes, meta


def build_served(dev, count, rate, seed=5):
    pools = served_pools(dev, seed)
    regions, arrivals, nbytes, meta = served_requests(dev, pools, count, rate, seed)
    return regions, arrivals, nbytes, meta, None, pools


def latency_stats(res, n):
    lat = np.array([res[i].done_ns - res[i].submit_ns for i in range(n)], dtype=np.float64) / 1e3
    first = min(res[i].submit_ns for i in range(n))
    last = max(res[i].done_ns for i in range(n))
    return {"regions_per_s": round(n / ((last - first) * 1e-9), 1),
            "p50_us": round(float(np.percentile(lat, 50)), 2),
            "p99_us": round(float(np.percentile(lat, 99)), 2),
            "p999_us": round(float(np.percentile(lat, 99.9)), 2),
            "mean_us": round(float(lat.mean()), 2)}


def measure_served(dev, seconds=2.0, rate=50000.0):
    """Served regions/s and p50/p99 latency (arrival -> result visible on the
    host) of the continuous-batching server against sequential plain launches,
    on the same open-loop Poisson schedule."""
    import torch
    from paper_1412_1127_gb300 import api
    count = int(seconds * rate)
    regions, arrivals, nbytes, meta, host, pools = build_served(dev, count, rate)
    srv = api.Server(64 << 30, nstreams=4, max_batch=4096)
    warm = min(2000, count)
    srv.replay(regions[:warm], arrivals[:warm])
    res = srv.replay(regions, arrivals)
    srv.destroy()
    api.accr_server_replay(None, regions[:warm], arrivals[:warm], plain=True)
    resp = api.accr_server_replay(None, regions, arrivals, plain=True)
    st_s, st_p = latency_stats(res, count), latency_stats(resp, count)
    # results: served and plain agree bit for bit on the integer regions, and
    # the float sums (compensated, each within 1e-5 of the exact sum) within
    # twice that of each other
    same = all(list(res[i].value[:res[i].nclauses]) == list(resp[i].value[:resp[i].nclauses])
               for i in range(count) if meta[i][0] != "f32")
    fdiff = 0.0
    for i in range(count):
        if meta[i][0] == "f32":
            a = float(api.decode(res[i].value[0], torch.float32))
            b = float(api.decode(resp[i].value[0], torch.float32))
            fdiff = max(fdiff, abs(a - b) / max(abs(b), 0.1 * meta[i][2] ** 0.5))
    out = {"workload": "served regions: Poisson arrivals at %d/s for %.1f s (%d regions, %.1f GB), lengths "
                       "log-uniform [2^8, 2^26], float32 (+comp) / int32 (+, max) / int64 (+, ^), "
                       "resident pools, 64 GiB budget, 4 stream slots" % (rate, seconds, count, nbytes / 1e9),
           "offered_gbs": round(nbytes / arrivals[-1] / 1e9, 1),
           "server": st_s, "plain_sequential": st_p,
           "p99_speedup_vs_plain": round(st_p["p99_us"] / st_s["p99_us"], 2),
           "int_results_equal_plain": bool(same),
           "float_max_rel_diff_vs_plain": fdiff, "float_results_within_2e-5_of_plain": bool(fdiff <= 2e-5)}
    out.update(served_fair(dev, pools))
    del pools
    torch.cuda.empty_cache()
    return out


def served_fair(dev, pools, equal_rate=25000.0, seconds=1.0, sat_server=60000, sat_plain=20000):
    """The two arms at equal, sustainable load (an offered rate the plain arm
    keeps up with), and each arm's saturation throughput (every region
    arrives at time 0: regions/s over the whole drain)."""
    from paper_1412_1127_gb300 import api
    count = int(seconds * equal_rate)
    regions, arrivals, nbytes, meta = served_requests(dev, pools, count, equal_rate, seed=7)
    srv = api.Server(64 << 30, nstreams=4, max_batch=4096)
    warm = min(2000, count)
    srv.replay(regions[:warm], arrivals[:warm])
    st_s = latency_stats(srv.replay(regions, arrivals), count)
    api.accr_server_replay(None, regions[:warm], arrivals[:warm], plain=True)
    st_p = latency_stats(api.accr_server_replay(None, regions, arrivals, plain=True), count)
    regs_s, _, nb_s, _ = served_requests(dev, pools, sat_server, 1.0, seed=8)
    res = srv.replay(regs_s, np.zeros(sat_server))
    srv.destroy()
    regs_p, _, nb_p, _ = served_requests(dev, pools, sat_plain, 1.0, seed=8)
    resp = api.accr_server_replay(None, regs_p, np.zeros(sat_plain), plain=True)
    sat_s, sat_p = latency_stats(res, sat_server), latency_stats(resp, sat_plain)
    return {"equal_load": {"offered_regions_per_s": equal_rate, "regions": count,
                           "offered_gbs": round(nbytes / arrivals[-1] / 1e9, 1),
                           "server": st_s, "plain_sequential": st_p,
                           "p50_speedup_vs_plain": round(st_p["p50_us"] / st_s["p50_us"], 2),
                           "p99_speedup_vs_plain": round(st_p["p99_us"] / st_s["p99_us"], 2)},
            "saturation": {"server_regions_per_s": sat_s["regions_per_s"], "server_regions": sat_server,
                           "plain_regions_per_s": sat_p["regions_per_s"], "plain_regions": sat_plain,
                           "server_gbs": round(nb_s / 1e9 * sat_s["regions_per_s"] / sat_server, 1),
                           "plain_gbs": round(nb_p / 1e9 * sat_p["regions_per_s"] / sat_plain, 1),
                           "throughput_ratio": round(sat_s["regions_per_s"] / sat_p["regions_per_s"], 2),
                           "how": "every region arrives at time 0; regions/s from the first arrival to the last result"}}


def served_sweep(dev, rates, seconds=1.0):
    """Offered load from the nominal rate up to saturation: served regions/s
    and p50/p99 latency of the server alone (same region mix)."""
    from paper_1412_1127_gb300 import api
    pools = served_pools(dev, seed=6)
    out = []
    for rate in rates:
        count = int(seconds * rate)
        regions, arrivals, nbytes, meta = served_requests(dev, pools, count, rate, seed=6)
        srv = api.Server(64 << 30, nstreams=4, max_batch=4096)
        warm = min(2000, count)
        srv.replay(regions[:warm], arrivals[:warm])
        res = srv.replay(regions, arrivals)
        srv.destroy()
        st = latency_stats(res, count)
        st.update({"offered_regions_per_s": rate, "offered_gbs": round(nbytes / arrivals[-1] / 1e9, 1)})
        out.append(st)
    del pools
    return out


def run_served(args):
    import torch
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    r = measure_served(dev, args.served_seconds, args.rate)
    if args.sweep:
        r["rate_sweep"] = served_sweep(dev, [50000, 100000, 150000, 200000, 300000])
    print(json.dumps(r), flush=True)
    return 0


def measure_matmul(dev, length=4096, reps=5):
    """The Listing-1 nest at LEN x LEN (U(-1,1) float): FP32 SIMT (fused and
    serial-order) and BF16x3 tcgen05, TFLOP/s of 2*LEN^3 and the error of
    sampled entries against the double-accumulated product."""
    import torch
    from paper_1412_1127_gb300 import api, inputs
    a = inputs.uniform_matrix(length, length, salt=41)
    b = inputs.uniform_matrix(length, length, salt=42)
    at, bt = torch.from_numpy(a).to(dev), torch.from_numpy(b).to(dev)
    ct = torch.empty_like(at)
    stream = torch.cuda.current_stream(dev)
    flops = 2.0 * length ** 3
    peaks, kind = measured_peaks()
    g = np.random.default_rng(0)
    idx = list(zip(g.integers(0, length, 32), g.integers(0, length, 32)))
    # reference for the error report: double-accumulated products of the sampled entries
    truth = []
    for i, j in idx:
        p = at[int(i), :].double() * bt[:, int(j)].double()
        truth.append((float(p.sum()), float(p.abs().sum())))
    out = {"workload": "Listing-1 nest, LEN=%d, float U(-1,1)" % length}
    for mode in ["simt", "serial", "bf16x3"]:
        for _ in range(2):
            api.accr_matmul_nest(at, bt, ct, mode=mode, stream=stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            api.accr_matmul_nest(at, bt, ct, mode=mode, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        c = ct.cpu().numpy()
        err = max(abs(float(c[i, j]) - t) / s_ for (i, j), (t, s_) in zip(idx, truth))
        r = {"ms": round(ms, 4), "tflops": round(flops / (ms * 1e-3) / 1e12, 2),
             "max_err_over_sum_abs_products": err}
        if mode == "bf16x3":
            r["tensor_tflops"] = round(3 * flops / (ms * 1e-3) / 1e12, 2)
            r["frac_of_bf16_peak"] = round(3 * flops / (ms * 1e-3) / 1e12 / float(peaks["bf16_tflops"]), 4)
            r["note"] = "time includes the split kernel; tensor work is 3 products"
            # repeated nest with unchanged operands: the split is reused, so this is the GEMM alone
            fl = api.ACCR_MM_REUSE_SPLIT
            api.accr_matmul_nest(at, bt, ct, mode=mode, flags=fl, stream=stream)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(reps):
                api.accr_matmul_nest(at, bt, ct, mode=mode, flags=fl, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            gms = e0.elapsed_time(e1) / reps
            r["reuse_split_ms"] = round(gms, 4)
            r["reuse_split_tensor_tflops"] = round(3 * flops / (gms * 1e-3) / 1e12, 2)
            r["reuse_split_frac_of_bf16_peak"] = round(3 * flops / (gms * 1e-3) / 1e12 / float(peaks["bf16_tflops"]), 4)
        out[mode] = r
    fp32 = measure_fp32_peak(dev)
    out["fp32_peak"] = fp32
    for mode in ("simt", "serial"):
        out[mode]["frac_of_fp32_peak"] = round(out[mode]["tflops"] / fp32["tflops"], 4)
    return out


def measure_fp32_peak(dev, rounds=1 << 15, reps=5):
    """Measured FP32 FMA peak (the SIMT nest's roofline): 16 independent FMA
    chains per thread, 4 CTAs of 256 threads per SM, issued as scalar
    instructions and as packed pairs; the peak is the larger rate."""
    import torch
    from paper_1412_1127_gb300 import api
    ctas = 4 * torch.cuda.get_device_properties(dev).multi_processor_count
    sink = torch.empty(256 * ctas, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def rate(fn, fmas):
        for _ in range(3):
            fn(ctas, rounds, sink, stream=stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn(ctas, rounds, sink, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        return 2.0 * fmas * 256 * ctas * rounds / (ms * 1e-3) / 1e12, ms

    scalar, ms_s = rate(api.accr_probe_fma, 16)
    packed, ms_p = rate(api.accr_probe_fma_packed, 32)
    return {"tflops": round(max(scalar, packed), 2), "scalar_tflops": round(scalar, 2),
            "packed_tflops": round(packed, 2), "ms": round(ms_s, 4), "ms_packed": round(ms_p, 4),
            "probe": "%d CTAs x 256 threads x %d rounds x 16 chains (scalar FMA, or packed pairs)" % (ctas, rounds)}


def measure_small_region(dev, n=1 << 20, reps=100):
    """One region of 2^20 int32 U[-1000, 1000] with reduction(+:s) into a
    64-bit variable and reduction(max:m): device time per region, back to
    back, with the inputs warm in L2, and with L2 flushed before each region
    (a 2 x L2 write; its own time, measured alone, is subtracted).  A 4 MiB
    region takes a few microseconds, less than one host call, so the calls
    are queued behind a long FMA probe launch and one event pair brackets
    all of them; the host time per call is reported beside it."""
    import torch
    from paper_1412_1127_gb300 import api, inputs
    x = torch.from_numpy(inputs.scalar_i32_small(n)).to(dev)
    s_ = torch.empty(1, dtype=torch.int64, device=dev)
    m_ = torch.empty(1, dtype=torch.int32, device=dev)
    cls = [api.clause("add", s_), api.clause("max", m_)]
    stream = torch.cuda.current_stream(dev)
    l2 = int(getattr(torch.cuda.get_device_properties(dev), "L2_cache_size", 0) or (128 << 20))
    flush = torch.empty(2 * l2 // 4, dtype=torch.int32, device=dev)
    ctas = 4 * torch.cuda.get_device_properties(dev).multi_processor_count
    sink = torch.empty(256 * ctas, dtype=torch.float32, device=dev)

    def queued(body):
        for _ in range(3):
            body()
        torch.cuda.synchronize()
        b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        b0.record(stream)
        api.accr_probe_fma(ctas, 1 << 18, sink, stream=stream)  # the GPU is busy while the host queues
        b1.record(stream)
        e0.record(stream)
        t0 = time.perf_counter()
        for _ in range(reps):
            body()
        host_s = time.perf_counter() - t0
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) * 1e3 / reps, host_s * 1e6 / reps, host_s * 1e3 < b0.elapsed_time(b1)

    region = lambda: api.accr_reduce(x, cls, stream=stream)
    warm, host_us, ahead = queued(region)
    flushed, _, ahead2 = queued(lambda: (flush.fill_(1), region()))
    flush_only, _, ahead3 = queued(lambda: flush.fill_(1))
    cold = flushed - flush_only
    # the C call alone (arguments marshalled once), and the launch floor: the
    # same call on an empty region, and an empty kernel, back to back
    arr, keep = api._clauses(cls)
    L, xp, sp = api.lib(), x.data_ptr(), stream.cuda_stream
    c_call = lambda: L.accr_reduce(xp, n, api.ACCR_I32, arr, 2, 0, sp)
    warm_c, host_c_us, ahead4 = queued(c_call)
    empty_region, _, ahead5 = queued(lambda: L.accr_reduce(xp, 0, api.ACCR_I32, arr, 2, 0, sp))
    empty_kernel, _, ahead6 = queued(lambda: torch.cuda._sleep(0))
    return {"workload": "one region, 2^20 int32, + (int64 variable) and max in one pass",
            "warm": {"us_per_region": round(warm, 2), "gbs": round(4.0 * n / (warm * 1e-6) / 1e9, 1)},
            "warm_c_call": {"us_per_region": round(warm_c, 2), "gbs": round(4.0 * n / (warm_c * 1e-6) / 1e9, 1)},
            "l2_flushed": {"us_per_region": round(cold, 2), "gbs": round(4.0 * n / (cold * 1e-6) / 1e9, 1)},
            "host_us_per_call": round(host_us, 2), "host_us_per_c_call": round(host_c_us, 2),
            "empty_region_us": round(empty_region, 2), "empty_kernel_us": round(empty_kernel, 2),
            "queued_ahead": bool(ahead and ahead2 and ahead3 and ahead4 and ahead5 and ahead6),
            "note": "back-to-back launches on one stream, queued behind a long probe launch; empty_region is "
                    "accr_reduce over n = 0 (the entry point's launch floor), empty_kernel a kernel that "
                    "does nothing (the stream's launch cadence); host_us_per_call goes through the Python "
                    "binding, host_us_per_c_call calls the C entry point with its arguments built once"}


def measure_rows(dev, rows=65536, cols=4096, steps=10, warmup=3):
    """The row nest: row sum and row max of a rows x cols float U(-1,1)
    matrix in one pass (two clauses), GB/s of the matrix read once."""
    import torch
    from paper_1412_1127_gb300 import api, inputs
    A = inputs.uniform_matrix(rows, cols)
    At = torch.from_numpy(A).to(dev)
    s = torch.empty(rows, dtype=torch.float32, device=dev)
    m = torch.empty(rows, dtype=torch.float32, device=dev)
    cls = [api.clause("add", s), api.clause("max", m)]
    stream = torch.cuda.current_stream(dev)
    for _ in range(max(warmup, 3)):
        api.accr_rowreduce(At, cls, stream=stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        api.accr_rowreduce(At, cls, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    nbytes = rows * cols * 4
    peaks, kind = measured_peaks()
    ok_max = bool(torch.equal(m, At.amax(dim=1)))
    form = "split-row (32 KiB chunks, an even run per CTA, CTA merge)" if cols * 4 >= (256 << 10) else "one warp per row"
    return {"workload": "row sum + row max (one pass), %d x %d float U(-1,1)" % (rows, cols), "form": form,
            "ms": round(ms, 4), "gbs": round(nbytes / (ms * 1e-3) / 1e9, 1),
            "frac_of_hbm": round(nbytes / (ms * 1e-3) / 1e9 / float(peaks["hbm_gbs"]), 4),
            "row_max_equals_torch_amax": ok_max}


def measure_rows_all(dev, rows=65536, steps=10, warmup=3):
    """The 65536 x 4096 row nest, plus a few long rows (4 x 2^24 and
    64 x 2^22, the split-row form) under the same name."""
    import torch
    out = measure_rows(dev, rows, 4096, steps, warmup)
    out["long_rows"] = []
    for r, c in [(4, 1 << 24), (64, 1 << 22)]:
        out["long_rows"].append(measure_rows(dev, r, c, steps, warmup))
        torch.cuda.empty_cache()
    return out


def run_rows(args):
    import torch
    torch.cuda.set_device(0)
    print(json.dumps(measure_rows_all(torch.device("cuda", 0), args.rows_m, args.steps, args.warmup)), flush=True)
    return 0


def device_ms(fn, stream, reps):
    """Device time per call of fn, calls back to back on `stream` (CUDA
    events around all of them; the host queues ahead of the GPU)."""
    import torch
    for _ in range(3):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def measure_patterns(dev, reps=10, which=("f1", "f2", "f3", "f4")):
    """The paper's two-level host merge against the single-pass merge (f1),
    the SRAD pattern fused and unfused (f2), the BFS convergence flag in its
    three forms (f3), and k-nearest (f4); `which` selects among them."""
    import torch
    from paper_1412_1127_gb300 import api, inputs
    stream = torch.cuda.current_stream(dev)
    out = {}

    def wall(fn, k):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(k):
            t0 = time.perf_counter()
            fn()
            ts.append(time.perf_counter() - t0)
        return float(np.median(ts)) * 1e3

    # f1: result of one region available on the host
    f1 = {}
    for lg in ((20, 24, 28) if "f1" in which else ()):
        x = torch.from_numpy(inputs.full_range_i32(1 << lg, salt=lg)).to(dev)
        sd = torch.empty(1, dtype=torch.int64, device=dev)
        sh = torch.empty(1, dtype=torch.int64).pin_memory()

        def single():
            # the last CTA writes the variable straight into pinned host memory
            api.accr_reduce(x, [api.clause("add", sh)], flags=api.ACCR_SYNC, stream=stream)

        def two_level():
            api.accr_reduce(x, [api.clause("add", sh)], flags=api.ACCR_TWO_LEVEL_HOST, stream=stream)

        a, b = wall(single, reps), wall(two_level, reps)
        f1["2^%d" % lg] = {"single_pass_ms": round(a, 4), "two_level_host_ms": round(b, 4)}
        del x
    if f1:
        out["f1_two_level_vs_single_pass"] = f1

    # f2: SRAD pattern (statistics, then the standardised array)
    f2 = {}
    for lg in ((22, 28) if "f2" in which else ()):
        n = 1 << lg
        x = torch.from_numpy(inputs.normal(n, np.float32, salt=lg)).to(dev)
        y = torch.empty_like(x)
        st = torch.empty(2, dtype=torch.float64, device=dev)
        r = {}
        for form, fl in [("fused", 0), ("unfused", api.ACCR_UNFUSED), ("two_level_host", api.ACCR_TWO_LEVEL_HOST)]:
            ms = wall(lambda: (api.accr_standardize(x, y, st, flags=fl, stream=stream), stream.synchronize()), reps)
            r[form] = {"ms": round(ms, 4), "gbs_3_passes": round(12.0 * n / (ms * 1e-3) / 1e9, 1)}
            if form != "two_level_host":  # (the host form waits for the host inside the call)
                dev_ms = device_ms(lambda: api.accr_standardize(x, y, st, flags=fl, stream=stream), stream, reps)
                r[form]["device_ms"] = round(dev_ms, 4)
                r[form]["device_gbs_3_passes"] = round(12.0 * n / (dev_ms * 1e-3) / 1e9, 1)
        f2["n=2^%d" % lg] = r
        del x, y
    if f2:
        out["f2_srad_pattern"] = f2
    if "f3" in which:
        out["f3_bfs_convergence"] = measure_bfs(dev, api, inputs, stream, wall)
    if "f4" in which:
        out["f4_nearest_k5"] = measure_nearest(dev, api, inputs, stream, reps)
    return out


def measure_bfs(dev, api, inputs, stream, wall):
    import torch

    # f3: BFS convergence loop on a 1024 x 1024 grid, 62 % open
    g = inputs.rng(23, 1)
    grid = (g.random((1024, 1024)) < 0.62).astype(np.uint8)
    src = 512 * 1024 + 512
    grid.flat[src] = 1
    gt = torch.from_numpy(grid).to(dev)
    dist = torch.empty((1024, 1024), dtype=torch.int32, device=dev)
    f3 = {}
    for mode in ["reduce", "guarded", "persistent"]:
        lv = [0]

        def run():
            lv[0] = api.accr_grid_bfs(gt, src, dist, mode=mode, stream=stream)
        ms = wall(run, 3)
        f3[mode] = {"ms": round(ms, 3), "levels": lv[0], "us_per_level": round(ms * 1e3 / max(lv[0], 1), 2)}
    return f3


def measure_nearest(dev, api, inputs, stream, reps):
    import torch
    n = 1 << 26
    pts = torch.from_numpy((inputs.rng(21, 5).random((n, 2), dtype=np.float32) * 100)).to(dev)
    idx = torch.empty(5, dtype=torch.int64, device=dev)
    d2 = torch.empty(5, dtype=torch.float32, device=dev)
    for _ in range(3):
        api.accr_nearest_k(pts, 41.5, 58.25, 5, idx, d2, stream=stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        api.accr_nearest_k(pts, 41.5, 58.25, 5, idx, d2, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    return {"n": n, "ms": round(ms, 4), "gbs": round(8.0 * n / (ms * 1e-3) / 1e9, 1)}


def run_patterns(args):
    import torch
    torch.cuda.set_device(0)
    which = tuple(w.strip() for w in args.patterns.split(",") if w.strip())
    print(json.dumps(measure_patterns(torch.device("cuda", 0), which=which)), flush=True)
    return 0


def run_matmul(args):
    import torch
    torch.cuda.set_device(0)
    print(json.dumps(measure_matmul(torch.device("cuda", 0), args.len)), flush=True)
    return 0


def run_batched(args):
    import torch
    import __graft_entry__
    torch.cuda.set_device(0)
    r = measure_batched(torch.device("cuda", 0), args.steps, args.warmup, args.regions, args.tune,
                        hi=args.batched_hi)
    print(json.dumps(r), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="accr", choices=["accr", "reference"])
    ap.add_argument("--workload", default="scalar", choices=["scalar", "batched", "served", "matmul", "rows", "patterns"])
    ap.add_argument("--len", type=int, default=4096, help="matmul: LEN")
    ap.add_argument("--rows-m", type=int, default=65536, help="rows: number of rows (4096 columns)")
    ap.add_argument("--patterns", default="f1,f2,f3,f4", help="patterns: which of f1,f2,f3,f4 to run")
    ap.add_argument("--served-seconds", type=float, default=10.0)
    ap.add_argument("--rate", type=float, default=50000.0)
    ap.add_argument("--no-extra", action="store_true",
                    help="scalar workload only (skip the batched and served sub-measurements)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--regions", type=int, default=20000, help="regions of the batched workload")
    ap.add_argument("--batched-hi", type=int, default=1 << 20,
                    help="batched workload: largest region length (2^20, or 2^17 for the second mix)")
    ap.add_argument("--tune", action="store_true", help="batched: autotune the split first")
    ap.add_argument("--sweep", action="store_true", help="served: sweep the offered rate to saturation")
    ap.add_argument("--n", type=int, default=N_SCALAR,
                    help="elements per region (default 2^28; smaller only for profiling captures)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    import __graft_entry__
    __graft_entry__.build()
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "served":
        return run_served(args)
    if args.workload == "matmul":
        return run_matmul(args)
    if args.workload == "rows":
        return run_rows(args)
    if args.workload == "patterns":
        return run_patterns(args)
    return run_scalar(args)


if __name__ == "__main__":
    sys.exit(main())
