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
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
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
    line = {"impl": "reference", "metric": "reduction GB/s (% of HBM peak)", "value": round(v, 4),
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
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
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

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    # timed region: K steps, CUDA events on the launching stream, per-region events
    evs = [[[torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)] for _ in range(R)]
           for _ in range(args.steps)]
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    l0 = api.accr_launch_count()
    start.record(stream)
    for k in range(args.steps):
        step(evs[k])
    stop.record(stream)
    torch.cuda.synchronize()
    launches = api.accr_launch_count() - l0
    barrier()
    clk = clocks.stop()
    ms = start.elapsed_time(stop)
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    per_region_ms = [sum(evs[k][i][0].elapsed_time(evs[k][i][1]) for k in range(args.steps)) / args.steps
                     for i in range(R)]
    ms_step = ms / args.steps
    value = bytes_step * world / (ms_step * 1e-3) / 1e9

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

        def e2e_step():
            for kind in ("i32", "f32", "f64"):
                devin[kind].copy_(pinned[kind], non_blocking=True)
            step()
            for i, o in enumerate(outs):
                res_host[i:i + 1].view(torch.uint8)[: o.element_size()].copy_(
                    o.view(torch.uint8), non_blocking=True)
            torch.cuda.current_stream(dev).synchronize()

        e2e_step()
        ek = max(2, min(args.steps, 5))
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
               "seconds": round(dt, 2)}

    if rank == 0:
        line = {
            "metric": "reduction GB/s (% of HBM peak)",
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
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="accr", choices=["accr", "reference"])
    ap.add_argument("--workload", default="scalar", choices=["scalar"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--n", type=int, default=N_SCALAR,
                    help="elements per region (default 2^28; smaller only for profiling captures)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    import __graft_entry__
    __graft_entry__.build()
    return run_scalar(args)


if __name__ == "__main__":
    sys.exit(main())
