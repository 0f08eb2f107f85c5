"""The bounds-checked debug library (libaccr_debug.so, -DACCR_DEBUG) runs the
main workloads with no violation.

In a debug build every global store of the row, batched-region, k-nearest and
tensor-core kernels checks its index against the bound the host computed; a
failed check does not trap, it is counted and the store skipped.  The child
process below loads the debug library through ACCR_LIBRARY, runs each path at
sizes that take its distinctive branches (the one-CTA and multi-CTA reduce,
split and warp-per-row rows, tiled and warp regions with three clauses, the
sampled bound of the k-nearest scan, ragged GEMM tiles), checks each result
loosely against plain PyTorch (exact parity is the other tests' job), and
prints what accr_debug_report counted.
"""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, math
import torch
from paper_1412_1127_gb300 import api, _native
assert _native.LIB_PATH.endswith("libaccr_debug.so"), _native.LIB_PATH
g = torch.Generator(device="cpu").manual_seed(1127)
dev = "cuda"
bad = []

def close(what, got, want, rel):
    got, want = float(got), float(want)
    if not abs(got - want) <= rel * max(1.0, abs(want)):
        bad.append("%s: %r vs %r" % (what, got, want))

_, _, checked = api.accr_debug_report(clear=True)

# one region: a single CTA and a full grid
for n in (1000, (1 << 24) + 37):
    x = torch.rand(n, generator=g).to(dev)
    s = torch.zeros(1, device=dev); m = torch.zeros(1, device=dev)
    api.accr_reduce(x, [api.clause("+", s), api.clause("max", m)], flags=api.ACCR_SYNC)
    close("reduce sum %d" % n, s.item(), x.double().sum().item(), 1e-5)
    close("reduce max %d" % n, m.item(), x.max().item(), 0.0)

# rows: warp per row, and rows long enough to be split over CTAs
for rows, cols in ((300, 1000), (4, (1 << 20) + 5), (3, (1 << 18) + 1)):
    A = torch.randn(rows, cols, generator=g).to(dev)
    s = torch.zeros(rows, device=dev); m = torch.zeros(rows, device=dev)
    api.accr_rowreduce(A, [api.clause("+", s), api.clause("min", m)], flags=api.ACCR_SYNC)
    want = A.double().sum(1).cpu()
    for i in range(rows):
        close("row sum %dx%d[%d]" % (rows, cols, i), s[i].item(), want[i].item(), 1e-4 * math.sqrt(cols))
    if not torch.equal(m, A.min(1).values):
        bad.append("row min %dx%d" % (rows, cols))

# batched regions: tiled and warp regions, one with three clauses
lens = [5, 100, 4096, 70000, 1 << 20, (1 << 21) + 3, 0, 31]
xs = [torch.randint(-1000, 1000, (n,), generator=g, dtype=torch.int64).to(dev) for n in lens]
outs = torch.zeros(len(lens), 3, dtype=torch.int64, device=dev)
regs = []
for i, x in enumerate(xs):
    cls = [api.clause("+", outs[i, 0:1])]
    if i % 2 == 0:
        cls += [api.clause("max", outs[i, 1:2]), api.clause("min", outs[i, 2:3])]
    regs.append((x, cls, 0))
api.accr_batch_reduce(regs, flags=api.ACCR_SYNC)
o = outs.cpu()
for i, x in enumerate(xs):
    xc = x.cpu()
    if o[i, 0].item() != int(xc.sum()):
        bad.append("batch sum %d" % i)
    if i % 2 == 0 and xc.numel() and (o[i, 1].item() != int(xc.max()) or o[i, 2].item() != int(xc.min())):
        bad.append("batch max/min %d" % i)

# k nearest: below and above the size at which the sampled bound is used
for n in (5000, (1 << 22) + 3):
    pts = torch.rand(n, 2, generator=g).to(dev)
    for k in (5, 12):
        idx = torch.empty(k, dtype=torch.int64, device=dev); d2 = torch.empty(k, device=dev)
        api.accr_nearest_k(pts, 0.25, 0.75, k, idx, d2, flags=api.ACCR_SYNC)
        dd = (pts[:, 0] - 0.25) ** 2 + (pts[:, 1] - 0.75) ** 2
        want = torch.topk(dd, k, largest=False).values
        if not torch.allclose(d2, want, rtol=1e-5, atol=1e-7):
            bad.append("nearest n=%d k=%d" % (n, k))

# tensor-core BF16x3 nest with ragged edge tiles
for L in (200, 300):
    a = torch.randn(L, L, generator=g).to(dev); b = torch.randn(L, L, generator=g).to(dev)
    c = torch.zeros(L, L, device=dev)
    api.accr_matmul_nest(a, b, c, mode="bf16x3", flags=api.ACCR_SYNC)
    want = (a.double() @ b.double()).float()
    err = (c - want).abs().max().item()
    if not err <= 1e-3 * math.sqrt(L):
        bad.append("bf16x3 %d: max error %g" % (L, err))

torch.cuda.synchronize()
v, site, _ = api.accr_debug_report(clear=True)
print(json.dumps({"checked": checked, "violations": v, "site": site, "bad": bad}))
"""


@pytest.mark.gpu
def test_debug_build_runs_the_workloads_without_violations():
    from paper_1412_1127_gb300 import build
    build.build(debug=True)
    env = dict(os.environ, ACCR_LIBRARY=build.DEBUG_LIB, PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-4000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["checked"] is True, "the debug library was built without -DACCR_DEBUG"
    assert out["bad"] == [], out["bad"]
    assert out["violations"] == 0, "first failing site %d" % out["site"]
