"""The served request loop on the GPU: results against the oracle, the same
bits alone and in a mix, admission by budget, poll semantics, replay."""
import ctypes
import math
import time

import numpy as np
import pytest
import torch

import oracle
from paper_1412_1127_gb300 import api, inputs
from paper_1412_1127_gb300._native import ACCR_EAGAIN, ACCR_EBUDGET, ACCR_ETIMEDOUT, AccrError
from tolerances import TOL_F32_COMP, same_bits

pytestmark = pytest.mark.gpu

TD = {"i32": torch.int32, "i64": torch.int64, "f32": torch.float32, "f64": torch.float64}


@pytest.fixture(scope="module")
def pools():
    n = 1 << 24
    host = {"f32": inputs.normal(n, np.float32, salt=77),
            "i32": inputs.full_range_i32(n, salt=78),
            "i64": inputs.uniform_i64(n, -(1 << 40), 1 << 40, salt=79)}
    dev = {k: torch.from_numpy(v).cuda() for k, v in host.items()}
    return host, dev


CLAUSES = {"f32": [("add", "f32")], "i32": [("add", "i64"), ("max", "i32")], "i64": [("add", "i64"), ("bxor", "i64")]}


def make_requests(pools, count, seed, lo=1, hi=1 << 20):
    host, dev = pools
    g = np.random.default_rng(seed)
    reqs = []
    for k in range(count):
        t = ["f32", "i32", "i64"][k % 3]
        n = int(np.exp(g.uniform(np.log(lo), np.log(hi))))
        off = int(g.integers(0, host[t].size - n))
        cls = [api.clause(op, torch.empty(1, dtype=TD[a], device="cuda")) for op, a in CLAUSES[t]]
        reqs.append((t, off, n, cls))
    return reqs


def region_of(pools, r):
    t, off, n, cls = r
    return (pools[1][t][off:off + n], cls, api.ACCR_COMPENSATED if t == "f32" else 0)


def check_result(pools, r, vals):
    t, off, n, cls = r
    x = pools[0][t][off:off + n]
    for (op, acc), v in zip(CLAUSES[t], vals):
        got = api.decode(v, TD[acc])
        if t == "f32":
            truth = oracle.truth_sum(x)
            assert abs(float(got) - truth) <= TOL_F32_COMP * max(abs(truth), 0.1 * math.sqrt(max(n, 1)))
        else:
            assert got == oracle.reduce(x, op, acc), (t, op, n)


def test_served_results_and_mix_determinism(pools):
    reqs = make_requests(pools, 600, seed=1)
    srv = api.Server(1 << 34, nstreams=4, max_batch=256)
    tickets = [srv.submit(*region_of(pools, r)) for r in reqs]
    mixed = [srv.poll(t)[1] for t in tickets]
    for r, v in zip(reqs, mixed):
        check_result(pools, r, v)
    # each region alone (idle server) gives the same bits as in the mix
    for k in [0, 1, 2, 7, 100, 333, 599]:
        t = srv.submit(*region_of(pools, reqs[k]))
        alone = srv.poll(t)[1]
        assert alone == mixed[k], k
    srv.destroy()


def test_admission_by_budget_and_errors(pools):
    reqs = make_requests(pools, 60, seed=2, lo=1 << 16, hi=1 << 20)
    biggest = max(r[2] * (4 if r[0] != "i64" else 8) for r in reqs)
    srv = api.Server(biggest, nstreams=2, max_batch=8)   # at most ~one region in flight
    tickets = [srv.submit(*region_of(pools, r)) for r in reqs]
    for r, t in zip(reqs, tickets):
        check_result(pools, r, srv.poll(t)[1])
    host, dev = pools
    with pytest.raises(AccrError) as e:
        srv.submit(dev["f32"][: biggest // 4 + 1000], [api.clause("add", torch.empty(1, device="cuda"))])
    assert e.value.code == ACCR_EBUDGET
    rc, vals, _ = srv.poll(123456789, timeout_us=0)
    assert rc == ACCR_EAGAIN and vals is None
    rc, vals, _ = srv.poll(123456789, timeout_us=2000)
    assert rc == ACCR_ETIMEDOUT
    with pytest.raises(AccrError):
        srv.submit(dev["f32"][:10], [api.clause("bxor", torch.empty(1, device="cuda"))])
    srv.destroy()


def test_replay_server_and_plain_agree(pools):
    reqs = make_requests(pools, 400, seed=3)
    regions = [region_of(pools, r) for r in reqs]
    arrivals = inputs.poisson_arrivals(20000, len(regions), salt=1)
    srv = api.Server(1 << 34, nstreams=4, max_batch=512)
    res_s = srv.replay(regions, arrivals)
    srv.destroy()
    res_p = api.accr_server_replay(None, regions, arrivals, plain=True)
    for k, r in enumerate(reqs):
        vs = list(res_s[k].value[: res_s[k].nclauses])
        check_result(pools, r, vs)
        if r[0] != "f32":
            assert vs == list(res_p[k].value[: res_p[k].nclauses])
        lat = res_s[k].done_ns - res_s[k].submit_ns
        assert 0 < lat < 5e9


@pytest.fixture(scope="module")
def big_pools():
    """Pools large enough for regions of up to 2^26 elements at random offsets."""
    n = 1 << 27
    host = {"f32": inputs.normal(n, np.float32, salt=87),
            "i32": inputs.full_range_i32(n, salt=88),
            "i64": inputs.uniform_i64(n, -(1 << 40), 1 << 40, salt=89)}
    dev = {k: torch.from_numpy(v).cuda() for k, v in host.items()}
    return host, dev


def _check_all(pools, reqs, values):
    """Every served result against the oracle (host threads; ctypes releases the GIL)."""
    import concurrent.futures as cf
    with cf.ThreadPoolExecutor(max_workers=16) as ex:
        list(ex.map(lambda rv: check_result(pools, *rv), zip(reqs, values)))


@pytest.mark.slow
def test_served_loop_at_full_request_shapes(big_pools):
    """2,000 requests with lengths log-uniform on [2^8, 2^26] over float,
    int32 and int64 (the served workload's shapes): regions up to 1,024 of the
    loop's 512 KiB tiles, batches too large to pass their plan in the kernel's
    parameters.  Every result against the oracle: integers bit-exact, float
    sums within the compensated tolerance of the exact sum; then a second
    pass of a subset through a fresh server gives the same bits."""
    reqs = make_requests(big_pools, 2000, seed=11, lo=1 << 8, hi=1 << 26)
    assert max(r[2] for r in reqs) > (1 << 25)
    srv = api.Server(64 << 30, nstreams=4, max_batch=1024)
    tickets = [srv.submit(*region_of(big_pools, r)) for r in reqs]
    vals = [srv.poll(t)[1] for t in tickets]
    srv.destroy()
    _check_all(big_pools, reqs, vals)
    srv = api.Server(64 << 30, nstreams=2, max_batch=64)
    for k in range(0, 2000, 97):
        t = srv.submit(*region_of(big_pools, reqs[k]))
        assert srv.poll(t)[1] == vals[k], k
    srv.destroy()


def test_admission_budget_binds_and_holds(pools):
    """Bytes in flight, reconstructed from each result's launch and done times
    (a batch's requests share both), never exceed the budget, and the budget
    binds: the requests' total is many times the budget, and the peak comes
    within one region of it."""
    reqs = make_requests(pools, 400, seed=12, lo=1 << 16, hi=1 << 22)
    nbytes = [r[2] * (8 if r[0] == "i64" else 4) for r in reqs]
    budget = 4 * max(nbytes)
    assert sum(nbytes) > 10 * budget
    srv = api.Server(budget, nstreams=4, max_batch=64)
    tickets = [srv.submit(*region_of(pools, r)) for r in reqs]
    res = []
    for r, t in zip(reqs, tickets):
        rc, v, full = srv.poll(t)
        check_result(pools, r, v)
        res.append((full.launch_ns, full.done_ns))
    srv.destroy()
    events = []
    for (lo, hi), b in zip(res, nbytes):
        assert 0 < lo <= hi
        events += [(lo, 1, b), (hi, 0, -b)]       # at equal times, ends first
    events.sort()
    cur = peak = 0
    for _, _, d in events:
        cur += d
        peak = max(peak, cur)
        assert cur <= budget, (cur, budget)
    assert cur == 0
    assert peak >= budget - max(nbytes), (peak, budget)


def test_submit_copies_prior_values(pools):
    """accr_submit keeps its own copy of each clause's prior value: overwriting
    it right after the call does not change the result."""
    host, dev = pools
    x = dev["i32"][1000:1000 + 300000]
    keep = []
    cls = [api.clause("add", torch.empty(1, dtype=torch.int64, device="cuda"), init=123456789),
           api.clause("max", torch.empty(1, dtype=torch.int32, device="cuda"), init=2 ** 31 - 5)]
    srv = api.Server(1 << 30, nstreams=1, max_batch=4)
    tickets = []
    for _ in range(8):
        g = api._region_desc(x, cls, 0, keep)
        t = ctypes.c_uint64()
        assert api.lib().accr_submit(srv.handle, ctypes.byref(g), ctypes.byref(t)) == 0
        for v in keep:               # the caller reuses its variables at once
            v.value = -1
        tickets.append(t.value)
    xs = host["i32"][1000:1000 + 300000]
    for t in tickets:
        vals = srv.poll(t)[1]
        assert api.decode(vals[0], torch.int64) == oracle.reduce(xs, "add", "i64", init=123456789)
        assert api.decode(vals[1], torch.int32) == oracle.reduce(xs, "max", "i32", init=2 ** 31 - 5)
    srv.destroy()
