"""The served request loop on the GPU: results against the oracle, the same
bits alone and in a mix, admission by budget, poll semantics, replay."""
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
