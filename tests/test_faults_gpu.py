"""Failure detection without a GPU fault: faults are made on the host
(injected allocation, launch and admission failures) or by a bounded wait that
runs out; each is reported as a status code and the context stays usable."""
import numpy as np
import pytest
import torch

import oracle
from paper_1412_1127_gb300 import api, inputs
from paper_1412_1127_gb300._native import (ACCR_EBUDGET, ACCR_ECUDA, ACCR_ENOMEM, ACCR_ETIMEDOUT,
                                           AccrError)

pytestmark = pytest.mark.gpu


def _region():
    x = inputs.full_range_i32((1 << 20) + 3, salt=31)
    return x, torch.from_numpy(x).cuda()


def test_injected_allocation_failure_then_recovery():
    x, xt = _region()
    s = torch.empty(1, dtype=torch.int64, device="cuda")
    fresh = torch.cuda.Stream()              # no scratch yet on this stream
    api.accr_fault_inject(api.ACCR_FAULT_ALLOC, 1)
    with pytest.raises(AccrError) as e:
        api.accr_reduce(xt, [api.clause("add", s)], stream=fresh)
    assert e.value.code == ACCR_ENOMEM
    api.accr_reduce(xt, [api.clause("add", s)], stream=fresh, flags=api.ACCR_SYNC)
    assert int(s.item()) == int(oracle.reduce(x, "add", "i64"))


def test_injected_launch_failure_leaves_output_untouched():
    x, xt = _region()
    s = torch.full((1,), 12345, dtype=torch.int64, device="cuda")
    api.accr_fault_inject(api.ACCR_FAULT_LAUNCH, 1)
    before = api.accr_launch_count()
    with pytest.raises(AccrError) as e:
        api.accr_reduce(xt, [api.clause("add", s)], flags=api.ACCR_SYNC)
    assert e.value.code == ACCR_ECUDA and "injected" in str(e.value)
    assert api.accr_launch_count() == before
    assert int(s.item()) == 12345
    api.accr_reduce(xt, [api.clause("add", s)], flags=api.ACCR_SYNC)
    assert int(s.item()) == int(oracle.reduce(x, "add", "i64"))
    api.accr_fault_inject(api.ACCR_FAULT_LAUNCH, 0)


def test_served_batch_failure_is_reported_per_request():
    x, xt = _region()
    srv = api.Server(1 << 30, nstreams=1, max_batch=64)
    api.accr_fault_inject(api.ACCR_FAULT_LAUNCH, 1)   # the next batch launch fails
    t = srv.submit(xt, [api.clause("add", torch.empty(1, dtype=torch.int64, device="cuda"))])
    with pytest.raises(AccrError) as e:
        srv.poll(t)
    assert e.value.code == ACCR_ECUDA
    t2 = srv.submit(xt, [api.clause("add", torch.empty(1, dtype=torch.int64, device="cuda"))])
    rc, vals, _ = srv.poll(t2)
    assert api.decode(vals[0], torch.int64) == oracle.reduce(x, "add", "i64")
    api.accr_fault_inject(api.ACCR_FAULT_ADMIT, 1)
    with pytest.raises(AccrError) as e:
        srv.submit(xt, [api.clause("add", torch.empty(1, dtype=torch.int64, device="cuda"))])
    assert e.value.code == ACCR_EBUDGET
    srv.destroy()


def test_bounded_wait_runs_out_and_context_survives():
    assert api.accr_selftest_wait_timeout(2000) == ACCR_ETIMEDOUT
    assert "bounded wait" in api.accr_last_error()
    x, xt = _region()
    m = torch.empty(1, dtype=torch.int32, device="cuda")
    api.accr_reduce(xt, [api.clause("max", m)], flags=api.ACCR_SYNC)
    assert int(m.item()) == int(x.max())
    a = inputs.small_int_matrix(64, 64)
    at = torch.from_numpy(a).cuda()
    c = torch.empty_like(at)
    api.accr_matmul_nest(at, at, c, mode="bf16x3", flags=api.ACCR_SYNC)
    assert np.array_equal(c.cpu().numpy(), (a.astype(np.int64) @ a.astype(np.int64)).astype(np.float32))
