"""The multi-rank path of bench.py on CPU: two gloo ranks on 127.0.0.1.

Every rank times its own independent copy of the workload; the reported time
is the slowest rank's and the value counts the units of all ranks.  The
reference arm runs on rank 0 only; other ranks exit without work."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    bench.init_ranks(world, "gloo")
    r, w, local = bench.dist_env()
    assert (r, w) == (rank, world)
    bench.barrier(world)
    my_ms = 10.0 * (rank + 1)              # the slower rank sets the time
    ms = bench.max_over_ranks(my_ms, world)
    rate = bench.whole_job_rate(1000.0, world, ms * 1e-3)
    import torch.distributed as dist
    dist.destroy_process_group()
    q.put((rank, ms, rate))


def test_two_gloo_ranks_take_the_max():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    ps = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, rate in res:
        assert ms == 20.0
        assert rate == pytest.approx(1000.0 * 2 / 0.020)


def test_reference_arm_other_ranks_exit_without_work(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        gpus, steps, warmup = 2, 1, 0
    assert bench.run_reference(A()) == 0
    assert capsys.readouterr().out == ""
