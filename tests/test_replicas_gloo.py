"""Multi-process path of the benchmark on CPU (gloo, world size 2): the path
runs as independent replicas, so the only cross-rank step is the timing: every
rank receives the slowest rank's step time, and the whole-job rate counts the
units of all ranks over it.  A rank that never joins ends the others' wait
with an error after the process-group timeout."""
import datetime
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q, step_ms):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=30))
    try:
        dist.barrier()
        ms = bench.slowest_rank_ms(step_ms[rank], dist, torch.device("cpu"))
        q.put((rank, ms, bench.whole_job_rate(world, 2.7e8 * 200, ms)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _lonely_rank(port, q):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    try:
        dist.init_process_group("gloo", rank=0, world_size=2, timeout=datetime.timedelta(seconds=3))
        bench.slowest_rank_ms(1.0, dist, torch.device("cpu"))
        q.put("returned")
    except Exception as e:          # the missing rank surfaces as an error, not a hang
        q.put(type(e).__name__)


def test_slowest_rank_and_job_rate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    step_ms = [81.5, 108.25]
    ps = [ctx.Process(target=_rank_main, args=(r, 2, port, q, step_ms)) for r in range(2)]
    for p in ps:
        p.start()
    got = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[1] for g in got] == [108.25, 108.25]
    rate = 2 * 2.7e8 * 200 / 108.25e-3 / 1e9
    assert all(abs(g[2] - rate) <= 1e-12 * rate for g in got)


def test_one_rank_alone():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.slowest_rank_ms(12.5, None, None) == 12.5
    assert bench.whole_job_rate(1, 1e9, 1000.0) == pytest.approx(1.0)


def test_missing_rank_ends_in_an_error():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    p = ctx.Process(target=_lonely_rank, args=(free_port(), q))
    p.start()
    out = q.get(timeout=120)
    p.join(timeout=60)
    assert out != "returned"
