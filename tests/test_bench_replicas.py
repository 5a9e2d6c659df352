"""The multi-rank (replica) bookkeeping of bench.py on the CPU: two gloo
ranks with different step times must agree on the slowest rank's time, and
the job's throughput counts every rank's units over that time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ws, r, local = bench.dist_env()
        t = bench.max_over_ranks([1.0 + rank, 10.0 - rank], torch.device("cpu"))
        out[rank] = (ws, r, local, t, bench.job_value(600, ws, t[0]))
    finally:
        dist.destroy_process_group()


def test_replica_timing_is_max_over_ranks():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    for r in (0, 1):
        ws, rank, local, t, value = res[r]
        assert (ws, rank, local) == (2, r, r)
        assert t == [2.0, 10.0]               # slowest rank, element-wise
        assert value == pytest.approx(2 * 600 / 2.0)


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks([3.0, 4.0], torch.device("cpu")) == [3.0, 4.0]
    assert bench.job_value(100, 1, 2.0) == 50.0
