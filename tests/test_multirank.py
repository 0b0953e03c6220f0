"""The multi-rank path of bench.py on CPU: two gloo ranks (127.0.0.1), each
timing its own replica; the job's time is the slowest rank's and the value
counts the units of both ranks."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    ws, r, local = bench.dist_env()
    assert (ws, r, local) == (world, rank, rank)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        secs = [1.5, 2.5][rank]                       # rank 1 is slower
        total = bench.slowest_rank_seconds(secs, dist, "cpu")
        value = bench.whole_job_rate(ws, 20 * 10, total)  # 10 steps of 20 frames per rank
        out.put((rank, total, value))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_slowest_rank_and_whole_job_value():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, total, value in res:
        assert total == 2.5                          # max over ranks
        assert value == pytest.approx(2 * 200 / 2.5)  # both ranks' frames / slowest time
