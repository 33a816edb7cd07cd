"""Multi-rank host logic of the benchmark on CPU (gloo, world size 2): ranks
run disjoint events, the time is the maximum over ranks, the value counts the
units of every rank."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        got = bench.max_over_ranks([1.5 + rank, 10.0 - 3 * rank, 7.0], ws)
        q.put((rank, got, bench._dist(), bench.event_seeds(rank, 32)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_maximum_and_disjoint_events():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res.sort()
    for rank, got, d, seeds in res:
        assert got == [2.5, 10.0, 7.0]
        assert d == (2, rank, rank)
    assert not set(res[0][3]) & set(res[1][3])


def test_single_rank_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([3.0, 4.0], 1) == [3.0, 4.0]
    assert bench.whole_job_rate(4, 300, 0.5) == pytest.approx(2400.0)
    assert bench.event_seeds(0, 3) == [0, 1, 2]
