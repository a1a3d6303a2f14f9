"""The N > 1 host logic of bench.py on CPU: every rank runs its own replica of the workload
(weak scaling, no collective on the data path) and the job's time is the slowest rank's,
taken with one all-reduce; checked with two gloo ranks on 127.0.0.1."""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys

    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ws, r, local = bench.dist_env()
        local_ms = 100.0 + 50.0 * rank  # rank 1 is the slow one
        out.put((r, ws, bench.max_over_ranks(local_ms, dist), bench.max_over_ranks(local_ms, None)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r for r, *_ in res] == [0, 1]
    assert all(ws == 2 for _, ws, *_ in res)
    assert all(m == pytest.approx(150.0) for _, _, m, _ in res)       # the job's time: the slowest rank
    assert [own for *_, own in res] == [100.0, 150.0]                  # one rank: its own time
