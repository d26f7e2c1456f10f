"""The benchmark's multi-rank host logic on CPU: two gloo ranks (world size 2).

Replicas shard across ranks with no data-path exchange; the only collective is
the max over ranks of the timed totals, and the whole-job rate divides the
units of all ranks by the slowest rank's time."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist          # noqa: E402
import torch.multiprocessing as mp        # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    mine = [1.0 + rank, 5.0 - 2 * rank]          # rank 0: (1, 5), rank 1: (2, 3)
    got = bench.reduce_max(mine, ws)
    rate = bench.whole_job_rate(100, 4, ws, got[0])
    q.put((rank, got, rate, bench.shard_seed(rank)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
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
    for rank, got, rate, seed in res:
        assert got == [2.0, 5.0]                 # max over ranks, element by element
        assert rate == 100 * 4 * 2 / 2.0         # all ranks' units / slowest time
    assert res[0][3] != res[1][3]                # disjoint shards
