"""The bench's N > 1 host path on CPU: two gloo ranks (replicas) combine
their timings as the slowest rank's and report the whole-job throughput."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    mine = [10.0 + rank, 5.0 * (rank + 1)]
    dist.barrier()
    got = bench.ranks_max(mine, "cpu")
    q.put((rank, got, bench.whole_job_gbs(world, 1e9, got[0])))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, gbs in out:
        assert got == [11.0, 10.0]
        assert gbs == pytest.approx(2 * 1e9 / (11.0e-3) / 1e9)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.ranks_max([3.0, 4.0], "cpu") == [3.0, 4.0]
    assert bench.whole_job_gbs(1, 2e9, 1000.0) == pytest.approx(2.0)
