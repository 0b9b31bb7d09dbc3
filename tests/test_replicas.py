"""Multi-GPU form of bench.py (independent replicas, no data-path collective) on CPU: two gloo ranks agree on
the slowest rank's time, take disjoint problem seeds, and report whole-job throughput."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.max_over_ranks(100.0 + 50.0 * rank, "cpu")
    seeds = bench.rank_seeds(rank, 4)
    gathered = [None] * world
    dist.all_gather_object(gathered, seeds)
    out.put((rank, t, gathered))
    dist.destroy_process_group()


def test_two_replicas_on_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, gathered in res:
        assert t == 150.0                      # the slowest rank's time on every rank
        a, b = gathered
        assert len(set(a) | set(b)) == 8       # disjoint seeds
    import bench
    assert bench.job_throughput(2, 4, 5, 2000.0) == pytest.approx(20.0)
