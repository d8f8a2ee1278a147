"""Multi-GPU host logic of bench.py on CPU: two gloo ranks, each with its own
workload seed; the job's time is the slowest rank's, and the throughput counts
every rank's labels (weak scaling).  The labeling path itself never crosses
ranks (edges are independent, eq. 10), so there is no data-path collective."""
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


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    seed = bench.rank_seed(7, rank)
    slowest = bench.max_over_ranks(10.0 * (rank + 1), dist, "cpu")
    value = bench.job_throughput(world, 1000, 64, 20, slowest)
    q.put((rank, seed, slowest, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_weak_scaling_logic():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    seeds = {o[1] for o in out}
    assert len(seeds) == world  # independent frames per rank
    assert all(o[2] == 20.0 for o in out)  # max over ranks
    assert all(abs(o[3] - world * 1000 * 64 * 20 / 0.020) < 1e-6 * o[3] for o in out)
