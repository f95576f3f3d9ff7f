"""The multi-GPU benchmark runs independent replicas: every rank optimises
its own seeded image and the ranks meet only in a barrier and the max over
ranks of the timed region.  Exercised here with two gloo ranks on CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, l = bench.dist_setup()
    assert (w, r, l) == (world, rank, rank)
    dist.barrier()
    mx = bench.max_over_ranks(10.0 + 5.0 * rank, "cpu")
    q.put((rank, mx, bench.replica_seed(1, rank)))
    dist.destroy_process_group()


def test_two_rank_aggregation_and_replica_seeds():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    assert [m for _, m, _ in res] == [15.0, 15.0]      # max over ranks on every rank
    assert [s for _, _, s in res] == [1, 2]            # distinct images per rank


def test_single_process_aggregation_is_identity():
    import bench
    assert bench.max_over_ranks(3.5, "cpu") == 3.5
