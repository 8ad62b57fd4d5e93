"""The replica path of bench.py on two CPU ranks (gloo): ranks time independent batches,
the job's time is the slowest rank's, and the whole-job throughput counts every rank's
units.  No GPU and no data-path collective are involved."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, local = bench.dist_env()
    per_rank_seconds = [2.0, 3.0][rank]
    slowest = bench.reduce_max(per_rank_seconds, "cpu")
    value = bench.throughput(64 * 5, w, slowest)
    dist.barrier()
    dist.destroy_process_group()
    q.put((r, w, slowest, value))


def test_two_rank_aggregation_gloo():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [x[0] for x in res] == [0, 1] and all(x[1] == 2 for x in res)
    assert all(x[2] == 3.0 for x in res)  # both ranks see the slowest rank's time
    assert all(abs(x[3] - 64 * 5 * 2 / 3.0) < 1e-9 for x in res)


def test_single_process_is_identity():
    import bench

    assert bench.reduce_max(1.5, "cpu") == 1.5
    assert bench.throughput(10, 1, 2.0) == 5.0
