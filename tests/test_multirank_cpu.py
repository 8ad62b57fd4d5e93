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


# ---- exchange of encrypted gradients (Sec. 4.2: the minibatch split over ranks) --------------
def _exchange_worker(rank, world, port, q, plan):
    import numpy as np
    import torch.distributed as dist

    from oracle import ckks
    from paper_1908_06972_gb300 import exchange, synth

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # the same chain on every rank (one 60-bit and two 50-bit primes at N = 2^10), each rank its
    # own gradient ciphertext
    o = ckks.Oracle(10, 3, 1, 1, 60, 50, 60, 2.0 ** 40, (5, 6, 7, 8))
    o.keygen([], False)
    cts = [o.encrypt_sk(o.encode(synth.slots(100 + r, 64)), 7 + r) for r in range(world)]
    mine = torch.from_numpy(cts[rank].c.view(np.int64).copy())

    def reduce_mod(acc, part):  # the oracle's modular addition, limb by limb
        a = ckks.Ciphertext(exchange.as_uint64(acc).copy(), 1.0)
        b = ckks.Ciphertext(exchange.as_uint64(part).copy(), 1.0)
        return torch.from_numpy(o.add(a, b).c.view(np.int64).copy())

    out, used = exchange.sum_words(mine, plan=plan, primes=o.q, reduce_mod=reduce_mod)
    words = exchange.as_uint64(out)
    if used == exchange.SUM:  # exact integer sums: reduce them modulo each limb's prime
        words = np.stack([np.stack([words[p, r] % np.uint64(o.q[r]) for r in range(3)]) for p in range(2)])
    want = cts[0]
    for c in cts[1:]:
        want = o.add(want, c)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, used, bool(np.array_equal(words, want.c))))


@pytest.mark.parametrize("plan", [None, "gather"])
def test_two_rank_gradient_exchange_gloo(plan):
    """Two ranks sum their ciphertexts: by one integer all-reduce (2 (q - 1) < 2^64, the plan the
    rule picks) and by gathering with modular additions; both equal the oracle's HADD."""
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_exchange_worker, args=(r, 2, port, q, plan)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert all(ok for _, _, ok in res), res
    assert all(u == (plan or "sum") for _, u, _ in res)


def test_exchange_rule():
    from paper_1908_06972_gb300 import exchange

    q60, q50 = (1 << 60) - 93, (1 << 50) - 27
    assert exchange.exchange_plan(16, [q60]) == "sum"       # 16 (q - 1) < 2^64
    assert exchange.exchange_plan(17, [q60]) == "gather"
    assert exchange.exchange_plan(16384, [q50]) == "sum"
    assert exchange.exchange_plan(2, [q60, q50]) == "sum"
