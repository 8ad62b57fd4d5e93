"""The device side of the gradient exchange (Sec. 4.2's minibatch split over GPUs): words copied
out of ciphertexts and summed as integers, then reduced by pft_ct_reduce_sum, equal the oracle's
HADD bit for bit; a one-rank all-reduce through exchange.allreduce_ciphertexts leaves the
ciphertext as it was; a sum that could exceed 64 bits is refused."""
import socket

import numpy as np
import pytest

from paper_1908_06972_gb300 import synth

from .pairs import Pair

pytestmark = pytest.mark.gpu


def test_reduce_sum_equals_hadd(gpu):
    import torch

    pf = gpu
    p = Pair(gpu, 12, 3, 1, 1, rot_steps=[], relin=False)
    try:
        o = p.orc
        cts = [o.encrypt_sk(o.encode(synth.slots(40 + i, 64)), 50 + i) for i in range(3)]
        hs = [p.ct(c) for c in cts]
        bufs = [torch.empty((2, 3, p.N), dtype=torch.int64, device="cuda") for _ in hs]
        for h, b in zip(hs, bufs):
            pf.pft_ct_copy_out(p.ctx, h, b.data_ptr())
        total = bufs[0] + bufs[1] + bufs[2]  # exact: 3 (q - 1) < 2^64
        out = p.empty()
        pf.pft_ct_reduce_sum(p.ctx, total.data_ptr(), 3, cts[0].scale, 3, out)
        want = o.add(o.add(cts[0], cts[1]), cts[2])
        p.assert_equal(out, want, "reduce_sum of three ciphertexts")
        with pytest.raises(pf.PftError) as e:  # 2^5 60-bit residues can exceed 2^64
            pf.pft_ct_reduce_sum(p.ctx, total.data_ptr(), 3, cts[0].scale, 32, out)
        assert e.value.code == pf.PFT_ERR_ARG
    finally:
        p.close()


def test_allreduce_one_rank_is_identity(gpu):
    import torch.distributed as dist

    from paper_1908_06972_gb300 import exchange

    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    dist.init_process_group("nccl", init_method="tcp://127.0.0.1:%d" % port, rank=0, world_size=1)
    p = Pair(gpu, 12, 3, 1, 1, rot_steps=[], relin=False)
    try:
        o = p.orc
        c = o.encrypt_sk(o.encode(synth.slots(60, 64)), 61)
        h = p.ct(c)
        exchange.allreduce_ciphertexts(gpu, p.ctx, [h])
        p.assert_equal(h, c, "one-rank all-reduce")
    finally:
        p.close()
        dist.destroy_process_group()
