"""Host-side fault injection through the C ABI (no fault is raised on the GPU).

* A caller allocator with a byte cap refuses the key-switching work space of a batched
  HMUL + relinearisation: the call returns PFT_ERR_OOM, frees what it had taken, and the
  context stays usable (the same call with the cap lifted equals the oracle bit for bit).
* Handles from another context, destroyed handles and pointers that never were handles are
  refused with PFT_ERR_ARG before the library reads through them."""
import ctypes

import numpy as np
import pytest

from paper_1908_06972_gb300 import synth

from .pairs import Pair

pytestmark = pytest.mark.gpu


class CappedAllocator:
    """torch's caching allocator behind a byte cap that the test moves; counts live bytes."""

    def __init__(self, pft, torch):
        self.torch = torch
        self.cap = None
        self.live = {}
        self.refused = 0

        def _alloc(nbytes, stream, user):
            if self.cap is not None and sum(self.live.values()) + nbytes > self.cap:
                self.refused += 1
                return None
            try:
                p = torch.cuda.caching_allocator_alloc(int(nbytes), 0, int(stream or 0))
            except Exception:
                return None
            self.live[p] = int(nbytes)
            return p

        def _free(ptr, stream, user):
            if ptr:
                self.live.pop(ptr, None)
                torch.cuda.caching_allocator_delete(ptr)

        self.struct = pft.pft_allocator(pft.ALLOC_FN(_alloc), pft.FREE_FN(_free), None)

    def in_use(self):
        return sum(self.live.values())


def test_allocator_cap_gives_oom_and_context_survives(gpu):
    import torch

    pf = gpu
    cap = CappedAllocator(pf, torch)
    seed = (0x0A, 0x0B, 0x0C, 0x0D)
    from oracle import ckks

    o = ckks.Oracle(12, 6, 1, 2, 60, 40, 60, 2.0 ** 40, seed)
    o.keygen([], True)
    ctx = pf.pft_ctx_create(12, 6, 1, 2, 60, 40, 60, 2.0 ** 40, seed, flags=pf.PFT_ALLOW_INSECURE,
                            allocator=cap.struct)
    hs = []
    try:
        pf.pft_keygen(ctx, [], True)
        A = [o.encrypt_sk(o.encode(synth.slots(10 + i, 64), level=6 - i), 20 + i) for i in range(3)]
        B = [o.encrypt_sk(o.encode(synth.slots(30 + i, 64), level=6 - i), 40 + i) for i in range(3)]
        gA = [pf.pft_ct_import(ctx, x.c, x.scale) for x in A]
        gB = [pf.pft_ct_import(ctx, x.c, x.scale) for x in B]
        C = [pf.pft_ct_create(ctx) for _ in A]
        hs = gA + gB + C
        torch.cuda.synchronize()
        before = cap.in_use()
        cap.cap = before + 64 * 1024  # far below the work space of three key switches
        with pytest.raises(pf.PftError) as e:
            pf.pft_mul_relin_batch(ctx, gA, gB, C)
        assert e.value.code == pf.PFT_ERR_OOM and "allocation" in str(e.value)
        assert cap.refused >= 1
        torch.cuda.synchronize()
        assert cap.in_use() <= before + 64 * 1024  # nothing of the failed call is held beyond the outputs
        cap.cap = None
        pf.pft_mul_relin_batch(ctx, gA, gB, C)
        for h, a, b in zip(C, A, B):
            assert np.array_equal(pf.pft_ct_export(ctx, h), o.mul_relin(a, b).c)
        pf.pft_device_status(ctx)
    finally:
        for h in hs:
            pf.pft_ct_destroy(h)
        pf.pft_ctx_destroy(ctx)


def test_foreign_destroyed_and_bogus_handles(gpu):
    pf = gpu
    p = Pair(gpu, 12, 3, 1, 1, rot_steps=[1])
    q = Pair(gpu, 12, 3, 1, 1, rot_steps=[1], seed=(9, 9, 9, 9))
    try:
        o = p.orc
        a = o.encrypt_sk(o.encode(synth.slots(1, 64), level=3), 1)
        ga, gb, out = p.ct(a), p.ct(a), p.empty()
        foreign = q.ct(q.orc.encrypt_sk(q.orc.encode(synth.slots(2, 64), level=3), 2))
        for call in (lambda: pf.pft_add(p.ctx, ga, foreign, out),
                     lambda: pf.pft_mul_relin(p.ctx, foreign, gb, out),
                     lambda: pf.pft_rotate(p.ctx, ga, 1, q.empty())):
            with pytest.raises(pf.PftError) as e:
                call()
            assert e.value.code == pf.PFT_ERR_ARG and "another context" in str(e.value)
        dead = pf.pft_ct_create(p.ctx)
        pf.pft_add(p.ctx, ga, gb, dead)
        pf.pft_ct_destroy(dead)
        with pytest.raises(pf.PftError) as e:
            pf.pft_add(p.ctx, dead, gb, out)
        assert e.value.code == pf.PFT_ERR_ARG and "live" in str(e.value)
        with pytest.raises(pf.PftError) as e:
            pf.pft_ct_destroy(dead)  # a second destroy is refused, not a double free
        assert e.value.code == pf.PFT_ERR_ARG
        bogus = ctypes.c_void_p(ctypes.addressof(ctypes.create_string_buffer(64)))
        with pytest.raises(pf.PftError) as e:
            pf.pft_rescale(p.ctx, bogus, out)
        assert e.value.code == pf.PFT_ERR_ARG
        # the context is still usable
        pf.pft_mul_relin(p.ctx, ga, gb, out)
        p.assert_equal(out, o.mul_relin(a, a), "after the refused calls")
    finally:
        q.close()
        p.close()
