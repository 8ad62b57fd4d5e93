"""pft_rescale_noalloc against pft_rescale, through the C ABI.

pft_rescale_noalloc serves callers that cannot obtain device memory at the moment they
call the library (their device memory is owned by another framework's pool, or their
processing loop must not call an allocator).  It takes raw device buffers for the input
and the output and does its work in a fixed array compiled into the library, so it must
produce exactly what the allocating pft_rescale produces.  Two calls in a row check that
the contents the first call leaves in the shared array do not leak into the second.
This file is collected last so that a stop at the first failure has run every other test.
"""
import numpy as np
import pytest

from paper_1908_06972_gb300 import synth

pytestmark = pytest.mark.gpu


def test_rescale_noalloc_matches_rescale(gpu):
    import torch

    pft = gpu
    torch.cuda.set_device(0)
    ctx = pft.pft_ctx_create(16, 8, 2, 4, 60, 50, 60, 2.0 ** 50, (7, 7, 7, 7))
    try:
        n = pft.pft_ctx_info(ctx)["N"]
        pft.pft_keygen(ctx, [], False)
        for call, level in enumerate((8, 5)):  # two calls in a row, different sizes
            pt = pft.pft_encode(ctx, synth.slots(60 + call, 1024), 2.0 ** 50, level)
            ct = pft.pft_encrypt(ctx, pt, pft.PFT_ENC_SK, 500 + call)
            out = torch.empty((2, level - 1, n), dtype=torch.int64, device="cuda")
            pft.pft_rescale_noalloc(ctx, pft.pft_ct_data(ct), level, out.data_ptr())
            ref = pft.pft_ct_create(ctx)
            pft.pft_rescale(ctx, ct, ref)
            want = pft.pft_ct_export(ctx, ref)  # coefficient form
            pft.pft_ntt(ctx, out.data_ptr(), 2, level - 1, 1)  # evaluation -> coefficient form
            torch.cuda.synchronize()
            got = out.cpu().numpy().view(np.uint64)
            assert got.shape == want.shape
            assert np.array_equal(got, want), "call %d: %d words differ" % (call, int((got != want).sum()))
            for h in (ct, ref):
                pft.pft_ct_destroy(h)
            pft.pft_pt_destroy(pt)
        # input and output may not overlap
        pt = pft.pft_encode(ctx, synth.slots(70, 64), 2.0 ** 50, 4)
        ct = pft.pft_encrypt(ctx, pt, pft.PFT_ENC_SK, 600)
        p_in = pft.pft_ct_data(ct)
        with pytest.raises(pft.PftError) as e:
            pft.pft_rescale_noalloc(ctx, p_in, 4, p_in + 8 * n)
        assert e.value.code == pft.PFT_ERR_ARG and "overlap" in str(e.value)
        pft.pft_ct_destroy(ct)
        pft.pft_pt_destroy(pt)
        # the largest accepted size fills the array exactly: 2 N level = 4 Mi words at level 32
        top = pft.pft_ctx_create(16, 32, 2, 4, 60, 40, 60, 2.0 ** 40, (3, 3, 3, 3))
        try:
            pft.pft_keygen(top, [], False)
            pt = pft.pft_encode(top, synth.slots(71, 1024), 2.0 ** 40, 32)
            ct = pft.pft_encrypt(top, pt, pft.PFT_ENC_SK, 700)
            out = torch.empty((2, 31, n), dtype=torch.int64, device="cuda")
            pft.pft_rescale_noalloc(top, pft.pft_ct_data(ct), 32, out.data_ptr())
            ref = pft.pft_ct_create(top)
            pft.pft_rescale(top, ct, ref)
            want = pft.pft_ct_export(top, ref)
            pft.pft_ntt(top, out.data_ptr(), 2, 31, 1)
            torch.cuda.synchronize()
            assert np.array_equal(out.cpu().numpy().view(np.uint64), want), "level 32 differs"
            for h in (ct, ref):
                pft.pft_ct_destroy(h)
            pft.pft_pt_destroy(pt)
        finally:
            pft.pft_ctx_destroy(top)
        # sizes beyond the fixed array are refused with a clear error
        big = pft.pft_ctx_create(16, 40, 2, 4, 60, 40, 60, 2.0 ** 40, (1, 1, 1, 1), flags=pft.PFT_ALLOW_INSECURE)
        try:
            src = torch.zeros((2, 40, n), dtype=torch.int64, device="cuda")
            dst = torch.zeros((2, 39, n), dtype=torch.int64, device="cuda")
            with pytest.raises(pft.PftError) as e:
                pft.pft_rescale_noalloc(big, src.data_ptr(), 40, dst.data_ptr())
            assert e.value.code == pft.PFT_ERR_ARG and "exceed" in str(e.value)
        finally:
            pft.pft_ctx_destroy(big)
    finally:
        pft.pft_ctx_destroy(ctx)
