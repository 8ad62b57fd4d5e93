"""Edge cases of the GPU path against the oracle and the layout definition.

* Transforms at every supported shape class (one pass N <= 2^14; at 2^15 and 2^16 every plan
  the autotuner searches: the specialised kernels and the generic passes of every stage split)
  with primes on both sides of the lazy-butterfly bound 2^57 (57-bit
  primes are the largest on the lazy path), the benchmark's 50-bit primes and small ones, on
  extreme inputs (every coefficient q - 1, alternating 0 / q - 1) and random ones: forward
  equal to the evaluation definition, inverse restoring the input exactly.
* Degenerate operations: empty batches, identity and wrap-around rotations, level-1
  ciphertexts (one prime: one digit), rescale refused at level 1."""
import numpy as np
import pytest

from oracle import _lib as OC
from oracle import params as OP
from paper_1908_06972_gb300 import synth

from .pairs import Pair

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("logn", [4, 8, 11, 15, 16])
@pytest.mark.parametrize("bits", [(59, 58, 60), (57, 57, 60), (58, 57, 58), (50, 50, 60), (30, 30, 31)])
def test_transform_extreme_inputs(gpu, logn, bits):
    import torch

    first, mid, special = bits
    p = Pair(gpu, logn, 3, 1, 1, first_bits=first, mid_bits=mid, special_bits=special, gpu_keys=False,
             rot_steps=(), relin=False)
    try:
        if logn >= 15:
            gpu.pft_autotune(p.ctx)
        primes = gpu.pft_ctx_info(p.ctx)["primes"]  # q0, q1, q2 and the special prime
        n = 1 << logn
        x = synth.residues(17, primes, n, polys=3)
        for r, q in enumerate(primes):
            x[0, r, :] = q - 1                        # every coefficient at its maximum
            x[1, r, :] = np.where(np.arange(n) % 2 == 0, 0, q - 1)
        idx = np.arange(n) if logn <= 11 else np.r_[0:32, n // 2 - 16:n // 2 + 16, n - 32:n]
        want = [[OC.eval_at(x[poly, r], OP.root_2n(q, logn), q, logn, idx) for r, q in enumerate(primes)]
                for poly in range(3)]
        # every transform plan the autotuner searches at N = 2^15 and 2^16
        plans = range(len(gpu.pft_autotune_report(p.ctx)["buckets"][0]["us_fwd_inv"])) if logn >= 15 else [None]
        for variant in plans:
            if variant is not None:
                gpu.pft_set_transform_plan(p.ctx, variant)
            t = torch.from_numpy(x.view(np.int64).copy()).cuda()
            gpu.pft_ntt(p.ctx, t.data_ptr(), 3, len(primes), 0)
            y = t.cpu().numpy().view(np.uint64)
            for poly in range(3):
                for r, q in enumerate(primes):
                    assert np.all(y[poly, r] < q), (variant, poly, r)
                    assert np.array_equal(y[poly, r][idx], want[poly][r]), (logn, bits, variant, poly, r)
            gpu.pft_ntt(p.ctx, t.data_ptr(), 3, len(primes), 1)
            assert np.array_equal(t.cpu().numpy().view(np.uint64), x), variant
    finally:
        p.close()


@pytest.fixture(scope="module")
def pe(gpu):
    p = Pair(gpu, 12, 3, 1, 1, rot_steps=[1, 2047, 1024], seed=(0xED6E, 1, 2, 3))
    yield p
    p.close()


def test_empty_batches(pe):
    pf, ctx = pe.pft, pe.ctx
    pf.pft_mul_relin_batch(ctx, [], [], [])
    pf.pft_rotate_batch(ctx, [], 1, [])
    pf.pft_rescale_batch(ctx, [], [])
    pf.pft_add_batch(ctx, [], [], [])
    assert pf.pft_ct_import_batch(ctx, [], []) == []
    pf.pft_ct_export_batch(ctx, [], [])
    pf.pft_device_status(ctx)


def test_identity_and_wraparound_rotations(pe):
    o, pf, ctx = pe.orc, pe.pft, pe.ctx
    t = pe.N // 2
    a = o.encrypt_sk(o.encode(synth.slots(3, t), level=3), 31)
    g = pe.ct(a)
    for step in (0, t, -t):  # g = 1: a copy
        out = pe.empty()
        pf.pft_rotate(ctx, g, step, out)
        pe.assert_equal(out, a, "rotate by %d" % step)
    for step, same in ((t - 1, -1), (-(t - 1), 1), (t // 2, -(t // 2))):
        out = pe.empty()
        pf.pft_rotate(ctx, g, step, out)
        pe.assert_equal(out, o.rotate(a, same), "rotate by %d" % step)


def test_level_one_ciphertexts(pe):
    """One prime left: the key switch has a single one-prime digit; rescale is refused."""
    o, pf, ctx = pe.orc, pe.pft, pe.ctx
    a = o.encrypt_sk(o.encode(synth.slots(4, 64), level=1), 41)
    b = o.encrypt_pk(o.encode(synth.slots(5, 64), level=1), 42)
    ga, gb = pe.ct(a), pe.ct(b)
    out = pe.empty()
    pf.pft_mul_relin(ctx, ga, gb, out)
    pe.assert_equal(out, o.mul_relin(a, b), "mul_relin at level 1")
    pf.pft_rotate(ctx, ga, 1, out)
    pe.assert_equal(out, o.rotate(a, 1), "rotate at level 1")
    with pytest.raises(pf.PftError) as e:
        pf.pft_rescale(ctx, ga, out)
    assert e.value.code == pf.PFT_ERR_LEVEL_MISMATCH


def test_butterfly_ceiling_is_below_the_derived_bound(pe):
    """The register-only butterfly rate is positive and below 152 SMs x 64 32-bit multiplies per
    clock x 2.07 GHz / 9 multiplies per butterfly."""
    v = pe.pft.pft_bfly_ceiling(pe.ctx)
    assert 1e10 < v < 152 * 64 * 2.07e9 / 9
