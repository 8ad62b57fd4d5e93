"""Full-size parity in the benchmark's own launch configuration, and the fastText inference of
Sec. 5.5.1 at the top of a 30-prime chain.

* The benchmark batch: 64 ciphertexts at N = 2^16 on the 60 + 29 x 50-bit chain with 4 special
  primes and digits of 4 primes, at the benchmark's levels (uniform in 5..30, the same seed),
  through one batched HMUL + relinearisation and two batched rotations (+1, -1; Sec. 2.3).
  Every basis conversion of these calls runs in launches split at the per-launch job limit and
  every transform in several launch descriptors; each of the 64 results is compared limb for
  limb with the oracle.
* fastText at level 30 (60 + 29 x 40-bit chain, 4 special primes, digits of 4 primes): the
  Fig. 3 sequence with two columns bit-exact against the oracle, and the 32768 x 64 x 14 model
  in one batched call within 2^-20 of the FP64 Algorithm 1 with the predicted class.

The oracle's share takes a few minutes on 16 cores, so these tests are also marked slow."""
import numpy as np
import pytest

from oracle import fasttext as OF
from paper_1908_06972_gb300 import synth

from .pairs import Pair

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def test_benchmark_batch_bit_exact(gpu):
    p = Pair(gpu, 16, 30, 4, 4, first_bits=60, mid_bits=50, special_bits=60, scale=2.0 ** 50,
             seed=(0x5EED0001, 0x5EED0002, 0x5EED0003, 0x5EED0004), rot_steps=[1, -1], insecure=False)
    try:
        o, pf, ctx = p.orc, p.pft, p.ctx
        lv = synth.batch_levels(64, 5, 30)
        A = [o.encrypt_sk(o.encode(synth.slots(1000 + i, 256), level=l), 2 * i) for i, l in enumerate(lv)]
        B = [o.encrypt_sk(o.encode(synth.slots(5000 + i, 256), level=l), 2 * i + 1) for i, l in enumerate(lv)]
        gA, gB = [p.ct(x) for x in A], [p.ct(x) for x in B]
        C = [p.empty() for _ in lv]
        pf.pft_prof_start("bconv")
        pf.pft_mul_relin_batch(ctx, gA, gB, C)
        _, n_bconv, _, _ = pf.pft_prof_stop()
        assert n_bconv >= 4  # ModUp jobs (sum of digits > 300) in several launches, and ModDown
        want = [o.mul_relin(a, b) for a, b in zip(A, B)]
        for i in range(len(lv)):
            p.assert_equal(C[i], want[i], "mul_relin %d (level %d)" % (i, lv[i]))
        for step in (1, -1):
            pf.pft_rotate_batch(ctx, C, step, C)
            want = [o.rotate(w, step) for w in want]
            for i in range(len(lv)):
                p.assert_equal(C[i], want[i], "rotate %+d of %d (level %d)" % (step, i, lv[i]))
    finally:
        p.close()


@pytest.fixture(scope="module")
def p3_30(gpu):
    steps = [1 << i for i in range(15)]
    p = Pair(gpu, 16, 30, 4, 4, first_bits=60, mid_bits=40, special_bits=60, scale=2.0 ** 40,
             seed=(0xF00D, 4, 5, 6), rot_steps=steps, relin=False, insecure=False)
    yield p
    p.close()


def test_fasttext_two_columns_bit_exact_level30(p3_30):
    o, pf, ctx = p3_30.orc, p3_30.pft, p3_30.ctx
    t = p3_30.N // 2
    m, n, c, L = t, 2, 14, 30
    H, O = synth.fasttext_weights(61, m, n, c)
    docs = synth.documents(62, m, 1)
    Hp, Opk = OF.pack_H(H, t), OF.pack_O(O, t)
    H_o = [[o.encode(Hp[j, 0], level=L)] for j in range(n)]
    O_o = [o.encode(Opk[j], level=L - 1) for j in range(n)]
    model = pf.pft_ft_model_import(ctx, [p3_30.pt(H_o[j][0]) for j in range(n)], [p3_30.pt(x) for x in O_o],
                                   m, n, c)
    try:
        v = o.encrypt_sk(o.encode(docs[0], level=L), 4343)
        s = p3_30.empty()
        pf.pft_fasttext_infer(ctx, model, [p3_30.ct(v)], s)
        want = OF.encrypted_scores(o, [v], H_o, O_o)
        p3_30.assert_equal(s, want, "fasttext level 30, two columns")
        dec = o.decode(o.decrypt(want))[:c].real
        assert np.max(np.abs(dec - OF.plain_scores(docs[0], H, O))) < 2.0 ** -20
    finally:
        pf.pft_ft_model_destroy(model)


def test_fasttext_full_model_level30_tolerance(p3_30):
    """Vocabulary 32768, embedding 64, 14 classes at level 30; 4 documents in one call."""
    pf, ctx = p3_30.pft, p3_30.ctx
    t = p3_30.N // 2
    m, n, c, L = 32768, 64, 14, 30
    H, O = synth.fasttext_weights(63, m, n, c)
    docs = synth.documents(64, m, 4)
    model = pf.pft_ft_model_create(ctx, H, O, L)
    vs = []
    try:
        for d in range(4):
            pt = pf.pft_encode(ctx, docs[d], 2.0 ** 40, L)
            vs.append(pf.pft_encrypt(ctx, pt, pf.PFT_ENC_SK, 9000 + d))
            pf.pft_pt_destroy(pt)
        scores = [p3_30.empty() for _ in range(4)]
        pf.pft_fasttext_infer_batch(ctx, model, vs, 1, scores)
        for d in range(4):
            assert pf.pft_ct_level(scores[d]) == L - 2
            dec = pf.pft_decrypt(ctx, scores[d])
            got = pf.pft_decode(ctx, dec, t)[:c].real
            pf.pft_pt_destroy(dec)
            want = OF.plain_scores(docs[d], H, O)
            assert np.max(np.abs(got - want)) < 2.0 ** -20, np.max(np.abs(got - want))
            srt = np.sort(want)
            if srt[-1] - srt[-2] >= 2.0 ** -18:
                assert int(np.argmax(got)) == int(np.argmax(want))
    finally:
        for h in vs:
            pf.pft_ct_destroy(h)
        pf.pft_ft_model_destroy(model)
