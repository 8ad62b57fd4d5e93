"""Bit-exact parity of batches large enough to be split across several launches.

A batched key switch issues its basis conversions in launches of at most 96 jobs (one
launch descriptor per group of jobs with the same number of source primes), its key inner
products in launches of at most 128 inputs, and its transforms, automorphisms and
elementwise passes in launch descriptors of at most 256 polynomials.  The benchmark's batch
of 64 ciphertexts at N = 2^16 always takes those split paths; these tests take them at
N = 2^12 (ten 40-bit primes after a 60-bit one, one special prime, one prime per digit, so a
ciphertext at level l brings l conversion jobs) and compare every ciphertext limb for limb
with the oracle (HMUL + relinearisation, ROTATE and RESCALE of Sec. 2.3; TotalSum of
Algorithm 2 inside the fastText sequence of Sec. 3.1).  Each test checks with the library's
launch counter that the split actually happened."""
import numpy as np
import pytest

from oracle import fasttext as OF
from paper_1908_06972_gb300 import synth

from .pairs import Pair

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def p10(gpu):
    p = Pair(gpu, 12, 10, 1, 1, rot_steps=[1 << i for i in range(11)] + [-1])
    yield p
    p.close()


def _levels(seed, count, lo, hi):
    rng = np.random.default_rng(seed)
    return [int(x) for x in rng.integers(lo, hi + 1, count)]


def _launches(pf, prefix, fn):
    pf.pft_prof_start(prefix)
    try:
        fn()
    finally:
        _, timed, _, _ = pf.pft_prof_stop()
    return timed


def _encrypt(o, seed, nonce, level):
    return o.encrypt_sk(o.encode(synth.slots(seed, 64), level=level), nonce)


def test_mul_relin_batch_over_conversion_launch_limit(p10):
    """16 pairs at levels U{5..10}: more than 96 ModUp jobs with one source prime, so the
    conversion runs in several launches; then the products rotated and rescaled as one batch."""
    o, pf, ctx = p10.orc, p10.pft, p10.ctx
    lv = _levels(7, 16, 5, 10)
    assert sum(lv) > 96
    A = [_encrypt(o, 100 + i, 1000 + i, l) for i, l in enumerate(lv)]
    B = [_encrypt(o, 200 + i, 2000 + i, l) for i, l in enumerate(lv)]
    gA, gB = [p10.ct(x) for x in A], [p10.ct(x) for x in B]
    C = [p10.empty() for _ in lv]
    n_bconv = _launches(pf, "bconv", lambda: pf.pft_mul_relin_batch(ctx, gA, gB, C))
    assert n_bconv >= 3  # ModUp split in two or more launches, plus ModDown
    M = [o.mul_relin(a, b) for a, b in zip(A, B)]
    for i in range(len(lv)):
        p10.assert_equal(C[i], M[i], "mul_relin %d (level %d)" % (i, lv[i]))
    pf.pft_rotate_batch(ctx, C, -1, C)
    R = [o.rotate(m, -1) for m in M]
    for i in range(len(lv)):
        p10.assert_equal(C[i], R[i], "rotate %d (level %d)" % (i, lv[i]))
    pf.pft_rescale_batch(ctx, C, C)
    for i in range(len(lv)):
        p10.assert_equal(C[i], o.rescale(R[i]), "rescale %d (level %d)" % (i, lv[i]))


def test_rotate_batch_over_inner_product_launch_limit(p10):
    """136 ciphertexts at levels U{1..10} rotated in one call: the key inner product takes two
    launches (128 + 8 inputs), the automorphism and transforms several descriptors of 256
    polynomials, the conversions many launches."""
    o, pf, ctx = p10.orc, p10.pft, p10.ctx
    lv = _levels(8, 136, 1, 10)
    A = [_encrypt(o, 300 + i, 3000 + i, l) for i, l in enumerate(lv)]
    gA = [p10.ct(x) for x in A]
    C = [p10.empty() for _ in lv]
    n_ks = _launches(pf, "ks_inner", lambda: pf.pft_rotate_batch(ctx, gA, 1, C))
    assert n_ks >= 2
    for i in range(len(lv)):
        p10.assert_equal(C[i], o.rotate(A[i], 1), "rotate %d (level %d)" % (i, lv[i]))
    keep = [i for i in range(len(lv)) if lv[i] >= 2]
    outs = [p10.empty() for _ in keep]
    pf.pft_rescale_batch(ctx, [C[i] for i in keep], outs)
    for j, i in enumerate(keep):
        p10.assert_equal(outs[j], o.rescale(o.rotate(A[i], 1)), "rescale %d" % i)


def test_fasttext_batch_over_inner_product_launch_limit(p10):
    """Encrypted fastText (Fig. 3 packing) of 9 documents with 16 columns at levels 3 and 4:
    every TotalSum step key-switches 144 column ciphertexts in one call (two inner-product
    launches); every score is compared with the oracle's canonical sequence."""
    o, pf, ctx = p10.orc, p10.pft, p10.ctx
    t = p10.N // 2
    m, n, c = t, 16, 5
    H, O = synth.fasttext_weights(41, m, n, c)
    docs = synth.documents(42, m, 9, 20, 60)
    Hp, Opk = OF.pack_H(H, t), OF.pack_O(O, t)
    top = 4
    H_o = [[o.encode(Hp[j, 0], level=top)] for j in range(n)]
    O_o = [o.encode(Opk[j], level=top - 1) for j in range(n)]
    model = pf.pft_ft_model_import(ctx, [p10.pt(H_o[j][0]) for j in range(n)], [p10.pt(x) for x in O_o], m, n, c)
    try:
        lv = [3 + (d % 2) for d in range(len(docs))]
        v_o = [o.encrypt_sk(o.encode(docs[d], level=lv[d]), 4000 + d) for d in range(len(docs))]
        v_g = [p10.ct(x) for x in v_o]
        scores = [p10.empty() for _ in docs]
        n_ks = _launches(pf, "ks_inner", lambda: pf.pft_fasttext_infer_batch(ctx, model, v_g, 1, scores))
        assert n_ks >= 2 * 11  # each of the 11 TotalSum steps in two launches
        for d in range(len(docs)):
            H_d = [[type(H_o[j][0])(H_o[j][0].m[:lv[d]], H_o[j][0].scale)] for j in range(n)]
            O_d = [type(O_o[j])(O_o[j].m[:lv[d] - 1], O_o[j].scale) for j in range(n)]
            want = OF.encrypted_scores(o, [v_o[d]], H_d, O_d)
            p10.assert_equal(scores[d], want, "fasttext doc %d (level %d)" % (d, lv[d]))
            dec = o.decode(o.decrypt(want))[:c].real
            assert np.max(np.abs(dec - OF.plain_scores(docs[d], H, O))) < 2.0 ** -20
    finally:
        pf.pft_ft_model_destroy(model)
