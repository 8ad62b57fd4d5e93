"""Full-size GPU parity: the benchmark's chain (N = 2^16, 30 primes: 60 + 29 x 50 bits,
4 special primes of 60 bits, digits of 4 primes) in the batched launch configuration the
benchmark times, against the oracle bit for bit; and the encrypted fastText inference at
N = 2^16 (32768 slots, 40-bit chain): a two-column model bit-exact against the oracle's
full sequence, the 64 x 14 model through the batched path against the FP64 Algorithm 1
within 2^-20."""
import numpy as np
import pytest

from oracle import fasttext as OF
from paper_1908_06972_gb300 import synth

from .pairs import Pair

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def p2(gpu):
    p = Pair(gpu, 16, 30, 4, 4, first_bits=60, mid_bits=50, special_bits=60, scale=2.0 ** 50,
             seed=(0x5EED0001, 0x5EED0002, 0x5EED0003, 0x5EED0004), rot_steps=[1, -1], insecure=False)
    yield p
    p.close()


def test_p2_batched_mul_relin_rescale_rotate(p2):
    o, pf, ctx = p2.orc, p2.pft, p2.ctx
    lv = [30, 17, 5]
    A = [o.encrypt_sk(o.encode(synth.slots(10 + i, 512), level=l), 100 + i) for i, l in enumerate(lv)]
    B = [o.encrypt_pk(o.encode(synth.slots(20 + i, 512), level=l), 200 + i) for i, l in enumerate(lv)]
    gA, gB = [p2.ct(x) for x in A], [p2.ct(x) for x in B]
    C = [p2.empty() for _ in lv]
    pf.pft_mul_relin_batch(ctx, gA, gB, C)
    M = [o.mul_relin(a, b) for a, b in zip(A, B)]
    for i in range(len(lv)):
        p2.assert_equal(C[i], M[i], "p2 mul_relin l=%d" % lv[i])
    pf.pft_rotate_batch(ctx, C, -1, C)
    R = [o.rotate(m, -1) for m in M]
    for i in range(len(lv)):
        p2.assert_equal(C[i], R[i], "p2 rotate l=%d" % lv[i])
    pf.pft_rescale_batch(ctx, C, C)
    for i in range(len(lv)):
        p2.assert_equal(C[i], o.rescale(R[i]), "p2 rescale l=%d" % lv[i])


def test_p2_keys_match(p2):
    assert np.array_equal(p2.pft.pft_key_export(p2.ctx, 0), p2.orc.keys[0])


def test_job_queue_two_rings_full_size(p2, gpu):
    """One persistent launch over the benchmark ring (N = 2^16, levels 30 and 11) and an
    N = 2^15 ring (60 + 17 x 40 bits, level 18), with a dependent job: bit for bit against the
    oracle's HADD / HMULPLAIN."""
    from oracle.ckks import Plaintext

    q = Pair(gpu, 15, 18, 2, 2, first_bits=60, mid_bits=40, special_bits=60, seed=(0x15, 1, 2, 3),
             relin=False, gpu_keys=False, insecure=False)
    try:
        pf, jobs, checks = p2.pft, [], []
        for p, lvl, tag in ((p2, 30, 300), (q, 18, 400), (p2, 11, 500)):
            o = p.orc
            x = o.encrypt_sk(o.encode(synth.slots(tag, 256), level=lvl), tag)
            y = o.encrypt_sk(o.encode(synth.slots(tag + 1, 256), level=lvl), tag + 1)
            pt = o.encode(synth.slots(tag + 2, 256), scale=2.0 ** 30, level=lvl)
            gx, gy, gp = p.ct(x), p.ct(y), p.pt(pt)
            s_, m_ = p.empty(), p.empty()
            jobs += [dict(op=pf.PFT_JOB_ADD, a=gx, b=gy, out=s_),
                     dict(op=pf.PFT_JOB_MUL_PLAIN, a=s_, p=gp, out=m_, after=len(jobs))]
            s = o.add(x, y)
            checks += [(p, s_, s, "add"), (p, m_, o.mul_plain(s, Plaintext(pt.m, pt.scale)), "mul_plain")]
        pf.pft_run_jobs(p2.ctx, jobs)
        pf.pft_device_status(p2.ctx)
        for p, h, want, what in checks:
            p.assert_equal(h, want, "%s N=%d level %d" % (what, p.N, want.c.shape[1]))
    finally:
        q.close()


@pytest.fixture(scope="module")
def p3(gpu):
    steps = [1 << i for i in range(15)]
    p = Pair(gpu, 16, 3, 4, 4, first_bits=60, mid_bits=40, special_bits=60, scale=2.0 ** 40,
             seed=(0xF00D, 1, 2, 3), rot_steps=steps, insecure=False)
    yield p
    p.close()


def test_fasttext_two_columns_bit_exact_n16(p3):
    o, pf, ctx = p3.orc, p3.pft, p3.ctx
    t = p3.N // 2
    m, n, c = t, 2, 14
    H, O = synth.fasttext_weights(31, m, n, c)
    docs = synth.documents(32, m, 1)
    Hp, Opk = OF.pack_H(H, t), OF.pack_O(O, t)
    H_o = [[o.encode(Hp[j, 0], level=3)] for j in range(n)]
    O_o = [o.encode(Opk[j], level=2) for j in range(n)]
    model = pf.pft_ft_model_import(ctx, [p3.pt(H_o[j][0]) for j in range(n)], [p3.pt(x) for x in O_o], m, n, c)
    try:
        v = o.encrypt_sk(o.encode(docs[0], level=3), 4242)
        s = p3.empty()
        pf.pft_fasttext_infer(ctx, model, [p3.ct(v)], s)
        want = OF.encrypted_scores(o, [v], H_o, O_o)
        p3.assert_equal(s, want, "fasttext n16 two columns")
        dec = o.decode(o.decrypt(want))[:c].real
        assert np.max(np.abs(dec - OF.plain_scores(docs[0], H, O))) < 2.0 ** -20
    finally:
        pf.pft_ft_model_destroy(model)


def test_fasttext_full_model_batched_tolerance(p3):
    """Vocabulary 32768, embedding 64, 14 classes; 4 documents in one batched call."""
    pf, ctx = p3.pft, p3.ctx
    t = p3.N // 2
    m, n, c = 32768, 64, 14
    H, O = synth.fasttext_weights(41, m, n, c)
    docs = synth.documents(42, m, 4)
    model = pf.pft_ft_model_create(ctx, H, O, 3)
    try:
        vs = []
        for d in range(4):
            pt = pf.pft_encode(ctx, docs[d], 2.0 ** 40, 3)
            vs.append(pf.pft_encrypt(ctx, pt, pf.PFT_ENC_SK, 7000 + d))
            pf.pft_pt_destroy(pt)
        scores = [p3.empty() for _ in range(4)]
        pf.pft_fasttext_infer_batch(ctx, model, vs, 1, scores)
        for d in range(4):
            dec = pf.pft_decrypt(ctx, scores[d])
            got = pf.pft_decode(ctx, dec, t)[:c].real
            pf.pft_pt_destroy(dec)
            want = OF.plain_scores(docs[d], H, O)
            assert np.max(np.abs(got - want)) < 2.0 ** -20, np.max(np.abs(got - want))
            srt = np.sort(want)
            if srt[-1] - srt[-2] >= 2.0 ** -18:
                assert int(np.argmax(got)) == int(np.argmax(want))
        for h in vs:
            pf.pft_ct_destroy(h)
    finally:
        pf.pft_ft_model_destroy(model)


def test_fasttext_diagonal_full_model_batched_tolerance(p3):
    """Rotation-light variant on the 32768 x 64 x 14 model: 4 documents in one call, scores in
    slots 64 c, within 2^-20 of the FP64 Algorithm 1.  The input is rotated before its
    plaintext product, so it is encrypted at scale 2^50 to keep key-switching noise small."""
    pf, ctx = p3.pft, p3.ctx
    t = p3.N // 2
    m, n, c = 32768, 64, 14
    pf.pft_add_rotation_keys(ctx, list(range(1, n)) + [n << s for s in range(9)])
    H, O = synth.fasttext_weights(43, m, n, c)
    docs = synth.documents(44, m, 4)
    model = pf.pft_ft_model_create_diag(ctx, H, O, 3)
    try:
        vs = []
        for d in range(4):
            pt = pf.pft_encode(ctx, docs[d], 2.0 ** 50, 3)
            vs.append(pf.pft_encrypt(ctx, pt, pf.PFT_ENC_SK, 8000 + d))
            pf.pft_pt_destroy(pt)
        scores = [p3.empty() for _ in range(4)]
        pf.pft_fasttext_infer_batch(ctx, model, vs, 1, scores)
        for d in range(4):
            dec = pf.pft_decrypt(ctx, scores[d])
            got = pf.pft_decode(ctx, dec, t).real[[n * cc for cc in range(c)]]
            pf.pft_pt_destroy(dec)
            want = OF.plain_scores(docs[d], H, O)
            assert np.max(np.abs(got - want)) < 2.0 ** -20, np.max(np.abs(got - want))
            srt = np.sort(want)
            if srt[-1] - srt[-2] >= 2.0 ** -18:  # the predicted class, unless two scores tie
                assert int(np.argmax(got)) == int(np.argmax(want))
        for h in vs:
            pf.pft_ct_destroy(h)
    finally:
        pf.pft_ft_model_destroy(model)


def test_training_step_full_size_vs_fp64(gpu):
    """Encrypted minibatch step at the training workload's sizes (vocabulary 8192 in one
    N = 2^16 ciphertext, dimension 32, 4 classes; 60 + 29 x 40-bit chain, 4 special primes,
    digits of 4) on 4 documents: decrypted gradients and updated weights within 2^-20 of FP64."""
    from oracle import fasttext as OF

    pf = gpu
    L, m, n, c, B, eta, sc = 30, 8192, 32, 4, 4, 0.25, 2.0 ** 40
    ctx = pf.pft_ctx_create(16, L, 4, 4, 60, 40, 60, sc, (0x7A11, 1, 2, 3))
    handles = []

    def enc(z, level, scale, nonce):
        pt = pf.pft_encode(ctx, z, scale, level)
        h = pf.pft_encrypt(ctx, pt, pf.PFT_ENC_SK, nonce)
        pf.pft_pt_destroy(pt)
        handles.append(h)
        return h

    def dec(h, k):
        pt = pf.pft_decrypt(ctx, h)
        z = pf.pft_decode(ctx, pt, k).real
        pf.pft_pt_destroy(pt)
        return z

    try:
        pf.pft_keygen(ctx, [1 << i for i in range(15)], True)
        H, O = synth.fasttext_weights(51, m, n, c)
        V = synth.documents(52, m, B)
        Y = np.eye(c)[np.random.default_rng(53).integers(0, c, B)]
        model = pf.pft_ft_enc_model_create(ctx, [enc(H[:, j], L, sc, 10 + j) for j in range(n)],
                                           [enc(O[j], L - 1, sc, 100 + j) for j in range(n)], m, n, c)
        try:
            dl, ll, ls = pf.pft_fasttext_train_spec(ctx, model, sc)
            docs = [enc(V[b], dl, sc, 200 + b) for b in range(B)]
            labels = [enc(Y[b] - 0.25, ll, ls, 300 + b) for b in range(B)]
            gH = [pf.pft_ct_create(ctx) for _ in range(n)]
            gO = [pf.pft_ct_create(ctx) for _ in range(n)]
            handles.extend(gH + gO)
            pf.pft_fasttext_train_step(ctx, model, docs, labels, eta, gH, gO)
            ref_H, ref_O = OF.train_grads_plain(V, Y, H, O)
            got_H = np.stack([dec(gH[j], m) for j in range(n)], 1)
            got_O = np.stack([dec(gO[j], c) for j in range(n)])
            assert np.max(np.abs(got_H - ref_H)) < 2.0 ** -20, np.max(np.abs(got_H - ref_H))
            assert np.max(np.abs(got_O - ref_O)) < 2.0 ** -20, np.max(np.abs(got_O - ref_O))
            assert pf.pft_ft_enc_model_levels(model) == (L - 6, L - 5)
            for j in (0, n - 1):
                for which, want in ((0, H[:, j] - eta * ref_H[:, j]), (1, O[j] - eta * ref_O[j])):
                    w = pf.pft_ct_create(ctx)
                    handles.append(w)
                    pf.pft_ft_enc_model_get(ctx, model, which, j, w)
                    got = dec(w, want.size)
                    assert np.max(np.abs(got - want)) < 2.0 ** -20
        finally:
            pf.pft_ft_enc_model_destroy(model)
    finally:
        for h in handles:
            pf.pft_ct_destroy(h)
        pf.pft_ctx_destroy(ctx)


def test_rotation_light_training_step_full_size_vs_fp64(gpu):
    """The diagonal-layout step at the same sizes, documents lifted by 2^10 (mask at 2^30):
    decrypted diagonals of dH, dO in the layout of P and the updated weights within 2^-20 of
    FP64; the model ends at levels L - 7 (diagonals) and L - 8 (P)."""
    from oracle import fasttext as OF

    pf = gpu
    L, m, n, c, B, eta, sc, lift = 30, 8192, 32, 4, 4, 0.25, 2.0 ** 40, 10
    ctx = pf.pft_ctx_create(16, L, 4, 4, 60, 40, 60, sc, (0x7A12, 1, 2, 3))
    t = 1 << 15
    handles = []

    def enc(z, level, scale, nonce):
        pt = pf.pft_encode(ctx, z, scale, level)
        h = pf.pft_encrypt(ctx, pt, pf.PFT_ENC_SK, nonce)
        pf.pft_pt_destroy(pt)
        handles.append(h)
        return h

    def dec(h, k):
        pt = pf.pft_decrypt(ctx, h)
        z = pf.pft_decode(ctx, pt, k).real
        pf.pft_pt_destroy(pt)
        return z

    mask = None
    try:
        pf.pft_keygen(ctx, [1 << i for i in range(15)] + [k for k in range(3, n) if k & (k - 1)]
                      + [-(1 << s) for s in range(5)], True)
        H, O = synth.fasttext_weights(54, m, n, c)
        V = np.zeros((B, t))
        V[:, :m] = synth.documents(55, m, B)
        Y = np.eye(c)[np.random.default_rng(56).integers(0, c, B)]
        D, P, Mv = OF.train_pack_diag(np.vstack([H, np.zeros((t - m, n))]), O, t)
        mask = pf.pft_encode(ctx, Mv, sc / 2.0 ** lift, L)
        model = pf.pft_ft_enc_model_create_diag(ctx, [enc(D[k], L, sc, 10 + k) for k in range(n)],
                                                enc(P, L - 1, sc, 100), mask, m, n, c, lift)
        try:
            dl, ll, ls = pf.pft_fasttext_train_spec(ctx, model, sc)
            docs = [enc(V[b], dl, sc, 200 + b) for b in range(B)]
            labels = [enc(OF.train_label_diag(Y[b], n, t), ll, ls, 300 + b) for b in range(B)]
            gD = [pf.pft_ct_create(ctx) for _ in range(n)]
            gP = [pf.pft_ct_create(ctx)]
            handles.extend(gD + gP)
            pf.pft_fasttext_train_step(ctx, model, docs, labels, eta, gD, gP)
            ref_H, ref_O = OF.train_grads_plain(V[:, :m], Y, H, O)
            ref_D, ref_P, _ = OF.train_pack_diag(np.vstack([ref_H, np.zeros((t - m, n))]), ref_O, t)
            for k in range(n):
                assert np.max(np.abs(dec(gD[k], t) - ref_D[k])) < 2.0 ** -20, k
            assert np.max(np.abs(dec(gP[0], n * c) - ref_P[:n * c])) < 2.0 ** -20
            assert pf.pft_ft_enc_model_levels(model) == (L - 7, L - 8)
            for which, j, want in ((0, 0, D[0] - eta * ref_D[0]), (0, n - 1, D[n - 1] - eta * ref_D[n - 1]),
                                   (1, 0, (P - eta * ref_P)[:n * c])):
                w = pf.pft_ct_create(ctx)
                handles.append(w)
                pf.pft_ft_enc_model_get(ctx, model, which, j, w)
                assert np.max(np.abs(dec(w, want.size) - want)) < 2.0 ** -20, (which, j)
        finally:
            pf.pft_ft_enc_model_destroy(model)
    finally:
        if mask is not None:
            pf.pft_pt_destroy(mask)
        for h in handles:
            pf.pft_ct_destroy(h)
        pf.pft_ctx_destroy(ctx)
