"""GPU (through the C ABI) against the oracle, element by element.

Bar: bit-exact canonical residues in coefficient form for every integer result
(keys, encryptions, HADD, HMULPLAIN, HMUL+relinearisation, ROTATE, RESCALE,
TotalSum, the fastText sequence); encoding within one unit per coefficient (it is
FP64 and the two sides use different FFTs); decrypted scores within 2^-20 of the
FP64 plaintext computation.  Sizes: N = 2^12 (one-pass transform) and N = 2^16
(two-pass transform, several tiles, digits with a ragged last one)."""
import numpy as np
import pytest

from oracle import _lib as OC
from oracle import ckks as OK
from oracle import fasttext as OF
from oracle import params as OP
from paper_1908_06972_gb300 import synth

from .pairs import Pair

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def p1(gpu):
    # toy smoke-test chain: N = 2^12, q0 60-bit, two 40-bit primes, one 60-bit special prime,
    # one prime per digit (the paper's "one key holds l ciphertexts" structure)
    p = Pair(gpu, 12, 3, 1, 1, rot_steps=[1, -1, 2, 4, 8, 16, 32, 64, 128, 256, 512, 1024, 3, 5, 6, 7])
    yield p
    p.close()


@pytest.fixture(scope="module")
def p16(gpu):
    # N = 2^16, 6 primes (60 + 5 x 50), 2 special, digits of 4 primes (last digit ragged)
    p = Pair(gpu, 16, 6, 2, 4, mid_bits=50, rot_steps=[1, 5, -1])
    yield p
    p.close()


# ---- transform layout ---------------------------------------------------------------------
@pytest.mark.parametrize("logn", [12, 16])
def test_ntt_layout_matches_definition(gpu, logn):
    import torch
    p = Pair(gpu, logn, 2, 1, 1, gpu_keys=False, rot_steps=())
    try:
        info = gpu.pft_ctx_info(p.ctx)
        primes = info["primes"]
        n = 1 << logn
        x = synth.residues(5, primes, n, polys=2)  # 2 polys x 3 rows (2 q's + 1 special)
        x[0, 0, :4] = [0, 1, primes[0] - 1, 0]
        t = torch.from_numpy(x.view(np.int64).copy()).cuda()
        gpu.pft_ntt(p.ctx, t.data_ptr(), 2, 3, 0)
        y = t.cpu().numpy().view(np.uint64)
        idx = np.arange(n) if logn <= 12 else np.r_[0:64, n // 2 - 32:n // 2 + 32, n - 64:n]
        for poly in range(2):
            for r, q in enumerate(primes):
                want = OC.eval_at(x[poly, r], OP.root_2n(q, logn), q, logn, idx)
                assert np.array_equal(y[poly, r][idx], want), (poly, r)
        gpu.pft_ntt(p.ctx, t.data_ptr(), 2, 3, 1)
        assert np.array_equal(t.cpu().numpy().view(np.uint64), x)
    finally:
        p.close()


# ---- keys and encryption ---------------------------------------------------------------------
def test_keys_bit_exact(p1):
    assert np.array_equal(p1.pft.pft_secret_export(p1.ctx), p1.orc.s)
    assert np.array_equal(p1.pft.pft_key_export(p1.ctx, 0), p1.orc.keys[0])
    g = OK.galois_element(1, p1.N)
    assert np.array_equal(p1.pft.pft_key_export(p1.ctx, g), p1.orc.keys[g])


def test_keys_bit_exact_n16(p16):
    assert np.array_equal(p16.pft.pft_key_export(p16.ctx, 0), p16.orc.keys[0])
    g = OK.galois_element(5, p16.N)
    assert np.array_equal(p16.pft.pft_key_export(p16.ctx, g), p16.orc.keys[g])


@pytest.mark.parametrize("level", [3, 2, 1])
def test_encrypt_bit_exact(p1, level):
    o = p1.orc
    pt_o = o.encode(synth.slots(level, p1.N // 2), level=level)
    pt_g = p1.pt(pt_o)
    for mode, fn in ((p1.pft.PFT_ENC_SK, o.encrypt_sk), (p1.pft.PFT_ENC_PK, o.encrypt_pk)):
        h = p1.pft.pft_encrypt(p1.ctx, pt_g, mode, 77 + level)
        p1.handles.append(("ct", h))
        p1.assert_equal(h, fn(pt_o, 77 + level), "encrypt mode %d" % mode)
        dec = p1.pft.pft_decrypt(p1.ctx, h)
        p1.handles.append(("pt", dec))
        assert np.array_equal(p1.pft.pft_pt_export(p1.ctx, dec), o.decrypt(fn(pt_o, 77 + level)).m)


def test_encode_within_one_unit(p1):
    z = synth.slots(3, p1.N // 2)
    h = p1.pft.pft_encode(p1.ctx, z, 2.0 ** 40, 3)
    p1.handles.append(("pt", h))
    got = OK.crt_centered(p1.pft.pft_pt_export(p1.ctx, h), p1.orc.q[:3])
    want = OK.crt_centered(p1.orc.encode(z).m, p1.orc.q[:3])
    diff = np.array([abs(int(a) - int(b)) for a, b in zip(got, want)])
    assert diff.max() <= 1
    assert (diff > 0).sum() <= p1.N // 100
    zz = p1.pft.pft_decode(p1.ctx, h, p1.N // 2)
    assert np.max(np.abs(zz - z)) < 2.0 ** -30


# ---- operations -------------------------------------------------------------------------------
@pytest.fixture(scope="module")
def cts1(p1):
    o = p1.orc
    za, zb = synth.slots(101, p1.N // 2), synth.slots(102, p1.N // 2)
    a, b = o.encrypt_sk(o.encode(za), 1), o.encrypt_pk(o.encode(zb), 2)
    return za, zb, a, b


def test_add_sub_plain_ops_bit_exact(p1, cts1):
    o, pf, ctx = p1.orc, p1.pft, p1.ctx
    za, zb, a, b = cts1
    ga, gb = p1.ct(a), p1.ct(b)
    out = p1.empty()
    pf.pft_add(ctx, ga, gb, out)
    p1.assert_equal(out, o.add(a, b), "add")
    pf.pft_sub(ctx, ga, gb, out)
    p1.assert_equal(out, o.sub(a, b), "sub")
    ptb = o.encode(zb)
    gp = p1.pt(ptb)
    pf.pft_mul_plain(ctx, ga, gp, out)
    p1.assert_equal(out, o.mul_plain(a, ptb), "mul_plain")
    pf.pft_add_plain(ctx, ga, gp, out)
    p1.assert_equal(out, o.add_plain(a, ptb), "add_plain")


def test_mul_relin_rescale_rotate_bit_exact(p1, cts1):
    o, pf, ctx = p1.orc, p1.pft, p1.ctx
    za, zb, a, b = cts1
    ga, gb = p1.ct(a), p1.ct(b)
    m = p1.empty()
    pf.pft_mul_relin(ctx, ga, gb, m)
    mo = o.mul_relin(a, b)
    p1.assert_equal(m, mo, "mul_relin")
    r = p1.empty()
    pf.pft_rescale(ctx, m, r)
    ro = o.rescale(mo)
    p1.assert_equal(r, ro, "rescale")
    # rescale again (level 2 -> 1), in place (output aliases input)
    pf.pft_rescale(ctx, r, r)
    p1.assert_equal(r, o.rescale(ro), "rescale in place")
    for step in (1, -1, 3):
        rt = p1.empty()
        pf.pft_rotate(ctx, ga, step, rt)
        p1.assert_equal(rt, o.rotate(a, step), "rotate %d" % step)
    # decrypted meaning (Sec. 2.3): z_a z_b after mul+rescale, left rotation
    dec = pf.pft_decrypt(ctx, p1.ct(ro))
    p1.handles.append(("pt", dec))
    assert np.max(np.abs(pf.pft_decode(ctx, dec, p1.N // 2) - za * zb)) < 2.0 ** -20


def test_in_place_ops(p1, cts1):
    o, pf, ctx = p1.orc, p1.pft, p1.ctx
    za, zb, a, b = cts1
    ga, gb = p1.ct(a), p1.ct(b)
    pf.pft_mul_relin(ctx, ga, gb, ga)
    p1.assert_equal(ga, o.mul_relin(a, b), "mul_relin in place")
    gb2 = p1.ct(b)
    pf.pft_rotate(ctx, gb2, 1, gb2)
    p1.assert_equal(gb2, o.rotate(b, 1), "rotate in place")


def test_errors(p1, cts1):
    pf, ctx = p1.pft, p1.ctx
    za, zb, a, b = cts1
    ga = p1.ct(a)
    low = p1.ct(p1.orc.rescale(a))
    out = p1.empty()
    with pytest.raises(pf.PftError) as e:
        pf.pft_add(ctx, ga, low, out)
    assert e.value.code == pf.PFT_ERR_LEVEL_MISMATCH
    with pytest.raises(pf.PftError) as e:
        pf.pft_rotate(ctx, ga, 9, out)
    assert e.value.code == pf.PFT_ERR_NO_KEY
    with pytest.raises(pf.PftError) as e:
        pf.pft_fasttext_train_step(ctx, None, [], [], 0.0)
    assert e.value.code == pf.PFT_ERR_ARG


def test_batched_uneven_levels(p1):
    o, pf, ctx = p1.orc, p1.pft, p1.ctx
    A, B = [], []
    for i, lvl in enumerate([3, 2, 3, 1, 2]):
        A.append(o.encrypt_sk(o.encode(synth.slots(200 + i, 64), level=lvl), 300 + i))
        B.append(o.encrypt_sk(o.encode(synth.slots(400 + i, 64), level=lvl), 500 + i))
    gA, gB = [p1.ct(x) for x in A], [p1.ct(x) for x in B]
    outs = [p1.empty() for _ in A]
    pf.pft_mul_relin_batch(ctx, gA, gB, outs)
    for i in range(len(A)):
        p1.assert_equal(outs[i], o.mul_relin(A[i], B[i]), "batch mul_relin %d" % i)
    rots = [p1.empty() for _ in A]
    pf.pft_rotate_batch(ctx, gA, -1, rots)
    for i in range(len(A)):
        p1.assert_equal(rots[i], o.rotate(A[i], -1), "batch rotate %d" % i)
    keep = [i for i in range(len(A)) if A[i].level >= 2]
    res = [p1.empty() for _ in keep]
    pf.pft_rescale_batch(ctx, [gA[i] for i in keep], res)
    for j, i in enumerate(keep):
        p1.assert_equal(res[j], o.rescale(A[i]), "batch rescale %d" % i)


def test_total_sum_and_fasttext_n12(p1):
    o, pf, ctx = p1.orc, p1.pft, p1.ctx
    t = p1.N // 2
    m, n, c = t, 4, 3
    H, O = synth.fasttext_weights(9, m, n, c)
    docs = synth.documents(10, m, 2, 20, 60)
    Hp, Opk = OF.pack_H(H, t), OF.pack_O(O, t)
    H_o = [[o.encode(Hp[j, 0], level=3)] for j in range(n)]
    O_o = [o.encode(Opk[j], level=2) for j in range(n)]
    model = pf.pft_ft_model_import(ctx, [p1.pt(H_o[j][0]) for j in range(n)], [p1.pt(x) for x in O_o], m, n, c)
    try:
        v_o = [o.encrypt_sk(o.encode(docs[d], level=3), 900 + d) for d in range(2)]
        v_g = [p1.ct(x) for x in v_o]
        scores = [p1.empty() for _ in range(2)]
        pf.pft_fasttext_infer_batch(ctx, model, v_g, 1, scores)
        one = p1.empty()
        pf.pft_fasttext_infer(ctx, model, [v_g[1]], one)
        for d in range(2):
            want = OF.encrypted_scores(o, [v_o[d]], H_o, O_o)
            p1.assert_equal(scores[d], want, "fasttext doc %d" % d)
            dec = o.decode(o.decrypt(want))[:c].real
            assert np.max(np.abs(dec - OF.plain_scores(docs[d], H, O))) < 2.0 ** -20
        p1.assert_equal(one, OF.encrypted_scores(o, [v_o[1]], H_o, O_o), "fasttext single")
    finally:
        pf.pft_ft_model_destroy(model)


# ---- N = 2^16 ---------------------------------------------------------------------------------
def test_ops_bit_exact_n15(gpu):
    """N = 2^15 (the smaller ring of the serving workload): 60 + 3 x 40-bit primes, two
    special primes, digits of two primes; generic two-pass transform (stages 8 + 7)."""
    p = Pair(gpu, 15, 4, 2, 2, rot_steps=[1, -3])
    try:
        o, pf, ctx = p.orc, p.pft, p.ctx
        assert np.array_equal(pf.pft_key_export(ctx, 0), o.keys[0])
        za, zb = synth.slots(31, 2048), synth.slots(32, 2048)
        for lvl in (4, 3):
            a = o.encrypt_sk(o.encode(za, level=lvl), 40 + lvl)
            b = o.encrypt_pk(o.encode(zb, level=lvl), 50 + lvl)
            ga, gb = p.ct(a), p.ct(b)
            m = p.empty()
            pf.pft_mul_relin(ctx, ga, gb, m)
            mo = o.mul_relin(a, b)
            p.assert_equal(m, mo, "mul_relin n15 l=%d" % lvl)
            r = p.empty()
            pf.pft_rescale(ctx, m, r)
            p.assert_equal(r, o.rescale(mo), "rescale n15 l=%d" % lvl)
            rt = p.empty()
            pf.pft_rotate(ctx, ga, -3, rt)
            p.assert_equal(rt, o.rotate(a, -3), "rotate n15 l=%d" % lvl)
    finally:
        p.close()


def test_ops_bit_exact_n16(p16):
    o, pf, ctx = p16.orc, p16.pft, p16.ctx
    za, zb = synth.slots(1, 4096), synth.slots(2, 4096)
    for lvl in (6, 5, 2):
        a = o.encrypt_sk(o.encode(za, level=lvl), 10 + lvl)
        b = o.encrypt_pk(o.encode(zb, level=lvl), 20 + lvl)
        ga, gb = p16.ct(a), p16.ct(b)
        m = p16.empty()
        pf.pft_mul_relin(ctx, ga, gb, m)
        mo = o.mul_relin(a, b)
        p16.assert_equal(m, mo, "mul_relin n16 l=%d" % lvl)
        r = p16.empty()
        pf.pft_rescale(ctx, m, r)
        p16.assert_equal(r, o.rescale(mo), "rescale n16 l=%d" % lvl)
        rt = p16.empty()
        pf.pft_rotate(ctx, ga, 5, rt)
        p16.assert_equal(rt, o.rotate(a, 5), "rotate n16 l=%d" % lvl)


def test_batched_import_export_round_trip(p1):
    o, pf = p1.orc, p1.pft
    cts = [o.encrypt_sk(o.encode(synth.slots(900 + i, 64), level=lvl), 600 + i) for i, lvl in enumerate([3, 1, 2])]
    hs = pf.pft_ct_import_batch(p1.ctx, [c.c for c in cts], [c.scale for c in cts])
    p1.handles += [("ct", h) for h in hs]
    for c, h in zip(cts, hs):
        p1.assert_equal(h, c, "import_batch")
    outs = [np.zeros_like(c.c) for c in cts]
    pf.pft_ct_export_batch(p1.ctx, hs, outs)
    for c, arr in zip(cts, outs):
        assert np.array_equal(arr, c.c)
    # asynchronous form into page-locked buffers, read after the stream has caught up
    import torch
    pinned = [torch.zeros(c.c.shape, dtype=torch.int64, pin_memory=True).numpy().view(np.uint64) for c in cts]
    pf.pft_ct_export_batch_async(p1.ctx, hs, pinned)
    torch.cuda.synchronize()
    for c, arr in zip(cts, pinned):
        assert np.array_equal(arr, c.c)
    # into existing handles: buffers reused (same addresses) when large enough, levels may change
    ptr = [pf.pft_ct_data(h) for h in hs]
    new = [o.encrypt_sk(o.encode(synth.slots(950 + i, 64), level=lvl), 650 + i) for i, lvl in enumerate([2, 1, 2])]
    pf.pft_ct_import_batch_into(p1.ctx, [c.c for c in new], [c.scale for c in new], hs)
    for c, h in zip(new, hs):
        p1.assert_equal(h, c, "import_batch_into")
    assert [pf.pft_ct_data(h) for h in hs] == ptr
    with pytest.raises(pf.PftError) as e:  # one handle twice
        pf.pft_ct_import_batch_into(p1.ctx, [c.c for c in new[:2]], [c.scale for c in new[:2]], [hs[0], hs[0]])
    assert e.value.code == pf.PFT_ERR_ARG


def test_graph_replay_matches_oracle(gpu):
    """A captured batched step (mul_relin then rotate) replayed twice equals the oracle."""
    import torch
    from oracle import ckks as K

    pf = gpu
    stream = torch.cuda.Stream()
    seed = (0x5EED, 11, 22, 33)
    orc = K.Oracle(12, 3, 1, 1, 60, 40, 60, 2.0 ** 40, seed)
    orc.keygen([1], True)
    ctx = pf.pft_ctx_create(12, 3, 1, 1, 60, 40, 60, 2.0 ** 40, seed, flags=pf.PFT_ALLOW_INSECURE, allocator=None,
                            stream=stream.cuda_stream)
    graph = None
    hs = []
    try:
        pf.pft_keygen(ctx, [1], True)
        A = [orc.encrypt_sk(orc.encode(synth.slots(70 + i, 64), level=lvl), 80 + i) for i, lvl in enumerate([3, 2])]
        B = [orc.encrypt_sk(orc.encode(synth.slots(90 + i, 64), level=lvl), 95 + i) for i, lvl in enumerate([3, 2])]
        gA = [pf.pft_ct_import(ctx, x.c, x.scale) for x in A]
        gB = [pf.pft_ct_import(ctx, x.c, x.scale) for x in B]
        C = [pf.pft_ct_create(ctx) for _ in A]
        hs = gA + gB + C
        pf.pft_mul_relin_batch(ctx, gA, gB, C)  # eager warm-up sizes the outputs
        pf.pft_rotate_batch(ctx, C, 1, C)
        pf.pft_graph_begin(ctx)
        pf.pft_mul_relin_batch(ctx, gA, gB, C)
        pf.pft_rotate_batch(ctx, C, 1, C)
        graph = pf.pft_graph_end(ctx)
        want = [orc.rotate(orc.mul_relin(a, b), 1) for a, b in zip(A, B)]
        for _ in range(2):
            pf.pft_graph_launch(ctx, graph)
            for h, w in zip(C, want):
                assert np.array_equal(pf.pft_ct_export(ctx, h), w.c)
    finally:
        if graph is not None:
            pf.pft_graph_destroy(graph)
        for h in hs:
            pf.pft_ct_destroy(h)
        pf.pft_ctx_destroy(ctx)


def test_every_transform_variant_bit_exact(p16):
    """pft_autotune searches the N = 2^16 transform plans per launch size; every plan (and so
    every choice it can make) gives the same bits, and so does every fixed variant."""
    o, pf, ctx = p16.orc, p16.pft, p16.ctx
    chosen, us = pf.pft_autotune(ctx)
    rep = pf.pft_autotune_report(ctx)
    names = list(rep["buckets"][-1]["us_fwd_inv"])
    assert rep["N"] == p16.N and len(rep["buckets"]) == 3 and len(names) >= 8
    assert 0 <= chosen < len(names) and all(u > 0 for u in us[:len(names)])
    for b in rep["buckets"]:
        assert b["chosen"] in b["us_fwd_inv"] and b["us_fwd_inv"][b["chosen"]] == min(b["us_fwd_inv"].values())
    a = o.encrypt_sk(o.encode(synth.slots(31, 512), level=6), 41)
    b = o.encrypt_sk(o.encode(synth.slots(32, 512), level=6), 42)
    want = o.mul_relin(a, b)
    ga, gb = p16.ct(a), p16.ct(b)
    for v in range(len(names)):
        pf.pft_set_transform_plan(ctx, v)
        m = p16.empty()
        pf.pft_mul_relin(ctx, ga, gb, m)
        p16.assert_equal(m, want, "mul_relin with transform plan %s" % names[v])
    for v in range(pf.PFT_NTT16_VARIANTS):
        pf.pft_set_transform_variant(ctx, v)
        m = p16.empty()
        pf.pft_mul_relin(ctx, ga, gb, m)
        p16.assert_equal(m, want, "mul_relin with transform variant %d" % v)
    pf.pft_set_transform_variant(ctx, 0)


@pytest.mark.parametrize("which", ["p1", "p16"])
def test_hoisted_rotations_bit_exact(which, request):
    p = request.getfixturevalue(which)
    o, pf, ctx = p.orc, p.pft, p.ctx
    steps = [1, -1] if which == "p16" else [1, 2, -1, 3, 1024]
    lvl = o.L if which == "p1" else 5
    a = o.encrypt_sk(o.encode(synth.slots(55, 256), level=lvl), 56)
    ga = p.ct(a)
    outs = [p.empty() for _ in steps]
    pf.pft_rotate_hoisted(ctx, ga, steps, outs)
    for h, w, st in zip(outs, o.rotate_hoisted(a, steps), steps):
        p.assert_equal(h, w, "hoisted rotate %d" % st)


def test_fasttext_diagonal_bit_exact_n12(p1):
    """Rotation-light matvec (diagonal packing, hoisted rotations) against the oracle's sequence."""
    o, pf, ctx = p1.orc, p1.pft, p1.ctx
    t = p1.N // 2
    m, n, c = t - 100, 8, 3
    H, O = synth.fasttext_weights(19, m, n, c)
    v = np.zeros(t)
    v[:m] = synth.documents(20, m, 1, 20, 60)[0]
    D, P = OF.pack_diag(H, O, t)
    D_o = [o.encode(D[k], level=3) for k in range(n)]
    P_o = o.encode(P, level=2)
    model = pf.pft_ft_model_import_diag(ctx, [p1.pt(x) for x in D_o], p1.pt(P_o), m, n, c)
    try:
        v_o = o.encrypt_sk(o.encode(v, level=3), 123)
        s = p1.empty()
        pf.pft_fasttext_infer(ctx, model, [p1.ct(v_o)], s)
        want = OF.encrypted_scores_diag(o, v_o, D_o, P_o)
        p1.assert_equal(s, want, "fasttext diagonal")
        got = o.decode(o.decrypt(want)).real[OF.diag_score_slots(n, c)]
        assert np.max(np.abs(got - OF.plain_scores(v[:m], H, O))) < 2.0 ** -20
    finally:
        pf.pft_ft_model_destroy(model)


def test_fasttext_diagonal_chunks_bit_exact_n12(p1):
    """Rotation-light matvec for a vocabulary of 2.5 ciphertexts (diagonals and hoisted rotations
    per chunk), two documents in one call, against the oracle's sequence."""
    o, pf, ctx = p1.orc, p1.pft, p1.ctx
    t = p1.N // 2
    m, n, c = 2 * t + t // 2, 8, 3
    H, O = synth.fasttext_weights(21, m, n, c)
    docs = synth.documents(22, m, 2, 20, 60)
    D, P = OF.pack_diag_chunks(H, O, t)
    D_o = [[o.encode(D[i, k], level=3) for k in range(n)] for i in range(3)]
    P_o = o.encode(P, level=2)
    model = pf.pft_ft_model_import_diag(ctx, [p1.pt(D_o[i][k]) for i in range(3) for k in range(n)], p1.pt(P_o),
                                        m, n, c)
    try:
        v = np.zeros((2, 3 * t))
        v[:, :m] = docs
        v_o = [[o.encrypt_sk(o.encode(v[d, i * t:(i + 1) * t], level=3), 130 + 3 * d + i) for i in range(3)]
               for d in range(2)]
        scores = [p1.empty() for _ in range(2)]
        pf.pft_fasttext_infer_batch(ctx, model, [p1.ct(x) for d in range(2) for x in v_o[d]], 3, scores)
        for d in range(2):
            want = OF.encrypted_scores_diag_chunks(o, v_o[d], D_o, P_o)
            p1.assert_equal(scores[d], want, "fasttext diagonal, 3 chunks, doc %d" % d)
            got = o.decode(o.decrypt(want)).real[OF.diag_score_slots(n, c)]
            assert np.max(np.abs(got - OF.plain_scores(docs[d], H, O))) < 2.0 ** -20
    finally:
        pf.pft_ft_model_destroy(model)


def test_tensor_core_basis_conversion_bit_exact(gpu, monkeypatch):
    """The tensor-core form of the basis conversion (four source primes: ModUp digits of 4 and
    ModDown from 4 special primes; opt-in) gives the same bits: HMUL + relinearisation, rotation
    and a batch at mixed levels against the oracle at N = 2^16."""
    monkeypatch.setenv("PFT_BCONV", "tc")
    p = Pair(gpu, 16, 8, 4, 4, mid_bits=50, rot_steps=[1])
    monkeypatch.delenv("PFT_BCONV")
    try:
        o, pf, ctx = p.orc, p.pft, p.ctx
        lv = [8, 6, 5]
        A = [o.encrypt_sk(o.encode(synth.slots(70 + i, 256), level=l), 170 + i) for i, l in enumerate(lv)]
        B = [o.encrypt_pk(o.encode(synth.slots(80 + i, 256), level=l), 180 + i) for i, l in enumerate(lv)]
        gA, gB = [p.ct(x) for x in A], [p.ct(x) for x in B]
        C = [p.empty() for _ in lv]
        pf.pft_mul_relin_batch(ctx, gA, gB, C)
        M = [o.mul_relin(a, b) for a, b in zip(A, B)]
        for i in range(len(lv)):
            p.assert_equal(C[i], M[i], "tensor-core conversion: mul_relin level %d" % lv[i])
        pf.pft_rotate_batch(ctx, C, 1, C)
        for i in range(len(lv)):
            p.assert_equal(C[i], o.rotate(M[i], 1), "tensor-core conversion: rotate level %d" % lv[i])
    finally:
        p.close()



@pytest.mark.parametrize("order", [0, 5])
def test_transform_memory_order_flags_bit_exact(gpu, monkeypatch, order):
    """The memory-order switches of the N = 2^16 two-pass transforms (PFT_NTT_ORDER: reverse second
    pass, L2 policy of the row twiddles, prefetch of the ModDown epilogue's operands; the default
    turns all on) change no bit: HMUL + relinearisation and rotation of a mixed-level batch against
    the oracle with the switches off (0) and with two of them (5)."""
    monkeypatch.setenv("PFT_NTT_ORDER", str(order))
    p = Pair(gpu, 16, 8, 4, 4, mid_bits=50, rot_steps=[1])
    monkeypatch.delenv("PFT_NTT_ORDER")
    try:
        o, pf, ctx = p.orc, p.pft, p.ctx
        lv = [8, 5]
        A = [o.encrypt_sk(o.encode(synth.slots(90 + i, 256), level=l), 190 + i) for i, l in enumerate(lv)]
        B = [o.encrypt_sk(o.encode(synth.slots(95 + i, 256), level=l), 195 + i) for i, l in enumerate(lv)]
        gA, gB = [p.ct(x) for x in A], [p.ct(x) for x in B]
        C = [p.empty() for _ in lv]
        pf.pft_mul_relin_batch(ctx, gA, gB, C)
        M = [o.mul_relin(a, b) for a, b in zip(A, B)]
        for i in range(len(lv)):
            p.assert_equal(C[i], M[i], "order %d: mul_relin level %d" % (order, lv[i]))
        pf.pft_rotate_batch(ctx, C, 1, C)
        for i in range(len(lv)):
            p.assert_equal(C[i], o.rotate(M[i], 1), "order %d: rotate level %d" % (order, lv[i]))
    finally:
        p.close()

# ---- seeded compressed switching keys -----------------------------------------------------------
@pytest.mark.parametrize("logn,L,k,alpha,mid", [(12, 3, 1, 1, 40), (12, 10, 1, 1, 40), (16, 6, 2, 4, 50)])
def test_compressed_keys_bit_exact(gpu, logn, L, k, alpha, mid):
    """Keys keep only b_j; the key inner product regenerates a_j from the seed.  Keys (with a_j
    regenerated for export), HMUL + relinearisation, rotations (plain and hoisted) and a
    mixed-level batch against the oracle's compressed keys.  L = 10 with one prime per digit
    takes the inner-product kernel for more than 8 digits."""
    p = Pair(gpu, logn, L, k, alpha, mid_bits=mid, rot_steps=[1, 3], compressed=True)
    try:
        o, pf, ctx = p.orc, p.pft, p.ctx
        assert np.array_equal(pf.pft_key_export(ctx, 0), o.keys[0])
        g = OK.galois_element(3, p.N)
        assert np.array_equal(pf.pft_key_export(ctx, g), o.keys[g])
        n_slots = min(p.N // 2, 512)
        lv = [L, max(1, L - 2), max(1, L // 2)]
        A = [o.encrypt_sk(o.encode(synth.slots(60 + i, n_slots), level=l), 70 + i) for i, l in enumerate(lv)]
        B = [o.encrypt_pk(o.encode(synth.slots(80 + i, n_slots), level=l), 90 + i) for i, l in enumerate(lv)]
        gA, gB = [p.ct(x) for x in A], [p.ct(x) for x in B]
        C = [p.empty() for _ in lv]
        pf.pft_mul_relin_batch(ctx, gA, gB, C)
        M = [o.mul_relin(a, b) for a, b in zip(A, B)]
        for i in range(len(lv)):
            p.assert_equal(C[i], M[i], "compressed mul_relin l=%d" % lv[i])
        pf.pft_rotate_batch(ctx, C, 1, C)
        for i in range(len(lv)):
            p.assert_equal(C[i], o.rotate(M[i], 1), "compressed rotate l=%d" % lv[i])
        outs = [p.empty(), p.empty()]
        pf.pft_rotate_hoisted(ctx, gA[0], [1, 3], outs)
        want = o.rotate_hoisted(A[0], [1, 3])
        for i in range(2):
            p.assert_equal(outs[i], want[i], "compressed hoisted %d" % i)
    finally:
        p.close()


def test_bounded_wait_reports_timeout(p1):
    """A wait that cannot complete gives up after its poll limit and the host reads
    PFT_ERR_TIMEOUT; the flag is cleared and the context stays usable."""
    pf, ctx = p1.pft, p1.ctx
    pf.pft_device_status(ctx)  # clean before
    pf.pft_wait_selftest(ctx, 1000)
    with pytest.raises(pf.PftError) as e:
        pf.pft_device_status(ctx)
    assert e.value.code == pf.PFT_ERR_TIMEOUT
    pf.pft_device_status(ctx)  # cleared
    a = p1.orc.encrypt_sk(p1.orc.encode(synth.slots(5, 64), level=3), 5)
    g, out = p1.ct(a), p1.empty()
    pf.pft_mul_relin(ctx, g, g, out)
    p1.assert_equal(out, p1.orc.mul_relin(a, a), "after the self-test")
    pf.pft_device_status(ctx)
