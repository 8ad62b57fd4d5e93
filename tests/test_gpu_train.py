"""Encrypted minibatch training (Sec. 4.2, Algorithm 5) on the GPU against the oracle.

N = 2^12, 8 primes (60 + 7 x 40 bits), two special primes (P above every digit modulus, so
key-switching noise stays far below 2^-20), digits of 2.  Bit for bit: the level/scale
operations, the gradients and the updated model of the fused step, the same through the
torch.autograd path, and the fused step in tiles of one document.  Decrypted
gradients against the FP64 gradient and central finite differences of the FP64 loss."""
import os

import numpy as np
import pytest

from oracle import ckks as OK
from oracle import fasttext as OF

from .pairs import Pair

pytestmark = pytest.mark.gpu

B, M_VOCAB, N_COLS, N_CLS, ETA, L0 = 3, 300, 2, 2, 0.5, 8


@pytest.fixture(scope="module")
def pair(gpu):
    p = Pair(gpu, 12, 8, 2, 2, seed=(0x7B, 5, 6, 7), rot_steps=[1 << i for i in range(11)])
    yield p
    p.close()


@pytest.fixture(scope="module")
def data(pair):
    o, t = pair.orc, pair.N // 2
    rng = np.random.default_rng(21)
    V = np.zeros((B, M_VOCAB))
    for b in range(B):
        np.add.at(V[b], rng.integers(0, M_VOCAB, 30), 1.0)
        V[b] /= V[b].sum()
    Y = np.eye(N_CLS)[[0, 1, 1]]
    H = rng.normal(0, 0.1, (M_VOCAB, N_COLS))
    O = rng.normal(0, 0.1, (N_COLS, N_CLS))
    pad = lambda x: np.concatenate([x, np.zeros(t - x.size)])  # noqa: E731
    v = [o.encrypt_sk(o.encode(pad(V[b]), level=L0), 100 + b) for b in range(B)]
    Hc = [o.encrypt_sk(o.encode(pad(H[:, j]), level=L0), 200 + j) for j in range(N_COLS)]
    Oc = [o.encrypt_pk(o.encode(pad(O[j]), level=L0 - 1), 300 + j) for j in range(N_COLS)]
    lw, sw = OF.train_label_spec(o, L0, v[0].scale, Hc[0].scale, Oc[0].scale)
    w = [o.encrypt_sk(o.encode(pad(Y[b] - 0.25), scale=sw, level=lw), 400 + b) for b in range(B)]
    want = OF.encrypted_train_step(o, v, w, Hc, Oc, ETA)
    return dict(V=V, Y=Y, H=H, O=O, v=v, w=w, Hc=Hc, Oc=Oc, spec=(lw, sw), want=want)


def gpu_model(pair, d):
    pf = pair.pft
    return pf.pft_ft_enc_model_create(pair.ctx, [pair.ct(x) for x in d["Hc"]], [pair.ct(x) for x in d["Oc"]],
                                      M_VOCAB, N_COLS, N_CLS)


def check_model(pair, model, want_H, want_O, what):
    pf = pair.pft
    for j in range(N_COLS):
        for which, want in ((0, want_H[j]), (1, want_O[j])):
            h = pair.empty()
            pf.pft_ft_enc_model_get(pair.ctx, model, which, j, h)
            pair.assert_equal(h, want, "%s %s_%d" % (what, "HO"[which], j))


def test_level_scale_constant_ops_bit_exact(pair):
    o, pf, ctx = pair.orc, pair.pft, pair.ctx
    z = np.random.default_rng(4).uniform(-1, 1, 2048)
    a = o.encrypt_sk(o.encode(z, level=6), 55)
    g = pair.ct(a)
    out = pair.empty()
    pf.pft_drop_level(ctx, g, 3, out)
    pair.assert_equal(out, o.drop_level(a, 3), "drop_level")
    for val in (2.0, -0.5, 0.123456789):
        pf.pft_add_const(ctx, g, val, out)
        pair.assert_equal(out, o.add_const(a, val), "add_const %r" % val)
    cs = float(o.q[5])  # the prime a following rescale drops
    pf.pft_mul_const(ctx, g, 0.3, cs, out)
    pair.assert_equal(out, o.mul_const(a, 0.3, cs), "mul_const")
    pf.pft_mul_const(ctx, g, -1.75, 2.0 ** 20, out)
    pair.assert_equal(out, o.mul_const(a, -1.75, 2.0 ** 20), "mul_const negative")
    pf.pft_add_const(ctx, g, 1.0, g)  # in place
    pair.assert_equal(g, o.add_const(a, 1.0), "add_const in place")
    pf.pft_ct_set_scale(g, 2.0 ** 43)
    assert pf.pft_ct_scale(g) == 2.0 ** 43


def test_train_spec_matches_oracle(pair, data):
    pf = pair.pft
    model = gpu_model(pair, data)
    try:
        dl, ll, ls = pf.pft_fasttext_train_spec(pair.ctx, model, data["v"][0].scale)
        assert (dl, ll, ls) == (L0, data["spec"][0], data["spec"][1])
        assert pf.pft_ft_enc_model_levels(model) == (L0, L0 - 1)
    finally:
        pf.pft_ft_enc_model_destroy(model)


def run_fused(pair, d):
    pf = pair.pft
    model = gpu_model(pair, d)
    gH = [pair.empty() for _ in range(N_COLS)]
    gO = [pair.empty() for _ in range(N_COLS)]
    pf.pft_fasttext_train_step(pair.ctx, model, [pair.ct(x) for x in d["v"]], [pair.ct(x) for x in d["w"]], ETA,
                               gH, gO)
    return model, gH, gO


def test_fused_step_bit_exact(pair, data):
    pf = pair.pft
    dH, dO, H1, O1 = data["want"]
    model, gH, gO = run_fused(pair, data)
    try:
        for j in range(N_COLS):
            pair.assert_equal(gH[j], dH[j], "dH_%d" % j)
            pair.assert_equal(gO[j], dO[j], "dO_%d" % j)
        assert pf.pft_ft_enc_model_levels(model) == (L0 - 6, L0 - 5)
        check_model(pair, model, H1, O1, "updated")
    finally:
        pf.pft_ft_enc_model_destroy(model)


def test_fused_step_in_tiles_of_one_document(pair, data):
    pf = pair.pft
    dH, dO, H1, O1 = data["want"]
    os.environ["PFT_TRAIN_TILE"] = "1"
    try:
        model, gH, gO = run_fused(pair, data)
    finally:
        del os.environ["PFT_TRAIN_TILE"]
    try:
        for j in range(N_COLS):
            pair.assert_equal(gH[j], dH[j], "tiled dH_%d" % j)
            pair.assert_equal(gO[j], dO[j], "tiled dO_%d" % j)
        check_model(pair, model, H1, O1, "tiled updated")
    finally:
        pf.pft_ft_enc_model_destroy(model)


def test_autograd_path_bit_exact(pair, data):
    import torch

    from paper_1908_06972_gb300 import train as T

    pf = pair.pft
    dH, dO, H1, O1 = data["want"]
    m = T.EncryptedFastText(pair.ctx, [pair.ct(x) for x in data["Hc"]], [pair.ct(x) for x in data["Oc"]],
                            M_VOCAB, N_COLS, N_CLS)
    try:
        opt = T.EncryptedSGD(m, ETA)
        docs = [pair.ct(x) for x in data["v"]]
        labels = [pair.ct(x) for x in data["w"]]
        loss = m.loss(docs, labels)
        assert isinstance(loss, torch.Tensor) and loss.requires_grad
        loss.backward()
        for j in range(N_COLS):
            pair.assert_equal(m.grad_H[j], dH[j], "autograd dH_%d" % j)
            pair.assert_equal(m.grad_O[j], dO[j], "autograd dO_%d" % j)
        opt.step()
        check_model(pair, m.model, H1, O1, "autograd updated")
        opt.zero_grad()
        assert m.grad_H is None
    finally:
        m.close()


def test_scores_of_the_forward_pass(pair, data):
    """The tape's encrypted scores decrypt to s = v H O."""
    pf, o = pair.pft, pair.orc
    model = gpu_model(pair, data)
    try:
        docs = [pair.ct(x) for x in data["v"]]
        tape = pf.pft_fasttext_train_forward(pair.ctx, model, docs, [pair.ct(x) for x in data["w"]])
        try:
            for b in range(B):
                s = pair.empty()
                pf.pft_ft_tape_score(pair.ctx, tape, b, s)
                got = o.decode(o.decrypt(OK.Ciphertext(pair.export(s), pf.pft_ct_scale(s))))[:N_CLS].real
                assert np.max(np.abs(got - OF.plain_scores(data["V"][b], data["H"], data["O"]))) < 2.0 ** -20
        finally:
            pf.pft_ft_tape_destroy(tape)
    finally:
        pf.pft_ft_enc_model_destroy(model)


def test_decrypted_gradients_vs_fp64_and_finite_differences(pair, data):
    o = pair.orc
    V, Y, H, O = data["V"], data["Y"], data["H"], data["O"]
    model, gH, gO = run_fused(pair, data)
    try:
        dec = lambda h, k: o.decode(o.decrypt(OK.Ciphertext(pair.export(h), pair.pft.pft_ct_scale(h))))[:k].real  # noqa
        got_H = np.stack([dec(gH[j], M_VOCAB) for j in range(N_COLS)], 1)
        got_O = np.stack([dec(gO[j], N_CLS) for j in range(N_COLS)])
    finally:
        pair.pft.pft_ft_enc_model_destroy(model)
    ref_H, ref_O = OF.train_grads_plain(V, Y, H, O)
    assert np.max(np.abs(got_H - ref_H)) < 2.0 ** -20
    assert np.max(np.abs(got_O - ref_O)) < 2.0 ** -20
    eps = 1e-4
    rng = np.random.default_rng(8)
    for X, G in ((H, got_H), (O, got_O)):
        picks = [tuple(int(rng.integers(0, s)) for s in X.shape) for _ in range(6)]
        for idx in picks:
            old = X[idx]
            X[idx] = old + eps
            lp = OF.train_loss_plain(V, Y, H, O)
            X[idx] = old - eps
            lm = OF.train_loss_plain(V, Y, H, O)
            X[idx] = old
            assert abs((lp - lm) / (2 * eps) - G[idx]) < 1e-6, idx


def test_training_errors(pair, data):
    pf = pair.pft
    model = gpu_model(pair, data)
    try:
        docs = [pair.ct(x) for x in data["v"]]
        o = pair.orc
        lw, sw = data["spec"]
        bad_scale = [pair.ct(o.encrypt_sk(o.encode(np.zeros(4), scale=2.0 ** 40, level=lw), 900 + b)) for b in range(B)]
        with pytest.raises(pf.PftError) as e:
            pf.pft_fasttext_train_step(pair.ctx, model, docs, bad_scale, ETA)
        assert e.value.code == pf.PFT_ERR_SCALE_MISMATCH
        bad_level = [pair.ct(o.encrypt_sk(o.encode(np.zeros(4), scale=sw, level=lw - 1), 950 + b)) for b in range(B)]
        with pytest.raises(pf.PftError) as e:
            pf.pft_fasttext_train_step(pair.ctx, model, docs, bad_level, ETA)
        assert e.value.code == pf.PFT_ERR_LEVEL_MISMATCH
        low = [pair.ct(o.drop_level(x, L0 - 1)) for x in data["v"]]
        with pytest.raises(pf.PftError) as e:
            pf.pft_fasttext_train_step(pair.ctx, model, low, [pair.ct(x) for x in data["w"]], ETA)
        assert e.value.code == pf.PFT_ERR_LEVEL_MISMATCH
    finally:
        pf.pft_ft_enc_model_destroy(model)


# ---- rotation-light training (diagonal layout) ------------------------------------------------
# N = 2^12 (t = 2048 slots), 10 primes so the seven levels of the step fit; n = 4 diagonals.
# Keys: 1..n-1 (hoisted document rotations), n 2^s (the replication sums over t/n blocks),
# -2^s (the spreading of the scores over their blocks) and relinearisation.  Each model is run
# unlifted (mask at 2^40) and with the documents lifted by 2^10 (mask at 2^30).

DL0, DN, DM, DC, DB = 10, 4, 400, 2, 3


@pytest.fixture(scope="module")
def pair_diag(gpu):
    t = 2048
    steps = list(range(1, DN)) + [DN << s for s in range(20) if (DN << s) < t] + [-(1 << s) for s in range(2)]
    p = Pair(gpu, 12, DL0, 2, 2, seed=(0x7C, 9, 9, 1), rot_steps=steps)
    yield p
    p.close()


@pytest.fixture(scope="module", params=[0, 10])
def data_diag(pair_diag, request):
    lift = request.param
    o, t = pair_diag.orc, pair_diag.N // 2
    rng = np.random.default_rng(31)
    V = np.zeros((DB, DM))
    for b in range(DB):
        np.add.at(V[b], rng.integers(0, DM, 25), 1.0)
        V[b] /= V[b].sum()
    Y = np.eye(DC)[[1, 0, 1]]
    H = rng.normal(0, 0.1, (DM, DN))
    O = rng.normal(0, 0.1, (DN, DC))
    D, P, Mv = OF.train_pack_diag(H, O, t)
    pad = lambda x: np.concatenate([x, np.zeros(t - x.size)])  # noqa: E731
    v = [o.encrypt_sk(o.encode(pad(V[b]), level=DL0), 100 + b) for b in range(DB)]
    Dc = [o.encrypt_sk(o.encode(D[k], level=DL0), 200 + k) for k in range(DN)]
    Pc = o.encrypt_pk(o.encode(P, level=DL0 - 1), 300)
    Mp = o.encode(Mv, scale=2.0 ** (40 - lift), level=DL0)
    lw, sw = OF.train_label_spec_diag(o, DL0, v[0].scale, Dc[0].scale, Pc.scale, Mp.scale, lift)
    w = [o.encrypt_sk(o.encode(OF.train_label_diag(Y[b], DN, t), scale=sw, level=lw), 400 + b) for b in range(DB)]
    want = OF.encrypted_train_step_diag(o, v, w, Dc, Pc, Mp, ETA, lift)
    return dict(V=V, Y=Y, H=H, O=O, v=v, w=w, Dc=Dc, Pc=Pc, Mp=Mp, spec=(lw, sw), want=want, lift=lift)


def gpu_model_diag(p, d):
    return p.pft.pft_ft_enc_model_create_diag(p.ctx, [p.ct(x) for x in d["Dc"]], p.ct(d["Pc"]), p.pt(d["Mp"]),
                                              DM, DN, DC, d["lift"])


def check_model_diag(p, model, want_D, want_P, what):
    pf = p.pft
    for k in range(DN):
        h = p.empty()
        pf.pft_ft_enc_model_get(p.ctx, model, 0, k, h)
        p.assert_equal(h, want_D[k], "%s D_%d" % (what, k))
    h = p.empty()
    pf.pft_ft_enc_model_get(p.ctx, model, 1, 0, h)
    p.assert_equal(h, want_P, "%s P" % what)


def run_fused_diag(p, d):
    model = gpu_model_diag(p, d)
    gD = [p.empty() for _ in range(DN)]
    gP = [p.empty()]
    p.pft.pft_fasttext_train_step(p.ctx, model, [p.ct(x) for x in d["v"]], [p.ct(x) for x in d["w"]], ETA, gD, gP)
    return model, gD, gP


def test_diag_spec_and_levels(pair_diag, data_diag):
    pf = pair_diag.pft
    model = gpu_model_diag(pair_diag, data_diag)
    try:
        assert pf.pft_fasttext_train_spec(pair_diag.ctx, model, data_diag["v"][0].scale) == \
            (DL0, data_diag["spec"][0], data_diag["spec"][1])
        assert pf.pft_ft_enc_model_levels(model) == (DL0, DL0 - 1)
    finally:
        pf.pft_ft_enc_model_destroy(model)


@pytest.mark.parametrize("tile", [None, "1"])
def test_diag_fused_step_bit_exact(pair_diag, data_diag, tile):
    pf = pair_diag.pft
    dD, dP, D1, P1 = data_diag["want"]
    if tile:
        os.environ["PFT_TRAIN_TILE"] = tile
    try:
        model, gD, gP = run_fused_diag(pair_diag, data_diag)
    finally:
        os.environ.pop("PFT_TRAIN_TILE", None)
    try:
        for k in range(DN):
            pair_diag.assert_equal(gD[k], dD[k], "dD_%d" % k)
        pair_diag.assert_equal(gP[0], dP, "dP")
        assert pf.pft_ft_enc_model_levels(model) == (DL0 - 7, DL0 - 8)
        check_model_diag(pair_diag, model, D1, P1, "updated")
    finally:
        pf.pft_ft_enc_model_destroy(model)


def test_diag_autograd_path_bit_exact(pair_diag, data_diag):
    from paper_1908_06972_gb300 import train as T

    p, d = pair_diag, data_diag
    dD, dP, D1, P1 = d["want"]
    m = T.EncryptedFastText.diag(p.ctx, [p.ct(x) for x in d["Dc"]], p.ct(d["Pc"]), p.pt(d["Mp"]), DM, DN, DC,
                                 d["lift"])
    try:
        opt = T.EncryptedSGD(m, ETA)
        m.loss([p.ct(x) for x in d["v"]], [p.ct(x) for x in d["w"]]).backward()
        assert len(m.grad_O) == 1
        for k in range(DN):
            p.assert_equal(m.grad_H[k], dD[k], "autograd dD_%d" % k)
        p.assert_equal(m.grad_O[0], dP, "autograd dP")
        opt.step()
        check_model_diag(p, m.model, D1, P1, "autograd updated")
    finally:
        m.close()


def test_diag_decrypted_gradients_vs_fp64(pair_diag, data_diag):
    p, d, o = pair_diag, data_diag, pair_diag.orc
    t = p.N // 2
    model, gD, gP = run_fused_diag(p, d)
    try:
        dec = lambda h: o.decode(o.decrypt(OK.Ciphertext(p.export(h), p.pft.pft_ct_scale(h)))).real  # noqa: E731
        got_D = [dec(gD[k]) for k in range(DN)]
        got_P = dec(gP[0])
    finally:
        p.pft.pft_ft_enc_model_destroy(model)
    gH, gO = OF.train_grads_plain(d["V"], d["Y"], d["H"], d["O"])
    ref_D, ref_P, _ = OF.train_pack_diag(np.vstack([gH, np.zeros((t - DM, DN))]), gO, t)
    for k in range(DN):
        assert np.max(np.abs(got_D[k] - ref_D[k])) < 2.0 ** -20, k
    assert np.max(np.abs(got_P[:DN * DC] - ref_P[:DN * DC])) < 2.0 ** -20


def test_diag_model_errors(pair_diag, data_diag):
    p, d = pair_diag, data_diag
    pf = p.pft
    D = [p.ct(x) for x in d["Dc"]]
    with pytest.raises(pf.PftError) as e:  # n not a power of two
        pf.pft_ft_enc_model_create_diag(p.ctx, D[:3], p.ct(d["Pc"]), p.pt(d["Mp"]), DM, 3, DC)
    assert e.value.code == pf.PFT_ERR_ARG
    with pytest.raises(pf.PftError) as e:  # lift out of range
        pf.pft_ft_enc_model_create_diag(p.ctx, D, p.ct(d["Pc"]), p.pt(d["Mp"]), DM, DN, DC, 31)
    assert e.value.code == pf.PFT_ERR_ARG
    with pytest.raises(pf.PftError) as e:  # P not one level below the diagonals
        pf.pft_ft_enc_model_create_diag(p.ctx, D, D[0], p.pt(d["Mp"]), DM, DN, DC)
    assert e.value.code == pf.PFT_ERR_LEVEL_MISMATCH
