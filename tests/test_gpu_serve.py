"""Request server (continuous batching of encrypted fastText inferences) on the GPU.

Two rings of different N run through one server: N = 2^12 (vocabulary in one input
ciphertext) and N = 2^11 (the same vocabulary spans two), both with the Fig. 3 sequence or both
with the rotation-light one (diagonal packing, per vocabulary chunk at N = 2^11).  Documents at every level from
3 to the top are submitted while others are in flight, so stages of different requests
share iterations.  Every score must equal, bit for bit, the oracle's sequence at the
request's level (model plaintexts encoded at that level: this pins that the top-level
model's leading limbs serve lower levels) and pft_fasttext_infer on the same input run
alone; admission must keep the admitted footprint within the budget."""
import numpy as np
import pytest

from oracle import ckks as OK
from oracle import fasttext as OF
from paper_1908_06972_gb300 import synth

from .pairs import Pair

pytestmark = pytest.mark.gpu

M_VOCAB, N_COLS, N_CLS = 2048, 4, 3


class Ring:
    def __init__(self, gpu, pair, H, O, diag=False):
        self.p, self.pf = pair, gpu
        o, t, L = pair.orc, pair.N // 2, pair.orc.L
        self.t, self.L, self.diag = t, L, diag
        self.H, self.O = H, O
        if diag:  # rotation-light packing, one set of diagonals per vocabulary chunk
            D, P = OF.pack_diag_chunks(H, O, t)
            self.chunks = D.shape[0]
            D_pts = [pair.pt(o.encode(D[i, k], level=L)) for i in range(self.chunks) for k in range(N_COLS)]
            self.model = gpu.pft_ft_model_import_diag(pair.ctx, D_pts, pair.pt(o.encode(P, level=L - 1)), M_VOCAB,
                                                      N_COLS, N_CLS)
            self.score_slots = OF.diag_score_slots(N_COLS, N_CLS)
        else:
            Hp, Op = OF.pack_H(H, t), OF.pack_O(O, t)
            self.chunks = Hp.shape[1]
            H_pts = [pair.pt(o.encode(Hp[j, i], level=L)) for j in range(N_COLS) for i in range(self.chunks)]
            O_pts = [pair.pt(o.encode(Op[j], level=L - 1)) for j in range(N_COLS)]
            self.model = gpu.pft_ft_model_import(pair.ctx, H_pts, O_pts, M_VOCAB, N_COLS, N_CLS)
            self.score_slots = list(range(N_CLS))

    def encrypt(self, doc, level, nonce):
        """The client's input: oracle ciphertexts (one per vocabulary chunk)."""
        o = self.p.orc
        v = np.zeros(self.chunks * self.t)
        v[:doc.size] = doc
        return [o.encrypt_sk(o.encode(v[i * self.t:(i + 1) * self.t], level=level), nonce + i)
                for i in range(self.chunks)]

    def oracle_scores(self, v_o, level):
        o = self.p.orc
        if self.diag:
            D, P = OF.pack_diag_chunks(self.H, self.O, self.t)
            D_o = [[o.encode(D[i, k], level=level) for k in range(N_COLS)] for i in range(self.chunks)]
            return OF.encrypted_scores_diag_chunks(o, v_o, D_o, o.encode(P, level=level - 1))
        Hp, Op = OF.pack_H(self.H, self.t), OF.pack_O(self.O, self.t)
        H_o = [[o.encode(Hp[j, i], level=level) for i in range(self.chunks)] for j in range(N_COLS)]
        O_o = [o.encode(Op[j], level=level - 1) for j in range(N_COLS)]
        return OF.encrypted_scores(o, v_o, H_o, O_o)

    def alone(self, v_o):
        """pft_fasttext_infer on the same input, exported to coefficient form."""
        s = self.p.empty()
        self.pf.pft_fasttext_infer(self.p.ctx, self.model, [self.p.ct(x) for x in v_o], s)
        return self.p.export(s), self.pf.pft_ct_scale(s)

    def close(self):
        self.pf.pft_ft_model_destroy(self.model)


@pytest.fixture(scope="module")
def pairs(gpu):
    """N = 2^12 with digits of two 40-bit primes (Fig. 3), N = 2^11 and N = 2^12 with one prime per
    digit.  The rotation-light sequence rotates its input at the input's scale, so it needs
    key-switching noise well below that scale: digits no larger than the 60-bit special prime."""
    a = Pair(gpu, 12, 5, 1, 2, seed=(0xA1, 2, 3, 4), rot_steps=[1 << i for i in range(11)] + [3])
    b = Pair(gpu, 11, 4, 1, 1, seed=(0xB2, 2, 3, 4), rot_steps=[1 << i for i in range(10)] + [3])
    a1 = Pair(gpu, 12, 5, 1, 1, seed=(0xA3, 2, 3, 4), rot_steps=[1 << i for i in range(11)] + [3])
    yield a, b, a1
    for p in (a, b, a1):
        p.close()


@pytest.fixture(scope="module", params=["fig3", "rotation_light"])
def rings(gpu, pairs, request):
    """The two rings serving the Fig. 3 sequence, or both serving the rotation-light one (the
    N = 2^11 ring's vocabulary spans two ciphertexts: diagonals per chunk)."""
    H, O = synth.fasttext_weights(71, M_VOCAB, N_COLS, N_CLS)
    diag = request.param == "rotation_light"
    rs = [Ring(gpu, pairs[2] if diag else pairs[0], H, O, diag=diag), Ring(gpu, pairs[1], H, O, diag=diag)]
    yield rs
    for r in rs:
        r.close()


def submit(pf, srv, ring, v_o, level, tag, keep):
    coeffs = np.ascontiguousarray(np.stack([x.c for x in v_o]))
    out = np.zeros((2, level - 2, ring.p.N), np.uint64)
    keep[tag] = (coeffs, out)
    pf.pft_server_submit(srv, rings_index(ring), coeffs, level, v_o[0].scale, out, tag)


_RING_INDEX = {}


def rings_index(ring):
    return _RING_INDEX[id(ring)]


def make_server(pf, rs, budget=0):
    for i, r in enumerate(rs):
        _RING_INDEX[id(r)] = i
    return pf.pft_server_create([r.p.ctx for r in rs], [r.model for r in rs], budget)


def test_server_mix_equals_alone_and_oracle(gpu, rings):
    pf = gpu
    docs = synth.documents(72, M_VOCAB, 7, 20, 80)
    plan = [(0, 5), (1, 4), (0, 3), (1, 3), (0, 4), (0, 5), (1, 4)]  # (ring, level) per request
    inputs = [rings[r].encrypt(docs[i], lv, 500 + 10 * i) for i, (r, lv) in enumerate(plan)]
    keep = {}
    srv = make_server(pf, rings)
    try:
        # staggered arrivals: later requests join while earlier ones are mid-sequence
        submit(pf, srv, rings[0], inputs[0], 5, 0, keep)
        submit(pf, srv, rings[1], inputs[1], 4, 1, keep)
        pf.pft_server_step(srv)
        pf.pft_server_step(srv)
        submit(pf, srv, rings[0], inputs[2], 3, 2, keep)
        submit(pf, srv, rings[1], inputs[3], 3, 3, keep)
        pf.pft_server_step(srv)
        for i in range(4, 7):
            r, lv = plan[i]
            submit(pf, srv, rings[r], inputs[i], lv, i, keep)
            pf.pft_server_step(srv)
        pf.pft_server_drain(srv)
        done = {d["tag"]: d for d in pf.pft_server_poll(srv)}
        st = pf.pft_server_get_stats(srv)
    finally:
        pf.pft_server_destroy(srv)
    assert sorted(done) == list(range(7))
    assert st["max_active"] >= 4 and st["completed"] == 7 and st["bytes_in_use"] == 0
    checked = set()
    for i, (r, lv) in enumerate(plan):
        ring = rings[r]
        got = keep[i][1]
        d = done[i]
        assert d["ring"] == r and d["level"] == lv - 2
        assert d["t_done"] >= d["t_submit"]
        alone, scale = ring.alone(inputs[i])
        assert np.array_equal(got, alone), "request %d differs from the same input run alone" % i
        assert d["scale"] == scale
        if (r, lv) not in checked:  # the oracle's sequence once per ring and level
            checked.add((r, lv))
            want = ring.oracle_scores(inputs[i], lv)
            assert np.array_equal(got, want.c), "request %d differs from the oracle" % i
            assert d["scale"] == want.scale
            dec = ring.p.orc.decode(ring.p.orc.decrypt(OK.Ciphertext(got, d["scale"]))).real[ring.score_slots]
            assert np.max(np.abs(dec - OF.plain_scores(docs[i], ring.H, ring.O))) < 2.0 ** -20


def test_server_admission_by_footprint(gpu, rings):
    pf = gpu
    ring = rings[0]
    docs = synth.documents(73, M_VOCAB, 5, 20, 80)
    inputs = [ring.encrypt(docs[i], 5, 900 + 10 * i) for i in range(5)]
    keep = {}
    probe = make_server(pf, [ring])
    fp5, fp4 = pf.pft_server_footprint(probe, 0, 5), pf.pft_server_footprint(probe, 0, 4)
    pf.pft_server_destroy(probe)
    assert fp4 < fp5
    srv = make_server(pf, [ring], budget=2 * fp5)
    try:
        for i in range(5):
            submit(pf, srv, ring, inputs[i], 5, i, keep)
        seen = []
        while True:
            left = pf.pft_server_step(srv)
            st = pf.pft_server_get_stats(srv)
            assert st["active"] <= 2 and st["bytes_in_use"] <= 2 * fp5
            seen += pf.pft_server_poll(srv)
            if left == 0 and st["waiting"] == 0 and st["active"] == 0:
                break
            if st["active"] == 0 and st["waiting"] == 0:
                pf.pft_server_drain(srv)
        seen += pf.pft_server_poll(srv)
        st = pf.pft_server_get_stats(srv)
    finally:
        pf.pft_server_destroy(srv)
    assert sorted(d["tag"] for d in seen) == list(range(5))
    assert st["max_active"] == 2 and st["peak_bytes"] == 2 * fp5
    # arrival order is kept: completions come in submission order
    assert [d["tag"] for d in sorted(seen, key=lambda d: d["t_done"])] == list(range(5))
    for i in range(5):
        assert np.array_equal(keep[i][1], ring.alone(inputs[i])[0])


def test_server_rejects_bad_requests(gpu, rings):
    pf = gpu
    ring = rings[0]
    probe = make_server(pf, [ring])
    fp5 = pf.pft_server_footprint(probe, 0, 5)
    pf.pft_server_destroy(probe)
    srv = make_server(pf, [ring], budget=fp5 - 1)
    z = np.zeros((1, 2, 5, ring.p.N), np.uint64)
    out = np.zeros((2, 3, ring.p.N), np.uint64)
    try:
        with pytest.raises(pf.PftError) as e:
            pf.pft_server_submit(srv, 0, z, 5, 2.0 ** 40, out, 1)
        assert e.value.code == pf.PFT_ERR_OOM and "budget" in str(e.value)
        for level, code in [(6, pf.PFT_ERR_LEVEL_MISMATCH), (2, pf.PFT_ERR_LEVEL_MISMATCH)]:
            with pytest.raises(pf.PftError) as e:
                pf.pft_server_submit(srv, 0, z, level, 2.0 ** 40, out, 2)
            assert e.value.code == code
        with pytest.raises(pf.PftError) as e:
            pf.pft_server_submit(srv, 3, z, 4, 2.0 ** 40, out, 3)
        assert e.value.code == pf.PFT_ERR_ARG
        assert pf.pft_server_get_stats(srv)["waiting"] == 0
    finally:
        pf.pft_server_destroy(srv)
    with pytest.raises(pf.PftError) as e:
        pf.pft_server_create([ring.p.ctx, ring.p.ctx], [ring.model, ring.model])
    assert e.value.code == pf.PFT_ERR_ARG and "context of its own" in str(e.value)


def test_server_diagonal_variant_bit_exact(gpu, pairs):
    """The rotation-light sequence through the server: two documents at levels 5 and 3."""
    pf = gpu
    H, O = synth.fasttext_weights(71, M_VOCAB, N_COLS, N_CLS)
    ring = Ring(gpu, pairs[2], H, O, diag=True)
    try:
        docs = synth.documents(74, M_VOCAB, 2, 20, 80)
        levels = [5, 3]
        inputs = [ring.encrypt(docs[i], levels[i], 700 + 10 * i) for i in range(2)]
        keep = {}
        srv = make_server(pf, [ring])
        try:
            submit(pf, srv, ring, inputs[0], 5, 0, keep)
            pf.pft_server_step(srv)
            submit(pf, srv, ring, inputs[1], 3, 1, keep)
            pf.pft_server_drain(srv)
            done = {d["tag"]: d for d in pf.pft_server_poll(srv)}
        finally:
            pf.pft_server_destroy(srv)
        for i in range(2):
            want = ring.oracle_scores(inputs[i], levels[i])
            assert np.array_equal(keep[i][1], want.c), "diagonal request %d differs from the oracle" % i
            assert done[i]["scale"] == want.scale
    finally:
        ring.close()
