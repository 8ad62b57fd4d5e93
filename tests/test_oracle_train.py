"""Pins of the oracle's minibatch training step (Sec. 4.2, Algorithm 5) -- no GPU.

* the paper's softmax polynomial P(s) = s^2/8 + s/2 + 1/4 is the derivative of the
  per-class loss s^3/24 + s^2/4 + s/4 - y s (plus y), closed form;
* the FP64 gradients equal central finite differences of the FP64 loss;
* the level/scale operations (drop, relabel, exact constants) keep their meaning;
* the encrypted oracle step decrypts to the FP64 gradients and SGD update within 2^-20.
"""
import numpy as np
import pytest

from oracle import ckks as OK
from oracle import fasttext as OF


def test_softmax_poly_coefficients_and_loss_derivative():
    s = np.linspace(-3, 3, 61)
    assert np.allclose(OF.softmax_poly(s), s * s / 8 + s / 2 + 0.25, rtol=0, atol=1e-15)
    assert OF.softmax_poly(0.0) == 0.25
    # d/ds of the degree-3 per-class loss, by exact polynomial differentiation
    loss = np.polynomial.Polynomial([0.0, 0.25, 0.25, 1.0 / 24.0])
    assert np.allclose(loss.deriv()(s), OF.softmax_poly(s), rtol=0, atol=1e-15)
    # P(s) = (s + 2)^2 / 8 - 1/4: the form the encrypted step evaluates
    assert np.allclose((s + 2) ** 2 / 8 - 0.25, OF.softmax_poly(s), rtol=0, atol=1e-15)


def test_fp64_gradients_match_central_differences():
    rng = np.random.default_rng(3)
    B, m, n, c = 3, 7, 4, 3
    V = rng.random((B, m))
    V /= V.sum(1, keepdims=True)
    Y = np.eye(c)[rng.integers(0, c, B)]
    H = rng.normal(0, 0.5, (m, n))
    O = rng.normal(0, 0.5, (n, c))
    dH, dO = OF.train_grads_plain(V, Y, H, O)
    eps = 1e-5
    for X, G in ((H, dH), (O, dO)):
        fd = np.zeros_like(X)
        for idx in np.ndindex(X.shape):
            old = X[idx]
            X[idx] = old + eps
            lp = OF.train_loss_plain(V, Y, H, O)
            X[idx] = old - eps
            lm = OF.train_loss_plain(V, Y, H, O)
            X[idx] = old
            fd[idx] = (lp - lm) / (2 * eps)
        assert np.max(np.abs(fd - G)) < 1e-8 * max(1.0, np.max(np.abs(G)))


def test_round_half_away():
    for x, k in [(2.5, 3), (-2.5, -3), (2.4999999999999996, 2), (-0.5, -1), (0.49999999999999994, 0),
                 (2.0 ** 52 + 1, 2 ** 52 + 1), (-(2.0 ** 60), -(2 ** 60)), (1e-300, 0)]:
        assert OK.round_half_away(x) == k, x


@pytest.fixture(scope="module")
def small():
    o = OK.Oracle(10, 8, 2, 2, 60, 40, 60, 2.0 ** 40, (0x7A, 1, 2, 3))  # P = 2^120 above every digit
    o.keygen([1 << i for i in range(9)], True)
    return o


def dec(o, ct, k):
    return o.decode(o.decrypt(ct))[:k].real


def test_level_scale_and_constant_ops(small):
    o = small
    rng = np.random.default_rng(5)
    z = rng.uniform(-1, 1, 512)
    ct = o.encrypt_sk(o.encode(z, level=5), 17)
    d = o.drop_level(ct, 3)
    assert d.level == 3 and np.max(np.abs(dec(o, d, 512) - z)) < 1e-9
    assert np.max(np.abs(dec(o, o.set_scale(ct, ct.scale * 8), 512) - z / 8)) < 1e-9
    assert np.max(np.abs(dec(o, o.add_const(ct, -0.75), 512) - (z - 0.75))) < 1e-9
    m = o.mul_const(ct, 0.3, float(o.q[4]))  # constant scale = the prime the rescale drops
    assert m.scale == ct.scale * float(o.q[4])
    r = o.rescale(m)
    assert r.scale == ct.scale and np.max(np.abs(dec(o, r, 512) - 0.3 * z)) < 1e-8
    # the constant goes to coefficient 0 of c0 only
    a = o.add_const(ct, 1.0)
    diff = (a.c.astype(object) - ct.c.astype(object))
    assert np.count_nonzero(diff[1]) == 0 and np.count_nonzero(diff[0][:, 1:]) == 0
    # lazy relinearisation of a sum of two products = sum of the two products' meaning
    y = rng.uniform(-1, 1, 512)
    cy = o.encrypt_sk(o.encode(y, level=5), 18)
    r = o.relin(*o.tensor_sum([(ct, cy), (cy, cy)]))
    assert np.max(np.abs(dec(o, o.rescale(r), 512) - (z * y + y * y))) < 2.0 ** -20


def test_encrypted_train_step_matches_fp64(small):
    o = small
    t = o.N // 2
    rng = np.random.default_rng(11)
    B, m, n, c, eta = 2, 300, 2, 2, 0.5
    V = np.zeros((B, m))
    for b in range(B):
        ids = rng.integers(0, m, 25)
        np.add.at(V[b], ids, 1.0)
        V[b] /= V[b].sum()
    Y = np.eye(c)[[0, 1]]
    H = rng.normal(0, 0.1, (m, n))
    O = rng.normal(0, 0.1, (n, c))
    l0 = 8
    pad = lambda x: np.concatenate([x, np.zeros(t - x.size)])  # noqa: E731
    v_ct = [o.encrypt_sk(o.encode(pad(V[b]), level=l0), 100 + b) for b in range(B)]
    H_ct = [o.encrypt_sk(o.encode(pad(H[:, j]), level=l0), 200 + j) for j in range(n)]
    O_ct = [o.encrypt_sk(o.encode(pad(O[j]), level=l0 - 1), 300 + j) for j in range(n)]
    lw, sw = OF.train_label_spec(o, l0, v_ct[0].scale, H_ct[0].scale, O_ct[0].scale)
    assert lw == l0 - 3
    w_ct = [o.encrypt_sk(o.encode(pad(Y[b] - 0.25), scale=sw, level=lw), 400 + b) for b in range(B)]
    dH, dO, H1, O1 = OF.encrypted_train_step(o, v_ct, w_ct, H_ct, O_ct, eta)
    gH, gO = OF.train_grads_plain(V, Y, H, O)
    tol = 2.0 ** -20
    for j in range(n):
        assert dH[j].level == l0 - 5 and dO[j].level == l0 - 4
        assert np.max(np.abs(dec(o, dH[j], m) - gH[:, j])) < tol
        assert np.max(np.abs(dec(o, dO[j], c) - gO[j])) < tol
        assert np.max(np.abs(dec(o, dO[j], t)[c:])) < tol  # nothing outside the class slots
        assert H1[j].level == l0 - 6 and O1[j].level == l0 - 5
        assert H1[j].scale == H_ct[j].scale and O1[j].scale == O_ct[j].scale
        assert np.max(np.abs(dec(o, H1[j], m) - (H[:, j] - eta * gH[:, j]))) < tol
        assert np.max(np.abs(dec(o, O1[j], c) - (O[j] - eta * gO[j]))) < tol
    # a gradient step lowers the loss
    assert OF.train_loss_plain(V, Y, H - eta * gH, O - eta * gO) < OF.train_loss_plain(V, Y, H, O)


@pytest.fixture(scope="module")
def small_diag():
    o = OK.Oracle(10, 10, 2, 2, 60, 40, 60, 2.0 ** 40, (0x7C, 1, 2, 3))
    n, t = 4, 512
    steps = list(range(1, n)) + [n << s for s in range(7)] + [-1, -2]
    o.keygen(steps, True)
    return o


@pytest.mark.parametrize("lift", [0, 10])
def test_encrypted_train_step_diag_matches_fp64(small_diag, lift):
    """The rotation-light training step (diagonal layout) decrypts to the diagonals of the FP64
    dH, to dO in the output layout, and to the SGD update; with the documents lifted by 2^10
    and the mask at 2^30 the scales come back to those of the unlifted step."""
    o = small_diag
    t = o.N // 2
    rng = np.random.default_rng(13)
    B, m, n, c, eta = 2, 400, 4, 2, 0.5
    V = np.zeros((B, m))
    for b in range(B):
        np.add.at(V[b], rng.integers(0, m, 25), 1.0)
        V[b] /= V[b].sum()
    Y = np.eye(c)[[1, 0]]
    H = rng.normal(0, 0.1, (m, n))
    O = rng.normal(0, 0.1, (n, c))
    D, P, M = OF.train_pack_diag(H, O, t)
    l0 = 10
    pad = lambda x: np.concatenate([x, np.zeros(t - x.size)])  # noqa: E731
    v_ct = [o.encrypt_sk(o.encode(pad(V[b]), level=l0), 100 + b) for b in range(B)]
    D_ct = [o.encrypt_sk(o.encode(D[k], level=l0), 200 + k) for k in range(n)]
    P_ct = o.encrypt_sk(o.encode(P, level=l0 - 1), 300)
    M_pt = o.encode(M, scale=2.0 ** (40 - lift), level=l0)
    lw, sw = OF.train_label_spec_diag(o, l0, v_ct[0].scale, D_ct[0].scale, P_ct.scale, M_pt.scale, lift)
    assert lw == l0 - 4
    if lift:  # the lift and the mask cancel: the labels sit at the unlifted step's scale
        assert sw == OF.train_label_spec_diag(o, l0, v_ct[0].scale, D_ct[0].scale, P_ct.scale, 2.0 ** 40)[1]
    w_ct = [o.encrypt_sk(o.encode(OF.train_label_diag(Y[b], n, t), scale=sw, level=lw), 400 + b) for b in range(B)]
    dD, dP, D1, P1 = OF.encrypted_train_step_diag(o, v_ct, w_ct, D_ct, P_ct, M_pt, eta, lift)
    gH, gO = OF.train_grads_plain(V, Y, H, O)
    gD, gP, _ = OF.train_pack_diag(np.vstack([gH, np.zeros((t - m, n))])[:t], gO, t)
    tol = 2.0 ** -20
    for k in range(n):
        assert dD[k].level == l0 - 6 and D1[k].level == l0 - 7 and D1[k].scale == D_ct[k].scale
        assert np.max(np.abs(dec(o, dD[k], t) - gD[k])) < tol
        assert np.max(np.abs(dec(o, D1[k], t) - (D[k] - eta * gD[k]))) < tol
    assert dP.level == l0 - 5 and P1.level == l0 - 8 and P1.scale == P_ct.scale
    assert np.max(np.abs(dec(o, dP, t)[: n * c] - gP[: n * c])) < tol
    assert np.max(np.abs(dec(o, P1, t)[: n * c] - (P - eta * gP)[: n * c])) < tol


def test_train_label_diag_layout():
    w = OF.train_label_diag([1.0, 0.0, 0.5], 4, 16)
    assert np.array_equal(w, [0.75] * 4 + [-0.25] * 4 + [0.25] * 4 + [0.0] * 4)
