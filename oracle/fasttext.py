"""fastText inference: the plaintext FP64 definition and the encrypted sequence
(test infrastructure only).

Passages (PrivFT, arXiv 1908.06972):
  * Algorithm 1, steps 2-3: h = (1/w) sum_i x_i H,  s = h O.
  * Sec. 3.1: the client sends v = sum_i x_i (here already divided by w, on
    the client); H is packed vertically (column j, vocabulary chunk i ->
    one plaintext), O horizontally (row j -> one plaintext, classes in slots
    0..c-1).  h_j = TotalSum(sum_i HMULPLAIN(v_i, Pt_{j,i})); the scores are
    sum_j HMULPLAIN(h_j, Pt(O_j)).
  * Algorithm 2 (TotalSum) with the reading i = 0 .. log2(t)-1.
Canonical order of this project: TotalSum at scale Delta^2, then one rescale
per column; the output product, then one final rescale.
"""
import numpy as np

from .ckks import Plaintext


def plain_scores(v, H, O):
    """Algorithm 1, steps 2-3 on the normalised count vector v (= (1/w) sum x_i)."""
    return (np.asarray(v, np.float64) @ np.asarray(H, np.float64)) @ np.asarray(O, np.float64)


def pack_H(H, t):
    """Slot vectors of the vertical packing: [n][ceil(m/t)][t]."""
    m, n = H.shape
    chunks = -(-m // t)
    out = np.zeros((n, chunks, t))
    for j in range(n):
        for i in range(chunks):
            col = H[i * t: (i + 1) * t, j]
            out[j, i, : col.size] = col
    return out


def pack_O(O, t):
    """Slot vectors of the horizontal packing: [n][t], row j in slots 0..c-1."""
    n, c = O.shape
    out = np.zeros((n, t))
    out[:, :c] = O
    return out


def encrypted_scores(orc, v_cts, H_pts, O_pts):
    """The server's canonical sequence on the oracle.

    v_cts: ceil(m/t) ciphertexts; H_pts[j][i]: plaintexts at the input level;
    O_pts[j]: plaintexts one level below.  Returns one ciphertext holding s in
    slots 0..c-1."""
    cols = []
    for j in range(len(H_pts)):
        t = orc.mul_plain(v_cts[0], H_pts[j][0])
        for i in range(1, len(v_cts)):
            t = orc.add(t, orc.mul_plain(v_cts[i], H_pts[j][i]))
        t = orc.total_sum(t)
        cols.append(orc.rescale(t))
    S = orc.mul_plain(cols[0], O_pts[0])
    for j in range(1, len(cols)):
        S = orc.add(S, orc.mul_plain(cols[j], O_pts[j]))
    return orc.rescale(S)


def column_total_sum(orc, v_cts, H_pts_j):
    """Column j of the first half of the sequence: TotalSum(sum_i v_i * H_{j,i}) then rescale."""
    t = orc.mul_plain(v_cts[0], H_pts_j[0])
    for i in range(1, len(v_cts)):
        t = orc.add(t, orc.mul_plain(v_cts[i], H_pts_j[i]))
    return orc.rescale(orc.total_sum(t))


# ---- rotation-light variant (diagonal packing; not in the paper) -----------------------------
# h_j = sum_u v_u H[u, j] for n columns (n a power of two dividing t, m <= t):
#   Q = sum_{k<n} rot(v, k) * D_k,  D_k[i] = H[(i + k) mod t, i mod n]   (hoisted rotations)
#   Q[i] = sum_k v[i+k] H[i+k, i mod n]; summing Q over the slots i + n r (r < t/n) -- a
#   rotate-and-sum with steps n 2^s -- gives h_{i mod n} in every slot i.
# Output layer: S = Q * P with P[n c + j] = O[j, c]; a rotate-and-sum with steps 2^s, s < log2 n,
# leaves s_c = sum_j h_j O[j, c] in slot n c.

# A vocabulary larger than one ciphertext (m > t) comes in chunks v_i = v[i t : i t + t]: with
# H_i the rows i t .. i t + t - 1 of H, h_j = sum_i sum_u v_i[u] H_i[u, j], so every chunk gets
# its own diagonals D_{i,k}[s] = H_i[(s + k) mod t, s mod n] and its own hoisted rotations, and
# Q = sum_i sum_k rot(v_i, k) D_{i,k}; the rest of the sequence is unchanged.

def pack_diag_chunks(H, O, t):
    """Slot vectors of the diagonal packing of a vocabulary in ceil(m/t) chunks: D [chunks][n][t]
    and P [t]."""
    m, n = H.shape
    c = O.shape[1]
    chunks = -(-m // t)
    Hp = np.zeros((chunks * t, n))
    Hp[:m] = H
    i = np.arange(t)
    D = np.stack([np.stack([Hp[ch * t + (i + k) % t, i % n] for k in range(n)]) for ch in range(chunks)])
    P = np.zeros(t)
    for cc in range(c):
        P[n * cc: n * cc + n] = O[:, cc]
    return D, P


def pack_diag(H, O, t):
    """Slot vectors of the diagonal packing of a vocabulary of at most t words: D [n][t] and P [t]."""
    assert H.shape[0] <= t
    D, P = pack_diag_chunks(H, O, t)
    return D[0], P


def diag_score_slots(n, c):
    """Slots holding the c scores in the diagonal variant."""
    return [n * cc for cc in range(c)]


def encrypted_scores_diag(orc, v_ct, D_pts, P_pt):
    """The rotation-light sequence on the oracle (one input ciphertext, m <= t)."""
    return encrypted_scores_diag_chunks(orc, [v_ct], [D_pts], P_pt)


def encrypted_scores_diag_chunks(orc, v_cts, D_pts, P_pt):
    """The rotation-light sequence on the oracle for a vocabulary in chunks: v_cts[i] the chunk
    ciphertexts, D_pts[i][k] the diagonals of chunk i; the products of chunk i, k = 0..n-1, are
    added in that order after those of chunk i - 1."""
    n = len(D_pts[0])
    t = orc.N // 2
    Q = None
    for v_ct, Dc in zip(v_cts, D_pts):
        R = [v_ct] + orc.rotate_hoisted(v_ct, list(range(1, n)))
        for k in range(n):
            term = orc.mul_plain(R[k], Dc[k])
            Q = term if Q is None else orc.add(Q, term)
    s = n
    while s < t:
        Q = orc.add(Q, orc.rotate(Q, s))
        s *= 2
    Q = orc.rescale(Q)
    S = orc.mul_plain(Q, P_pt)
    s = 1
    while s < n:
        S = orc.add(S, orc.rotate(S, s))
        s *= 2
    return orc.rescale(S)


# ---- minibatch training (Sec. 4.2, Algorithm 5) -----------------------------------------------
# Forward per document: h = v H, s = h O (Algorithm 1 with encrypted weights, HMUL for
# HMULPLAIN).  The softmax is replaced by the paper's minimax polynomial
#   P(s) = s^2/8 + s/2 + 1/4,
# and the loss is the polynomial whose gradient in s is P(s) - y:
#   L = sum_b sum_c [ s^3/24 + s^2/4 + s/4 - y s ]   (degree 3).
# Gradients: g = P(s) - y,  dL/dO = sum_b h^T g,  dL/dH = sum_b v^T (g O^T).
# Minibatch SGD (Algorithm 5): H <- H - eta dH, O <- O - eta dO.

def softmax_poly(s):
    """The paper's minimax approximation of softmax, P(s) = s^2/8 + s/2 + 1/4."""
    s = np.asarray(s, np.float64)
    return s * s / 8.0 + s / 2.0 + 0.25


def train_loss_plain(V, Y, H, O):
    """L(H, O) in FP64 for documents V [B][m] and one-hot labels Y [B][c]."""
    S = (np.asarray(V, np.float64) @ H) @ O
    return float(np.sum(S ** 3 / 24.0 + S ** 2 / 4.0 + S / 4.0 - np.asarray(Y, np.float64) * S))


def train_grads_plain(V, Y, H, O):
    """(dL/dH, dL/dO) in FP64."""
    V = np.asarray(V, np.float64)
    Hh = V @ H                        # [B][n]
    S = Hh @ O                        # [B][c]
    G = softmax_poly(S) - np.asarray(Y, np.float64)
    return V.T @ (G @ O.T), Hh.T @ G


# Encrypted step.  Layout as for inference: H_j holds column j of H over the vocabulary
# slots (one ciphertext per column, m <= t), O_j holds row j of O in slots 0..c-1, v_b is the
# document, and the client sends w_b = y_b - 1/4 on the c class slots (zero elsewhere), so the
# constant term of P never has to be masked on the server.  All constants the server adds
# are constant polynomials (every slot): with u = s + 2, u^2/8 - 1/2 = s^2/8 + s/2.
#   forward  h_bj = Rescale(TotalSum(Relin(v_b x H_j)))                      level l0-1
#            s_b  = Rescale(Relin(sum_j h_bj x O_j))                        level l0-2
#            U_b  = Rescale(Relin(u_b x u_b)), u_b = s_b + 2                level l0-3
#            g_b  = [U_b read at 8x its scale] - 1/2 - w_b   (= P(s_b) - y_b)
#   backward dO_j = Rescale(Relin(sum_b h_bj x g_b))                        level l0-4
#            e_bj = Rescale(TotalSum(Relin(g_b x O_j)))                     level l0-4
#            dH_j = Rescale(Relin(sum_b v_b x e_bj))                        level l0-5
#   update   O_j <- O_j - Align(dO_j), H_j <- H_j - Align(dH_j):  Align multiplies by
#            eta at the constant scale that brings the result, after one rescale, back to
#            the model's own scale (then read at exactly that scale).
# Operands at a higher level than needed are dropped to the lower level first; products
# summed before one relinearisation share their scale.

def train_label_spec(orc, level, sc_v, sc_H, sc_O):
    """Level and scale at which the client encrypts w_b for a model at `level`."""
    q = orc.q
    sh = sc_v * sc_H / float(q[level - 1])
    ss = sh * sc_O / float(q[level - 2])
    su = ss * ss / float(q[level - 3])
    return level - 3, 8.0 * su


def _align(orc, x, eta, target):
    c_sc = target * float(orc.q[x.level - 1]) / x.scale
    return orc.set_scale(orc.rescale(orc.mul_const(x, eta, c_sc)), target)


def encrypted_train_step(orc, v_cts, w_cts, H_cts, O_cts, eta):
    """One minibatch step on the oracle.  Returns (dH [n], dO [n], H' [n], O' [n]); with
    eta == 0 the model is returned unchanged."""
    B, n = len(v_cts), len(H_cts)
    l0 = H_cts[0].level
    assert all(x.level == l0 for x in v_cts + H_cts) and all(o.level == l0 - 1 for o in O_cts)
    h = [[None] * n for _ in range(B)]
    g = []
    for b in range(B):
        for j in range(n):
            t = orc.relin(*orc.tensor_sum([(v_cts[b], H_cts[j])]))
            h[b][j] = orc.rescale(orc.total_sum(t))
        s = orc.rescale(orc.relin(*orc.tensor_sum([(h[b][j], O_cts[j]) for j in range(n)])))
        u = orc.add_const(s, 2.0)
        U = orc.rescale(orc.relin(*orc.tensor_sum([(u, u)])))
        U = orc.add_const(orc.set_scale(U, 8.0 * U.scale), -0.5)
        g.append(orc.sub(U, w_cts[b]))
    lg = l0 - 3
    dO = [orc.rescale(orc.relin(*orc.tensor_sum([(orc.drop_level(h[b][j], lg), g[b]) for b in range(B)])))
          for j in range(n)]
    dH = []
    for j in range(n):
        Oj = orc.drop_level(O_cts[j], lg)
        e = [orc.rescale(orc.total_sum(orc.relin(*orc.tensor_sum([(g[b], Oj)])))) for b in range(B)]
        dH.append(orc.rescale(orc.relin(*orc.tensor_sum(
            [(orc.drop_level(v_cts[b], e[b].level), e[b]) for b in range(B)]))))
    if eta == 0:
        return dH, dO, list(H_cts), list(O_cts)
    O_new, H_new = [], []
    for j in range(n):
        a = _align(orc, dO[j], eta, O_cts[j].scale)
        O_new.append(orc.sub(orc.drop_level(O_cts[j], a.level), a))
        a = _align(orc, dH[j], eta, H_cts[j].scale)
        H_new.append(orc.sub(orc.drop_level(H_cts[j], a.level), a))
    return dH, dO, H_new, O_new


# ---- rotation-light training (diagonal packing; not in the paper) ------------------------------
# Model: D_k[i] = H[(i + k) mod t, i mod n] (k < n, the diagonals of the inference variant) at
# level l0 and P[n c + j] = O[j, c] (one ciphertext) at level l0 - 1; a plaintext mask M with
# 1 in the score slots n c.  The client sends v_b (m <= t) and w_b = y_b - 1/4 spread over the
# class blocks (w_b[c] in slots n c .. n c + n - 1).
#   lift     v'_b = 2^K v_b (an exact integer product: the scale grows by 2^K)
#   forward  R_bk = rot(v'_b, k) (hoisted), Q_b = Relin(sum_k R_bk x D_k),
#            Hb = Rescale(Q_b + rot(Q_b, n 2^s) ...)             h_b[i mod n] in slot i, l0-1
#            Sb = Rescale(S + rot(S, 2^s) ..., S = Relin(Hb x P)) s_b[c] in slot n c,  l0-2
#            Sm = Rescale(Z + rot(Z, -2^s) ..., Z = Sb * M)       s_b[c] over block c, l0-3
#            Gb = [Rescale(Relin(u x u)), u = Sm + 2] at 8x its scale - 1/2 - w_b,     l0-4
#   backward dP = Rescale(Relin(sum_b Hb x Gb))                   dO[j, c] in slot n c + j, l0-5
#            Eb = Rescale(X + rot(X, n 2^s) ..., X = Relin(Gb x P)) e_b[i mod n] in slot i, l0-5
#            dD_k = Rescale(Relin(sum_b R_bk x Eb))              the diagonals of dH, l0-6
#   update   D_k <- D_k - Align(dD_k) (l0-7), P <- drop(P - Align(dP), l0-8): one level below D.
# Noise: the document rotations are the only key switches applied at the input scale; their
# rounding noise is summed over the vocabulary in Hb, and the lift by 2^K divides it by 2^K
# (a mask encoded at 2^-K times the usual scale brings the scores back).  The scores are spread
# over their blocks before the rescale that follows the mask, so that the rescale noise of the
# slots around a score is not summed into it.

def train_pack_diag(H, O, t):
    """Slot vectors of the diagonal training layout: D [n][t], P [t], mask M [t]."""
    D, P = pack_diag(H, O, t)
    n, c = O.shape
    M = np.zeros(t)
    M[[n * cc for cc in range(c)]] = 1.0
    return D, P, M


def train_label_diag(y, n, t):
    """Label slot vector of the diagonal layout: y[c] - 1/4 over block c."""
    w = np.zeros(t)
    w[: n * len(y)] = np.repeat(np.asarray(y, np.float64) - 0.25, n)
    return w


def train_label_spec_diag(orc, level, sc_v, sc_D, sc_P, sc_M, lift_bits=0):
    q = orc.q
    sh = sc_v * 2.0 ** lift_bits * sc_D / float(q[level - 1])
    ss = sh * sc_P / float(q[level - 2])
    sm = ss * sc_M / float(q[level - 3])
    su = sm * sm / float(q[level - 4])
    return level - 4, 8.0 * su


def encrypted_train_step_diag(orc, v_cts, w_cts, D_cts, P_ct, M_pt, eta, lift_bits=0):
    """One minibatch step of the diagonal layout on the oracle.  Returns (dD [n], dP, D' [n], P')."""
    B, n = len(v_cts), len(D_cts)
    t = orc.N // 2
    l0 = D_cts[0].level
    assert all(x.level == l0 for x in v_cts + D_cts) and P_ct.level == l0 - 1
    R, Hs, G = [], [], []
    for b in range(B):
        v = orc.mul_const(v_cts[b], 1.0, 2.0 ** lift_bits) if lift_bits else v_cts[b]
        Rb = [v] + orc.rotate_hoisted(v, list(range(1, n)))
        R.append(Rb)
        Q = orc.relin(*orc.tensor_sum([(Rb[k], D_cts[k]) for k in range(n)]))
        st = n
        while st < t:
            Q = orc.add(Q, orc.rotate(Q, st))
            st *= 2
        Hb = orc.rescale(Q)
        Hs.append(Hb)
        S = orc.relin(*orc.tensor_sum([(Hb, P_ct)]))
        st = 1
        while st < n:
            S = orc.add(S, orc.rotate(S, st))
            st *= 2
        Sb = orc.rescale(S)
        Z = orc.mul_plain(Sb, Plaintext(M_pt.m[:Sb.level], M_pt.scale))
        st = 1
        while st < n:
            Z = orc.add(Z, orc.rotate(Z, -st))
            st *= 2
        u = orc.add_const(orc.rescale(Z), 2.0)
        U = orc.rescale(orc.relin(*orc.tensor_sum([(u, u)])))
        U = orc.add_const(orc.set_scale(U, 8.0 * U.scale), -0.5)
        G.append(orc.sub(U, w_cts[b]))
    lg = G[0].level
    dP = orc.rescale(orc.relin(*orc.tensor_sum([(orc.drop_level(Hs[b], lg), G[b]) for b in range(B)])))
    Pg = orc.drop_level(P_ct, lg)
    E = []
    for b in range(B):
        X = orc.relin(*orc.tensor_sum([(G[b], Pg)]))
        st = n
        while st < t:
            X = orc.add(X, orc.rotate(X, st))
            st *= 2
        E.append(orc.rescale(X))
    le = E[0].level
    dD = [orc.rescale(orc.relin(*orc.tensor_sum([(orc.drop_level(R[b][k], le), E[b]) for b in range(B)])))
          for k in range(n)]
    if eta == 0:
        return dD, dP, list(D_cts), P_ct
    D_new = []
    for k in range(n):
        a = _align(orc, dD[k], eta, D_cts[k].scale)
        D_new.append(orc.sub(orc.drop_level(D_cts[k], a.level), a))
    a = _align(orc, dP, eta, P_ct.scale)
    P_new = orc.drop_level(orc.sub(orc.drop_level(P_ct, a.level), a), D_new[0].level - 1)
    return dD, dP, D_new, P_new
