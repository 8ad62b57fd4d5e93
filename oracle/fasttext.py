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

def pack_diag(H, O, t):
    """Slot vectors of the diagonal packing: D [n][t] and P [t]."""
    m, n = H.shape
    c = O.shape[1]
    Hp = np.zeros((t, n))
    Hp[:m] = H
    i = np.arange(t)
    D = np.stack([Hp[(i + k) % t, i % n] for k in range(n)])
    P = np.zeros(t)
    for cc in range(c):
        P[n * cc: n * cc + n] = O[:, cc]
    return D, P


def diag_score_slots(n, c):
    """Slots holding the c scores in the diagonal variant."""
    return [n * cc for cc in range(c)]


def encrypted_scores_diag(orc, v_ct, D_pts, P_pt):
    """The rotation-light sequence on the oracle (one input ciphertext, m <= t)."""
    n = len(D_pts)
    t = orc.N // 2
    R = [v_ct] + orc.rotate_hoisted(v_ct, list(range(1, n)))
    Q = orc.mul_plain(R[0], D_pts[0])
    for k in range(1, n):
        Q = orc.add(Q, orc.mul_plain(R[k], D_pts[k]))
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
