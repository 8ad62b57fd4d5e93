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
