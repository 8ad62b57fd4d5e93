"""Plain RNS-CKKS oracle (test infrastructure only -- never used by the product).

Everything here works on polynomials in COEFFICIENT form, one row per RNS
prime, canonical residues in [0, q).  Products are negacyclic products taken
from the oracle's own C primitives (textbook transform, pinned against the
schoolbook sum); nothing is shared with the CUDA library.

Passages (PrivFT, arXiv 1908.06972), with this project's readings where the
text is garbled or silent:
  * Sec. 2.3 KEYGEN:  s <- ternary; pk = (b, a), b = -a s + e.
  * Sec. 2.3 ENC:     the printed formula pairs the terms so that c0 + c1 s
    does not cancel; the reading used is c0 = v b + mu + e0, c1 = v a + e1
    with an ephemeral TERNARY v (public-key mode), and the symmetric form
    c0 = -a s + mu + e, c1 = a (secret-key mode).
  * Sec. 2.3 DEC:     mu = c0 + c1 s mod q_l.
  * Sec. 2.3 ENCODE/DECODE: mu = round(IDFT(Delta z)) over the canonical
    embedding, slot j <-> root omega^(5^j mod 2N), omega = exp(i pi / N).
  * Sec. 2.3 HADD, HMUL (tensor), HADDPLAIN, HMULPLAIN.
  * Sec. 2.3 HMUL relinearisation and the ROTATE footnote: key switching
    (not spelled out in the paper).  Reading: hybrid key switching with
    digits of alpha primes, fast basis conversion up (ModUp) and down
    (ModDown) without correction, key_j = (-a_j s + e_j + [i in digit j] P s', a_j).
  * Sec. 2.3 ROTATE and Sec. 5.3: X -> X^g with g = 5^r mod 2N, one key per g.
  * Eq. 1 / Algorithm 3 (RESCALE): divide by the last prime; the output
    is rounded (Sec. 2.3 RESCALE), i.e. floor((c + floor(p/2)) / p); the
    plain floor of Eq. 1 is kept as an option.
"""
import math

import numpy as np

from . import _lib as C
from . import params as P

# sampler stream domains (the first nonce word)
DOM_SECRET, DOM_PK_A, DOM_PK_E, DOM_KSK_A, DOM_KSK_E = 1, 2, 3, 4, 5
DOM_ENC_A, DOM_ENC_E, DOM_ENC_V, DOM_ENC_E0, DOM_ENC_E1 = 6, 7, 8, 9, 10
DOM_KSK_A_EVAL = 11  # a_j of seeded compressed keys, drawn in the library's evaluation layout


class Ciphertext:
    """(c0, c1) as a [2][l][N] uint64 array in coefficient form, with its scale."""

    def __init__(self, c, scale):
        self.c = np.ascontiguousarray(c, np.uint64)
        self.scale = float(scale)

    @property
    def level(self):
        return self.c.shape[1]


class Plaintext:
    """mu as an [l][N] uint64 array in coefficient form, with its scale."""

    def __init__(self, m, scale):
        self.m = np.ascontiguousarray(m, np.uint64)
        self.scale = float(scale)

    @property
    def level(self):
        return self.m.shape[0]


def round_half_away(x):
    """The integer nearest to the double x, ties away from zero (exact for every double)."""
    x = float(x)
    f = math.floor(x)
    d = x - f  # exact: x and floor(x) are within one unit of each other's exponent range
    if d > 0.5 or (d == 0.5 and x > 0):
        return int(f) + 1
    return int(f)


def galois_element(step, n):
    """g = 5^step mod 2N (5 has order N/2 modulo 2N, so negative steps wrap)."""
    return pow(5, step % (n // 2), 2 * n)


def crt_centered(rows, primes):
    """CRT-reconstruct each column into the integer in (-Q/2, Q/2] (Python ints)."""
    primes = [int(p) for p in primes]
    Q = math.prod(primes)
    acc = np.zeros(rows.shape[1], dtype=object)
    for i, qi in enumerate(primes):
        qhat = Q // qi
        inv = pow(qhat % qi, -1, qi)
        acc = acc + (rows[i].astype(object) * inv % qi) * qhat
    acc = acc % Q
    return np.where(acc > Q // 2, acc - Q, acc)


class Oracle:
    def __init__(self, logn, n_limbs, n_special, alpha, first_bits=60, mid_bits=40,
                 special_bits=60, scale=2.0 ** 40, seed=(1, 2, 3, 4), sigma="3.2",
                 primes=None, special_primes=None, compressed_keys=False):
        self.logn, self.N = logn, 1 << logn
        if primes is None:
            self.q, self.p = P.prime_chain(logn, n_limbs, n_special, first_bits, mid_bits, special_bits)
        else:
            self.q, self.p = [int(x) for x in primes], [int(x) for x in special_primes]
        self.L, self.k, self.alpha = len(self.q), len(self.p), alpha
        self.scale = float(scale)
        self.seed = tuple(int(s) for s in seed)
        self.cdt = np.array(P.gauss_cdt(sigma), np.uint32)
        self.Pprod = math.prod(self.p)
        self.keys = {}
        self.compressed_keys = compressed_keys

    # ---- sampler (counter-based ChaCha20 streams) --------------------------------------
    def uniform_rows(self, dom, obj, subs, primes):
        return np.stack([C.sample_uniform(self.seed, dom, obj, s, q, self.N) for s, q in zip(subs, primes)])

    def ternary(self, dom, obj, sub=0):
        return C.sample_ternary(self.seed, dom, obj, sub, self.N)

    def gauss(self, dom, obj, sub=0):
        return C.sample_gauss(self.seed, dom, obj, sub, self.N, self.cdt)

    # ---- KEYGEN (Sec. 2.3) -------------------------------------------------------------
    def keygen(self, rot_steps=(), relin=True):
        q, L = self.q, self.L
        self.s = self.ternary(DOM_SECRET, 0)
        s_q = C.reduce_signed(self.s, q)
        a = self.uniform_rows(DOM_PK_A, 0, range(L), q)
        e = C.reduce_signed(self.gauss(DOM_PK_E, 0), q)
        self.pk = (C.vsub(e, C.polymul(a, s_q, q), q), a)
        basis = q + self.p
        s_b = C.reduce_signed(self.s, basis)
        if relin:
            self.keys[0] = self.switch_key(C.polymul(s_b, s_b, basis), 0)
        for r in rot_steps:
            g = galois_element(r, self.N)
            if g != 1 and g not in self.keys:
                self.keys[g] = self.switch_key(C.automorph(s_b, basis, g), g)

    def switch_key(self, sp, key_id):
        """Key switching key from s' (rows over the basis q_0..q_{L-1}, p_0..p_{k-1}) to s.

        Digit j (primes j*alpha .. (j+1)*alpha-1 of the chain):
          a_j uniform, e_j Gaussian,
          b_j = -a_j s + e_j + P s'   on the primes of digit j,
          b_j = -a_j s + e_j          on every other prime (P = 0 mod p_i).
        Returned as [beta][2 (b, a)][L+k][N].
        """
        basis = self.q + self.p
        nb, L, alpha = len(basis), self.L, self.alpha
        beta = -(-L // alpha)
        s_b = C.reduce_signed(self.s, basis)
        K = np.empty((beta, 2, nb, self.N), np.uint64)
        for j in range(beta):
            if self.compressed_keys:
                # seeded compressed keys: a_j drawn as evaluation-layout entries (entry i of
                # row m = the uniform residue of word pair i of stream (key_id, 256 j + m)),
                # i.e. a_j is the polynomial interpolating those values
                ev = self.uniform_rows(DOM_KSK_A_EVAL, key_id, [j * 256 + m for m in range(nb)], basis)
                a = np.stack([C.interp_layout(ev[m], P.root_2n(basis[m], self.logn), basis[m], self.logn)
                              for m in range(nb)])
            else:
                a = self.uniform_rows(DOM_KSK_A, key_id, [j * 256 + m for m in range(nb)], basis)
            e = C.reduce_signed(self.gauss(DOM_KSK_E, key_id, j), basis)
            b = C.vsub(e, C.polymul(a, s_b, basis), basis)
            for i in range(j * alpha, min((j + 1) * alpha, L)):
                qi = basis[i]
                b[i] = C.vadd(b[i:i + 1], C.vscale(sp[i:i + 1], [self.Pprod % qi], [qi]), [qi])[0]
            K[j, 0], K[j, 1] = b, a
        return K

    # ---- ENCODE / DECODE (Sec. 2.3) ----------------------------------------------------
    def slot_exponents(self):
        """e_j = 5^j mod 2N for the N/2 slots."""
        n2 = 2 * self.N
        return np.array([pow(5, j, n2) for j in range(self.N // 2)], np.int64)

    def encode_real(self, z, scale):
        """Real coefficients (before rounding) of the polynomial whose value at
        omega^(5^j) is scale * z_j and at the conjugate root its conjugate."""
        N = self.N
        z = np.zeros(N // 2, complex) if z is None else np.asarray(z, complex)
        zz = np.zeros(N // 2, complex)
        zz[: z.size] = z
        e = self.slot_exponents()
        W = np.zeros(N, complex)
        W[(e - 1) // 2] = scale * zz
        W[(2 * N - e - 1) // 2] = np.conj(scale * zz)
        k = np.arange(N)
        # m_k = (1/N) sum_u W[u] omega^(-(2u+1)k) = omega^(-k) * DFT(W)[k] / N
        return (np.exp(-1j * np.pi * k / N) * np.fft.fft(W) / N).real

    def encode(self, z, scale=None, level=None):
        scale = self.scale if scale is None else float(scale)
        level = self.L if level is None else level
        m = self.encode_real(z, scale)
        mi = np.sign(m) * np.floor(np.abs(m) + 0.5)  # round half away from zero
        if np.any(np.abs(mi) >= 2.0 ** 62):
            raise ValueError("encoded coefficient exceeds 2^62")
        return Plaintext(C.reduce_signed(mi.astype(np.int64), self.q[:level]), scale)

    def decode_int(self, m, scale, nslots=None):
        """Slot values of an integer polynomial m (centered coefficients)."""
        N = self.N
        mf = np.array([float(x) for x in m], np.float64)
        k = np.arange(N)
        vals = N * np.fft.ifft(mf * np.exp(1j * np.pi * k / N))  # m(omega^(2u+1))
        z = vals[(self.slot_exponents() - 1) // 2] / scale
        return z if nslots is None else z[:nslots]

    def decode(self, pt, nslots=None):
        return self.decode_int(crt_centered(pt.m, self.q[: pt.level]), pt.scale, nslots)

    # ---- ENC / DEC (Sec. 2.3) ----------------------------------------------------------
    def encrypt_sk(self, pt, nonce):
        l, q = pt.level, self.q[: pt.level]
        a = self.uniform_rows(DOM_ENC_A, nonce, range(l), q)
        e = C.reduce_signed(self.gauss(DOM_ENC_E, nonce), q)
        s_q = C.reduce_signed(self.s, q)
        c0 = C.vadd(C.vsub(e, C.polymul(a, s_q, q), q), pt.m, q)
        return Ciphertext(np.stack([c0, a]), pt.scale)

    def encrypt_pk(self, pt, nonce):
        l, q = pt.level, self.q[: pt.level]
        v = C.reduce_signed(self.ternary(DOM_ENC_V, nonce), q)
        e0 = C.reduce_signed(self.gauss(DOM_ENC_E0, nonce), q)
        e1 = C.reduce_signed(self.gauss(DOM_ENC_E1, nonce), q)
        b, a = self.pk[0][:l], self.pk[1][:l]
        c0 = C.vadd(C.vadd(C.polymul(v, b, q), pt.m, q), e0, q)
        c1 = C.vadd(C.polymul(v, a, q), e1, q)
        return Ciphertext(np.stack([c0, c1]), pt.scale)

    def decrypt(self, ct):
        q = self.q[: ct.level]
        s_q = C.reduce_signed(self.s, q)
        return Plaintext(C.vadd(ct.c[0], C.polymul(ct.c[1], s_q, q), q), ct.scale)

    # ---- homomorphic operations (Sec. 2.3) ---------------------------------------------
    def _q(self, ct):
        return self.q[: ct.level]

    def add(self, a, b):
        assert a.level == b.level and a.scale == b.scale
        q = self._q(a)
        return Ciphertext(np.stack([C.vadd(a.c[i], b.c[i], q) for i in range(2)]), a.scale)

    def sub(self, a, b):
        assert a.level == b.level and a.scale == b.scale
        q = self._q(a)
        return Ciphertext(np.stack([C.vsub(a.c[i], b.c[i], q) for i in range(2)]), a.scale)

    def add_plain(self, ct, pt):
        assert ct.level == pt.level and ct.scale == pt.scale
        q = self._q(ct)
        return Ciphertext(np.stack([C.vadd(ct.c[0], pt.m, q), ct.c[1]]), ct.scale)

    def mul_plain(self, ct, pt):
        assert ct.level == pt.level
        q = self._q(ct)
        return Ciphertext(np.stack([C.polymul(ct.c[i], pt.m, q) for i in range(2)]), ct.scale * pt.scale)

    def tensor(self, a, b):
        """HMUL before relinearisation: (c00 c10, c00 c11 + c01 c10, c01 c11)."""
        assert a.level == b.level
        q = self._q(a)
        d0 = C.polymul(a.c[0], b.c[0], q)
        d1 = C.vadd(C.polymul(a.c[0], b.c[1], q), C.polymul(a.c[1], b.c[0], q), q)
        d2 = C.polymul(a.c[1], b.c[1], q)
        return d0, d1, d2

    # ---- level and scale management (used by the training step) --------------------------
    def drop_level(self, ct, level):
        """The same message with the primes above `level` dropped (exact: the residues
        modulo q_0..q_{level-1} of the same integers)."""
        assert 1 <= level <= ct.level
        return Ciphertext(ct.c[:, :level].copy(), ct.scale)

    def set_scale(self, ct, scale):
        """Relabel: the same integers read at another scale (message times old/new)."""
        return Ciphertext(ct.c.copy(), scale)

    def add_const(self, ct, value):
        """Adds `value` to every slot: the constant polynomial round(value * scale) added to c0."""
        q = self._q(ct)
        k = round_half_away(value * ct.scale)
        c = ct.c.copy()
        for i, qi in enumerate(q):
            c[0, i, 0] = np.uint64((int(c[0, i, 0]) + k) % qi)
        return Ciphertext(c, ct.scale)

    def mul_const(self, ct, value, const_scale):
        """Multiplies every slot by `value`: both polynomials times the integer
        round(value * const_scale); the scale is multiplied by const_scale."""
        q = self._q(ct)
        k = round_half_away(value * const_scale)
        kk = [k % qi for qi in q]
        return Ciphertext(np.stack([C.vscale(ct.c[i], kk, q) for i in range(2)]), ct.scale * const_scale)

    def tensor_sum(self, pairs):
        """sum_k tensor(a_k, b_k) (three polynomials) and its scale; all products share one
        level and one scale."""
        a0, b0 = pairs[0]
        q = self._q(a0)
        sc = a0.scale * b0.scale
        acc = [np.zeros((a0.level, self.N), np.uint64) for _ in range(3)]
        for a, b in pairs:
            assert a.level == a0.level and b.level == a0.level and a.scale * b.scale == sc
            for i, d in enumerate(self.tensor(a, b)):
                acc[i] = C.vadd(acc[i], d, q)
        return acc, sc

    def relin(self, d, scale):
        """(d0, d1, d2) -> (d0 + u0, d1 + u1) with u0 + u1 s ~= d2 s^2 (relinearisation key)."""
        d0, d1, d2 = d
        q = self.q[: d0.shape[0]]
        k0, k1 = self.keyswitch(d2, 0)
        return Ciphertext(np.stack([C.vadd(d0, k0, q), C.vadd(d1, k1, q)]), scale)

    def modup_digit(self, d, j):
        """Digit j of d (rows at level l) extended to the basis q_0..q_{l-1}, p_0..p_{k-1}.

        Rows inside the digit are copied; every other row is the fast basis
        conversion of the digit's rows (approximate: off by u*Q_j, 0 <= u < alpha)."""
        l = d.shape[0]
        basis = self.q[:l] + self.p
        lo, hi = j * self.alpha, min((j + 1) * self.alpha, l)
        others = [m for m in range(l + self.k) if not lo <= m < hi]
        ext = np.empty((l + self.k, self.N), np.uint64)
        ext[lo:hi] = d[lo:hi]
        ext[others] = C.bconv(d[lo:hi], self.q[lo:hi], [basis[m] for m in others])
        return ext

    def moddown(self, u, l):
        """(x_Q - BConv_{P->Q}(x_P)) * P^-1 mod each q_i (no correction)."""
        q = self.q[:l]
        conv = C.bconv(u[l:], self.p, q)
        pinv = [pow(self.Pprod % qi, -1, qi) for qi in q]
        return C.vscale(C.vsub(u[:l], conv, q), pinv, q)

    def keyswitch(self, d, key_id):
        """(u0, u1) at level l with u0 + u1 s ~= d s' (s' = the key's source secret)."""
        l = d.shape[0]
        basis = self.q[:l] + self.p
        rows = list(range(l)) + list(range(self.L, self.L + self.k))
        K = self.keys[key_id]
        beta = -(-l // self.alpha)
        u0 = np.zeros((l + self.k, self.N), np.uint64)
        u1 = np.zeros((l + self.k, self.N), np.uint64)
        for j in range(beta):
            ext = self.modup_digit(d, j)
            u0 = C.vadd(u0, C.polymul(ext, K[j, 0][rows], basis), basis)
            u1 = C.vadd(u1, C.polymul(ext, K[j, 1][rows], basis), basis)
        return self.moddown(u0, l), self.moddown(u1, l)

    def mul_relin(self, a, b):
        d0, d1, d2 = self.tensor(a, b)
        k0, k1 = self.keyswitch(d2, 0)
        q = self._q(a)
        return Ciphertext(np.stack([C.vadd(d0, k0, q), C.vadd(d1, k1, q)]), a.scale * b.scale)

    def automorph(self, ct, g):
        q = self._q(ct)
        return Ciphertext(np.stack([C.automorph(ct.c[i], q, g) for i in range(2)]), ct.scale)

    def rotate(self, ct, step):
        """Slot j of the result holds slot j+step of the input (left rotation)."""
        g = galois_element(step, self.N)
        if g == 1:
            return Ciphertext(ct.c.copy(), ct.scale)
        r = self.automorph(ct, g)
        k0, k1 = self.keyswitch(r.c[1], g)
        q = self._q(ct)
        return Ciphertext(np.stack([C.vadd(r.c[0], k0, q), k1]), ct.scale)

    def rotate_hoisted(self, ct, steps):
        """Rotations of one ciphertext sharing one ModUp (hoisting): the digits of c1 are
        extended once, and for each step the automorphism is applied to the extended digits
        (coefficient rows, mod each row's prime) before the inner product with that step's
        key and ModDown.  Fast basis conversion does not commute exactly with negating
        coefficients, so the result differs from rotate() by small noise, not in meaning."""
        l = ct.level
        basis = self.q[:l] + self.p
        rows = list(range(l)) + list(range(self.L, self.L + self.k))
        q = self._q(ct)
        beta = -(-l // self.alpha)
        exts = [self.modup_digit(ct.c[1], j) for j in range(beta)]
        out = []
        for step in steps:
            g = galois_element(step, self.N)
            K = self.keys[g]
            u0 = np.zeros((l + self.k, self.N), np.uint64)
            u1 = np.zeros((l + self.k, self.N), np.uint64)
            for j in range(beta):
                e = C.automorph(exts[j], basis, g)
                u0 = C.vadd(u0, C.polymul(e, K[j, 0][rows], basis), basis)
                u1 = C.vadd(u1, C.polymul(e, K[j, 1][rows], basis), basis)
            k0, k1 = self.moddown(u0, l), self.moddown(u1, l)
            c0 = C.automorph(ct.c[0], q, g)
            out.append(Ciphertext(np.stack([C.vadd(c0, k0, q), k1]), ct.scale))
        return out

    def rescale(self, ct, rounding=True):
        """Drop q_{l-1}: c'_k = (c_k + h - r) * p^-1 mod q_k, r = (c_{l-1} + h) mod p,
        h = floor(p/2) when rounding (h = 0 reproduces the floor of Eq. 1)."""
        l = ct.level
        assert l >= 2
        p = self.q[l - 1]
        h = p // 2 if rounding else 0
        out = np.empty((2, l - 1, self.N), np.uint64)
        for i in range(2):
            r = C.vadd(ct.c[i][l - 1: l], np.full((1, self.N), h, np.uint64), [p])[0]
            for kk in range(l - 1):
                qk = self.q[kk]
                rk = (r % np.uint64(qk)).reshape(1, -1)
                t = C.vsub(C.vadd(ct.c[i][kk: kk + 1], np.full((1, self.N), h % qk, np.uint64), [qk]), rk, [qk])
                out[i, kk] = C.vscale(t, [pow(p, -1, qk)], [qk])[0]
        return Ciphertext(out, ct.scale / p)

    def total_sum(self, ct, nslots=None):
        """TotalSum (Algorithm 2) with the reading i = 0 .. log2(t)-1, rotating by 2^i."""
        t = self.N // 2 if nslots is None else nslots
        for i in range(int(math.log2(t))):
            ct = self.add(ct, self.rotate(ct, 1 << i))
        return ct
