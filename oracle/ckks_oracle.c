/*
 * Plain CPU oracle primitives for RNS-CKKS (test infrastructure only).
 *
 * This file is part of the ORACLE: a slow, obviously correct restatement of
 * what the GPU library computes, used only by tests/, by the smoke check and by
 * the CPU-baseline leg of the benchmark.  It shares no code, header, table or
 * constant with the CUDA library; nothing in the product links it.
 *
 * Every modular operation is the textbook one: a full 128-bit product followed
 * by the C `%` operator.  No Shoup, Barrett or Montgomery tricks, no lazy
 * reduction.  Each function handles a batch of limbs (rows) so that the Python
 * layer can stay readable; OpenMP only splits independent rows.
 *
 * Paper passages followed (PrivFT, arXiv 1908.06972):
 *   - ring R_q = Z_q[X]/(X^N+1) and the RNS chain of small primes: Sec. 2.3
 *   - HMUL / HMULPLAIN products are negacyclic polynomial products: Sec. 2.3
 *   - ROTATE = Galois automorphism X -> X^k of both polynomials: Sec. 2.3 and
 *     the rotation discussion of Sec. 5.3 (one key switch per automorphism).
 * The fast basis conversion (used by key switching) follows the RNS-CKKS
 * variant the paper builds on (its citation of the full-RNS CKKS scheme).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef uint64_t u64;
typedef int64_t i64;
typedef uint32_t u32;
typedef unsigned __int128 u128;

static u64 mulmod(u64 a, u64 b, u64 q) { return (u64)(((u128)a * b) % q); }
static u64 addmod(u64 a, u64 b, u64 q) { return (u64)(((u128)a + b) % q); }
static u64 submod(u64 a, u64 b, u64 q) { return (u64)(((u128)a + q - (b % q)) % q); }
static u64 powmod(u64 b, u64 e, u64 q) {
    u64 r = 1 % q;
    b %= q;
    while (e) {
        if (e & 1) r = mulmod(r, b, q);
        b = mulmod(b, b, q);
        e >>= 1;
    }
    return r;
}
/* inverse by Fermat (q prime) */
static u64 invmod(u64 a, u64 q) { return powmod(a, q - 2, q); }

/* ------------------------------------------------------------------------ */
/* ChaCha20 block function, RFC 8439 section 2.3                             */
/* ------------------------------------------------------------------------ */
static u32 rotl32(u32 x, int n) { return (x << n) | (x >> (32 - n)); }
#define QR(a, b, c, d)            \
    a += b; d ^= a; d = rotl32(d, 16); \
    c += d; b ^= c; b = rotl32(b, 12); \
    a += b; d ^= a; d = rotl32(d, 8);  \
    c += d; b ^= c; b = rotl32(b, 7);

void orc_chacha20_block(const u32 key[8], u32 counter, const u32 nonce[3], u32 out[16]) {
    u32 s[16], x[16];
    s[0] = 0x61707865u; s[1] = 0x3320646eu; s[2] = 0x79622d32u; s[3] = 0x6b206574u;
    for (int i = 0; i < 8; i++) s[4 + i] = key[i];
    s[12] = counter;
    s[13] = nonce[0]; s[14] = nonce[1]; s[15] = nonce[2];
    memcpy(x, s, sizeof(s));
    for (int r = 0; r < 10; r++) {
        QR(x[0], x[4], x[8], x[12]);
        QR(x[1], x[5], x[9], x[13]);
        QR(x[2], x[6], x[10], x[14]);
        QR(x[3], x[7], x[11], x[15]);
        QR(x[0], x[5], x[10], x[15]);
        QR(x[1], x[6], x[11], x[12]);
        QR(x[2], x[7], x[8], x[13]);
        QR(x[3], x[4], x[9], x[14]);
    }
    for (int i = 0; i < 16; i++) out[i] = x[i] + s[i];
}

/* The sampler's word stream: 64-bit word w of stream (seed, dom, obj, sub) is
 * built from the block with counter w/8, 32-bit words 2*(w%8) (low half) and
 * 2*(w%8)+1 (high half).  The 256-bit key is seed[0..3], each split into its
 * low then high 32-bit half; the nonce is (dom, obj, sub). */
void orc_stream_words(const u64 seed[4], u32 dom, u32 obj, u32 sub, u64 nwords, u64* out) {
    u32 key[8], nonce[3] = {dom, obj, sub}, blk[16];
    for (int i = 0; i < 4; i++) {
        key[2 * i] = (u32)(seed[i] & 0xffffffffu);
        key[2 * i + 1] = (u32)(seed[i] >> 32);
    }
    for (u64 w = 0; w < nwords; w++) {
        if (w % 8 == 0) orc_chacha20_block(key, (u32)(w / 8), nonce, blk);
        int r = (int)(w % 8);
        out[w] = (u64)blk[2 * r] | ((u64)blk[2 * r + 1] << 32);
    }
}

/* uniform residue mod q: coefficient c takes words 2c (low) and 2c+1 (high)
 * of the stream and reduces the 128-bit value mod q. */
void orc_sample_uniform(const u64 seed[4], u32 dom, u32 obj, u32 sub, u64 q, int n, u64* out) {
    u64* w = (u64*)malloc(sizeof(u64) * 2 * (size_t)n);
    orc_stream_words(seed, dom, obj, sub, 2 * (u64)n, w);
    for (int c = 0; c < n; c++) out[c] = (u64)((((u128)w[2 * c + 1]) << 64 | w[2 * c]) % q);
    free(w);
}

/* uniform ternary {-1,0,1}: word c mod 3, minus 1 */
void orc_sample_ternary(const u64 seed[4], u32 dom, u32 obj, u32 sub, int n, i64* out) {
    u64* w = (u64*)malloc(sizeof(u64) * (size_t)n);
    orc_stream_words(seed, dom, obj, sub, (u64)n, w);
    for (int c = 0; c < n; c++) out[c] = (i64)(w[c] % 3) - 1;
    free(w);
}

/* discrete Gaussian by cumulative table: magnitude k = number of thresholds
 * T[0..nt-1] that the top 32 bits of word c reach; the lowest bit of the word
 * is the sign. */
void orc_sample_gauss(const u64 seed[4], u32 dom, u32 obj, u32 sub, int n, const u32* cdt, int nt, i64* out) {
    u64* w = (u64*)malloc(sizeof(u64) * (size_t)n);
    orc_stream_words(seed, dom, obj, sub, (u64)n, w);
    for (int c = 0; c < n; c++) {
        u32 v = (u32)(w[c] >> 32);
        i64 k = 0;
        for (int j = 0; j < nt; j++)
            if (v >= cdt[j]) k++;
        out[c] = (w[c] & 1) ? -k : k;
    }
    free(w);
}

/* ------------------------------------------------------------------------ */
/* Row-wise modular vector arithmetic.  x, y, out are [rows][n]; row r is    */
/* reduced modulo q[r].                                                      */
/* ------------------------------------------------------------------------ */
void orc_vadd(const u64* x, const u64* y, const u64* q, int rows, int n, u64* out) {
    for (int r = 0; r < rows; r++)
        for (int c = 0; c < n; c++) out[(size_t)r * n + c] = addmod(x[(size_t)r * n + c], y[(size_t)r * n + c], q[r]);
}
void orc_vsub(const u64* x, const u64* y, const u64* q, int rows, int n, u64* out) {
    for (int r = 0; r < rows; r++)
        for (int c = 0; c < n; c++) out[(size_t)r * n + c] = submod(x[(size_t)r * n + c], y[(size_t)r * n + c], q[r]);
}
void orc_vmul(const u64* x, const u64* y, const u64* q, int rows, int n, u64* out) {
    for (int r = 0; r < rows; r++)
        for (int c = 0; c < n; c++) out[(size_t)r * n + c] = mulmod(x[(size_t)r * n + c] % q[r], y[(size_t)r * n + c] % q[r], q[r]);
}
/* out = x * s[r] mod q[r] (one scalar per row) */
void orc_vscale(const u64* x, const u64* s, const u64* q, int rows, int n, u64* out) {
    for (int r = 0; r < rows; r++)
        for (int c = 0; c < n; c++) out[(size_t)r * n + c] = mulmod(x[(size_t)r * n + c] % q[r], s[r] % q[r], q[r]);
}
/* reduce a signed integer polynomial into each row modulus */
void orc_reduce_signed(const i64* x, const u64* q, int rows, int n, u64* out) {
    for (int r = 0; r < rows; r++)
        for (int c = 0; c < n; c++) {
            __int128 m = ((__int128)x[c] % (__int128)q[r] + (__int128)q[r]) % (__int128)q[r];
            out[(size_t)r * n + c] = (u64)m;
        }
}

/* ------------------------------------------------------------------------ */
/* Negacyclic products in Z_q[X]/(X^n+1)                                     */
/* ------------------------------------------------------------------------ */

/* schoolbook: c_k = sum_{i+j=k} a_i b_j - sum_{i+j=k+n} a_i b_j */
static void negacyclic_schoolbook(const u64* a, const u64* b, u64 q, int n, u64* out) {
    for (int k = 0; k < n; k++) {
        u128 pos = 0, neg = 0;
        int cnt = 0;
        for (int i = 0; i < n; i++) {
            int j = k - i;
            u128 p = (u128)(a[i] % q) * (b[(j + n) % n] % q);
            if (j >= 0) pos += p; else neg += p;
            if (++cnt == 64) { pos %= q; neg %= q; cnt = 0; }
        }
        out[k] = submod((u64)(pos % q), (u64)(neg % q), q);
    }
}
void orc_polymul_schoolbook(const u64* a, const u64* b, const u64* q, int rows, int n, u64* out) {
#pragma omp parallel for schedule(dynamic)
    for (int r = 0; r < rows; r++) negacyclic_schoolbook(a + (size_t)r * n, b + (size_t)r * n, q[r], n, out + (size_t)r * n);
}

/* a primitive 2n-th root of unity: x^((q-1)/2n) for the smallest quadratic
 * non-residue x (its n-th power is -1, so its order is exactly 2n). */
static u64 root_2n(u64 q, int n) {
    for (u64 x = 2;; x++)
        if (powmod(x, (q - 1) / 2, q) == q - 1) return powmod(x, (q - 1) / (2 * (u64)n), q);
}

/* textbook iterative cyclic transform (bit-reversal, then butterflies of
 * growing length) with root w of order n */
static void cyclic_ntt(u64* a, int n, u64 w, u64 q) {
    for (int i = 1, j = 0; i < n; i++) {
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) { u64 t = a[i]; a[i] = a[j]; a[j] = t; }
    }
    for (int len = 2; len <= n; len <<= 1) {
        u64 wl = powmod(w, (u64)(n / len), q);
        for (int i = 0; i < n; i += len) {
            u64 wc = 1;
            for (int j = 0; j < len / 2; j++) {
                u64 u = a[i + j], v = mulmod(a[i + j + len / 2], wc, q);
                a[i + j] = addmod(u, v, q);
                a[i + j + len / 2] = submod(u, v, q);
                wc = mulmod(wc, wl, q);
            }
        }
    }
}

/* negacyclic product via a psi-twisted cyclic transform:
 * a'_j = a_j psi^j, b'_j = b_j psi^j, c' = IDFT(DFT(a') . DFT(b')), c_j = c'_j psi^-j */
static void negacyclic_ntt(const u64* a, const u64* b, u64 q, int n, u64* out) {
    u64 psi = root_2n(q, n), w = mulmod(psi, psi, q);
    u64* x = (u64*)malloc(sizeof(u64) * n);
    u64* y = (u64*)malloc(sizeof(u64) * n);
    u64 pj = 1;
    for (int j = 0; j < n; j++) {
        x[j] = mulmod(a[j] % q, pj, q);
        y[j] = mulmod(b[j] % q, pj, q);
        pj = mulmod(pj, psi, q);
    }
    cyclic_ntt(x, n, w, q);
    cyclic_ntt(y, n, w, q);
    for (int j = 0; j < n; j++) x[j] = mulmod(x[j], y[j], q);
    cyclic_ntt(x, n, invmod(w, q), q);
    u64 ninv = invmod((u64)n % q, q), psi_inv = invmod(psi, q);
    pj = ninv;
    for (int j = 0; j < n; j++) {
        out[j] = mulmod(x[j], pj, q);
        pj = mulmod(pj, psi_inv, q);
    }
    free(x);
    free(y);
}
void orc_polymul(const u64* a, const u64* b, const u64* q, int rows, int n, u64* out) {
#pragma omp parallel for schedule(dynamic)
    for (int r = 0; r < rows; r++) negacyclic_ntt(a + (size_t)r * n, b + (size_t)r * n, q[r], n, out + (size_t)r * n);
}

/* one coefficient k of the negacyclic product, by its defining sum (spot
 * checks of large products) */
u64 orc_polymul_coeff(const u64* a, const u64* b, u64 q, int n, int k) {
    u64 acc = 0;
    for (int i = 0; i < n; i++) {
        int j = k - i;
        u64 p = mulmod(a[i] % q, b[(j + n) % n] % q, q);
        acc = (j >= 0) ? addmod(acc, p, q) : submod(acc, p, q);
    }
    return acc;
}

/* ------------------------------------------------------------------------ */
/* Galois automorphism X -> X^g on coefficient vectors (g odd, mod 2n):      */
/* coefficient i moves to i*g mod 2n, negated when that index is >= n.       */
/* ------------------------------------------------------------------------ */
void orc_automorph(const u64* x, const u64* q, int rows, int n, u64 g, u64* out) {
    for (int r = 0; r < rows; r++)
        for (int i = 0; i < n; i++) {
            u64 e = ((u64)i * g) % (2 * (u64)n);
            u64 v = x[(size_t)r * n + i] % q[r];
            if (e < (u64)n) out[(size_t)r * n + e] = v;
            else out[(size_t)r * n + (e - n)] = submod(0, v, q[r]);
        }
}

/* ------------------------------------------------------------------------ */
/* Fast (approximate) RNS basis conversion.  For each coefficient, with       */
/* inputs x_i mod s_i (i < ns) and Qs = prod s_i, qhat_i = Qs / s_i:          */
/*   y_i   = x_i * (qhat_i)^-1 mod s_i                                       */
/*   out_m = sum_i y_i * (qhat_i mod d_m)   mod d_m                          */
/* The result is (x + u*Qs) mod d_m for some 0 <= u < ns.                     */
/* ------------------------------------------------------------------------ */
void orc_bconv(const u64* in, const u64* s, int ns, const u64* d, int nd, int n, u64* out) {
    u64* qhat_inv = (u64*)malloc(sizeof(u64) * ns);
    u64* qhat_mod = (u64*)malloc(sizeof(u64) * (size_t)ns * nd);
    for (int i = 0; i < ns; i++) {
        u64 h = 1;
        for (int i2 = 0; i2 < ns; i2++)
            if (i2 != i) h = mulmod(h, s[i2] % s[i], s[i]);
        qhat_inv[i] = invmod(h, s[i]);
        for (int m = 0; m < nd; m++) {
            u64 hm = 1;
            for (int i2 = 0; i2 < ns; i2++)
                if (i2 != i) hm = mulmod(hm, s[i2] % d[m], d[m]);
            qhat_mod[(size_t)i * nd + m] = hm;
        }
    }
#pragma omp parallel for schedule(static)
    for (int c = 0; c < n; c++) {
        for (int m = 0; m < nd; m++) {
            u64 acc = 0;
            for (int i = 0; i < ns; i++) {
                u64 y = mulmod(in[(size_t)i * n + c] % s[i], qhat_inv[i], s[i]);
                acc = addmod(acc, mulmod(y % d[m], qhat_mod[(size_t)i * nd + m], d[m]), d[m]);
            }
            out[(size_t)m * n + c] = acc;
        }
    }
    free(qhat_inv);
    free(qhat_mod);
}

/* ------------------------------------------------------------------------ */
/* The GPU library keeps polynomials in an evaluation ("NTT") domain.  Its     */
/* documented layout: entry i holds a(psi^(2*brv(i)+1)), brv = log2(n)-bit    */
/* bit reversal, psi the chain's primitive 2n-th root.  These two functions   */
/* evaluate that definition directly (O(n^2) / O(n) per entry).              */
/* ------------------------------------------------------------------------ */
static u64 brv(u64 x, int bits) {
    u64 r = 0;
    for (int b = 0; b < bits; b++) r |= ((x >> b) & 1) << (bits - 1 - b);
    return r;
}
void orc_eval_at(const u64* a, u64 psi, u64 q, int logn, const i64* idx, int nidx, u64* out) {
    int n = 1 << logn;
    u64* pw = (u64*)malloc(sizeof(u64) * 2 * (size_t)n);
    pw[0] = 1;
    for (int e = 1; e < 2 * n; e++) pw[e] = mulmod(pw[e - 1], psi, q);
#pragma omp parallel for schedule(static)
    for (int t = 0; t < nidx; t++) {
        u64 e = 2 * brv((u64)idx[t], logn) + 1, acc = 0;
        for (int j = 0; j < n; j++) acc = addmod(acc, mulmod(a[j] % q, pw[(e * (u64)j) % (2 * (u64)n)], q), q);
        out[t] = acc;
    }
    free(pw);
}

/* The inverse of that layout: the coefficients of the polynomial whose value at
 * psi^(2*brv(i)+1) is A[i].  With V_m = A[brv(m)] = sum_j (a_j psi^j) w^(m j),
 * w = psi^2, the twisted coefficients are the inverse cyclic transform of V:
 * a_j = n^-1 psi^-j sum_m V_m w^(-m j). */
void orc_interp_layout(const u64* A, u64 psi, u64 q, int logn, u64* out) {
    int n = 1 << logn;
    u64* v = (u64*)malloc(sizeof(u64) * (size_t)n);
    for (int m = 0; m < n; m++) v[m] = A[brv((u64)m, logn)] % q;
    cyclic_ntt(v, n, invmod(mulmod(psi, psi, q), q), q);
    u64 ninv = invmod((u64)n % q, q), psi_inv = invmod(psi, q), pj = ninv;
    for (int j = 0; j < n; j++) {
        out[j] = mulmod(v[j], pj, q);
        pj = mulmod(pj, psi_inv, q);
    }
    free(v);
}
