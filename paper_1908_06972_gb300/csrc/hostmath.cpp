// Host-side number theory and the CKKS encoder of the library.
//
//  * primes: for a bit size b the candidates 2^b - j 2N + 1 (j = 1, 2, ...), tested
//    with Miller-Rabin on the first 12 prime bases (deterministic below 3.3e24).
//  * psi: x^((q-1)/2N) for the smallest quadratic non-residue x (order exactly 2N).
//  * Gaussian table: T_j = floor(2^32 P(|X| <= j)), j < tail = floor(6 sigma), for
//    P(X = x) ~ exp(-x^2 / 2 sigma^2) on [-tail, tail] (Sec. 5.4: sigma = 3.2).
//  * ENCODE / DECODE (Sec. 2.3) over the canonical embedding: slot j <-> root
//    omega^(5^j mod 2N), omega = exp(i pi / N), evaluated with one N-point FFT
//    (the encoder runs on the client CPU, as in the paper's Sec. 4.1).
#include <cmath>
#include <complex>
#include <cstring>

#include "pft_internal.h"

namespace pft {

typedef unsigned __int128 u128;

u64 mulmod_host(u64 a, u64 b, u64 q) { return (u64)(((u128)a * b) % q); }
u64 powmod_host(u64 a, u64 e, u64 q) {
    u64 r = 1 % q;
    a %= q;
    while (e) {
        if (e & 1) r = mulmod_host(r, a, q);
        a = mulmod_host(a, a, q);
        e >>= 1;
    }
    return r;
}
u64 invmod_host(u64 a, u64 q) { return powmod_host(a, q - 2, q); }

static bool is_prime_u64(u64 n) {
    static const u64 bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return false;
    for (u64 p : bases)
        if (n % p == 0) return n == p;
    u64 d = n - 1;
    int s = 0;
    while ((d & 1) == 0) {
        d >>= 1;
        s++;
    }
    for (u64 a : bases) {
        u64 x = powmod_host(a, d, n);
        if (x == 1 || x == n - 1) continue;
        bool comp = true;
        for (int r = 1; r < s; r++) {
            x = mulmod_host(x, x, n);
            if (x == n - 1) {
                comp = false;
                break;
            }
        }
        if (comp) return false;
    }
    return true;
}

std::vector<u64> gen_primes(int logn, int bits, int count, const std::vector<u64>& exclude) {
    if (bits < 20 || bits > 60 || logn < 1 || logn > 20) fail(PFT_ERR_ARG, "prime size out of range (20..60 bits)");
    std::vector<u64> out;
    const u64 step = (u64)2 << logn;
    for (u64 j = 1; (int)out.size() < count; j++) {
        const u64 top = (u64)1 << bits;
        if (j * step >= top - ((u64)1 << (bits - 1))) fail(PFT_ERR_ARG, "not enough primes of this size for N");
        const u64 c = top - j * step + 1;
        bool ex = false;
        for (u64 e : exclude) ex |= (e == c);
        if (!ex && is_prime_u64(c)) out.push_back(c);
    }
    return out;
}

u64 root_2n_host(u64 q, int logn) {
    for (u64 x = 2;; x++)
        if (powmod_host(x, (q - 1) / 2, q) == q - 1) return powmod_host(x, (q - 1) >> (logn + 1), q);
}

std::vector<u32> gauss_cdt(double sigma, int* tail_out) {
    const int tail = (int)std::floor(6.0 * sigma);
    if (!(sigma > 0) || tail < 1 || tail > 64) fail(PFT_ERR_ARG, "sigma out of range");
    std::vector<double> rho(tail + 1);
    for (int k = 0; k <= tail; k++) rho[k] = std::exp(-(double)k * k / (2.0 * sigma * sigma));
    double z = rho[0];
    for (int k = 1; k <= tail; k++) z += 2 * rho[k];
    std::vector<u32> out(tail);
    double acc = rho[0];
    for (int j = 0; j < tail; j++) {
        if (j > 0) acc += 2 * rho[j];
        out[j] = (u32)std::floor(acc / z * 4294967296.0);
    }
    if (tail_out) *tail_out = tail;
    return out;
}

// ---- FFT (iterative radix-2, sign -1 forward / +1 backward, no scaling) ----------------
typedef std::complex<double> cd;
static void fft(std::vector<cd>& a, int sign) {
    const int n = (int)a.size();
    for (int i = 1, j = 0; i < n; i++) {
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) std::swap(a[i], a[j]);
    }
    std::vector<cd> root(n / 2);
    for (int k = 0; k < n / 2; k++) {
        const double ang = 2.0 * M_PI * k / n;
        root[k] = cd(std::cos(ang), sign * std::sin(ang));
    }
    for (int len = 2; len <= n; len <<= 1) {
        const int stride = n / len;
        for (int i = 0; i < n; i += len)
            for (int j = 0; j < len / 2; j++) {
                const cd u = a[i + j], v = a[i + j + len / 2] * root[j * stride];
                a[i + j] = u + v;
                a[i + j + len / 2] = u - v;
            }
    }
}

// m_k = (1/N) sum_u W[u] omega^(-(2u+1)k), W[(e_j - 1)/2] = scale z_j and
// W[(2N - e_j - 1)/2] = its conjugate, e_j = 5^j mod 2N.
bool encode_slots(int logn, const double* re_im, int n_slots, double scale, std::vector<i64>& coeffs) {
    const int n = 1 << logn;
    std::vector<cd> W(n, cd(0, 0));
    u64 e = 1;
    const u64 mask = (2ull << logn) - 1;
    for (int j = 0; j < n / 2; j++) {
        cd z(0, 0);
        if (j < n_slots) z = cd(re_im[2 * j], re_im[2 * j + 1]) * scale;
        W[(e - 1) / 2] = z;
        W[((2ull << logn) - e - 1) / 2] = std::conj(z);
        e = (e * 5) & mask;
    }
    fft(W, -1);
    coeffs.resize(n);
    for (int k = 0; k < n; k++) {
        const double ang = -M_PI * k / n;
        const double v = (W[k] * cd(std::cos(ang), std::sin(ang))).real() / n;
        const double r = std::round(v);  // half away from zero
        if (!(std::fabs(r) < 4611686018427387904.0)) return false;  // 2^62
        coeffs[k] = (i64)r;
    }
    return true;
}

// z_j = mu(omega^(e_j)) / scale, mu(omega^(2u+1)) = sum_k (mu_k omega^k) exp(2 pi i u k / N)
void decode_coeffs(int logn, const std::vector<double>& coeffs, double scale, double* re_im, int n_slots) {
    const int n = 1 << logn;
    std::vector<cd> a(n);
    for (int k = 0; k < n; k++) {
        const double ang = M_PI * k / n;
        a[k] = coeffs[k] * cd(std::cos(ang), std::sin(ang));
    }
    fft(a, +1);
    u64 e = 1;
    const u64 mask = (2ull << logn) - 1;
    for (int j = 0; j < n_slots && j < n / 2; j++) {
        const cd z = a[(e - 1) / 2] / scale;
        re_im[2 * j] = z.real();
        re_im[2 * j + 1] = z.imag();
        e = (e * 5) & mask;
    }
}

// ---- multi-precision CRT to centered doubles ---------------------------------------------
typedef std::vector<u64> Big;  // little-endian words, fixed length

static void big_muladd(Big& acc, const Big& x, u64 s) {  // acc += x * s
    u128 carry = 0;
    for (size_t i = 0; i < acc.size(); i++) {
        const u128 t = (u128)(i < x.size() ? x[i] : 0) * s + acc[i] + carry;
        acc[i] = (u64)t;
        carry = t >> 64;
    }
}
static void big_submul(Big& acc, const Big& x, u64 s) {  // acc -= x * s (result known >= 0)
    u128 carry = 0;
    u64 borrow = 0;
    for (size_t i = 0; i < acc.size(); i++) {
        const u128 t = (u128)(i < x.size() ? x[i] : 0) * s + carry;
        const u64 lo = (u64)t;
        carry = t >> 64;
        const u64 a = acc[i];
        const u64 r = a - lo - borrow;
        borrow = (a < lo || (a - lo) < borrow) ? 1 : 0;
        acc[i] = r;
    }
}
static int big_cmp(const Big& a, const Big& b) {
    for (size_t i = a.size(); i-- > 0;) {
        const u64 bi = i < b.size() ? b[i] : 0;
        if (a[i] != bi) return a[i] < bi ? -1 : 1;
    }
    return 0;
}
static double big_to_double(const Big& a) {
    double d = 0;
    for (size_t i = a.size(); i-- > 0;) d = d * 18446744073709551616.0 + (double)a[i];
    return d;
}

void crt_to_double(const std::vector<u64>& primes, const u64* rows, int n, std::vector<double>& out) {
    const int l = (int)primes.size();
    const size_t W = (size_t)l + 2;
    Big Q(W, 0);
    Q[0] = 1;
    for (u64 p : primes) {
        Big t(W, 0);
        big_muladd(t, Q, p);
        Q = t;
    }
    std::vector<Big> qhat(l, Big(W, 0));
    std::vector<u64> qhat_inv(l);
    for (int i = 0; i < l; i++) {
        Big h(W, 0);
        h[0] = 1;
        u64 hm = 1;
        for (int j = 0; j < l; j++)
            if (j != i) {
                Big t(W, 0);
                big_muladd(t, h, primes[j]);
                h = t;
                hm = mulmod_host(hm, primes[j] % primes[i], primes[i]);
            }
        qhat[i] = h;
        qhat_inv[i] = invmod_host(hm, primes[i]);
    }
    Big half(W, 0);  // floor(Q / 2)
    for (size_t i = 0; i < W; i++) half[i] = (Q[i] >> 1) | (i + 1 < W ? (Q[i + 1] << 63) : 0);
    out.resize(n);
    Big acc(W);
    for (int c = 0; c < n; c++) {
        std::fill(acc.begin(), acc.end(), 0);
        long double frac = 0;
        for (int i = 0; i < l; i++) {
            const u64 y = mulmod_host(rows[(size_t)i * n + c], qhat_inv[i], primes[i]);
            big_muladd(acc, qhat[i], y);
            frac += (long double)y / (long double)primes[i];
        }
        // acc = x + v Q with v = floor(sum y_i / q_i); subtract (v - 1) Q, then fix up
        long long v = (long long)std::floor(frac);
        if (v > 1) big_submul(acc, Q, (u64)(v - 1));
        while (big_cmp(acc, Q) >= 0) big_submul(acc, Q, 1);
        if (big_cmp(acc, half) > 0) {
            Big neg = Q;
            big_submul(neg, acc, 1);
            out[c] = -big_to_double(neg);
        } else {
            out[c] = big_to_double(acc);
        }
    }
}

}  // namespace pft
