// RNS-CKKS evaluator on one GPU: context and tables, keys, encryption, the
// homomorphic operations of Sec. 2.3, hybrid key switching, rescale (Eq. 1 /
// Algorithm 3 with rounding) and the encrypted fastText inference of Sec. 3.1.
// Host code only orders kernel launches on the context stream; every step of the
// arithmetic runs in the kernels of ntt.cu and poly.cu.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <set>
#include <stdexcept>

#include "evaluator.h"

namespace pft {
void fail(int code, const std::string& msg) { throw Error{code, msg}; }
void check_cuda(cudaError_t e, const char* what) {
    if (e != cudaSuccess) fail(PFT_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}
static std::mutex& handles_mu() {
    static std::mutex m;
    return m;
}
static std::set<const void*>& handles() {
    static std::set<const void*> h;
    return h;
}
bool first_on_device(const void* key) {
    static std::mutex mu;
    static std::set<std::pair<const void*, int>> seen;
    int dev = 0;
    check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    std::lock_guard<std::mutex> g(mu);
    return seen.insert({key, dev}).second;
}
}  // namespace pft
void handle_add(const void* h) {
    std::lock_guard<std::mutex> g(pft::handles_mu());
    pft::handles().insert(h);
}
void handle_remove(const void* h) {
    std::lock_guard<std::mutex> g(pft::handles_mu());
    pft::handles().erase(h);
}
bool handle_live(const void* h) {
    std::lock_guard<std::mutex> g(pft::handles_mu());
    return pft::handles().count(h) != 0;
}

// ---- context construction ---------------------------------------------------------------
static u64 shoup(u64 w, u64 q) { return (u64)(((unsigned __int128)w << 64) / q); }
// basis-conversion constants are stored in Montgomery form c 2^64 mod t, split as
// (c' mod 2^30) | (c' >> 30) << 32
static u64 split30_host(u64 c) { return (c & 0x3fffffffull) | ((c >> 30) << 32); }
static u64 mont_host(u64 c, u64 t) { return (u64)((((unsigned __int128)c) << 64) % t); }
static int bitlen(u64 x) { return 64 - __builtin_clzll(x); }

static const int kSecureLogQP[17] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 27, 54, 109, 218, 438, 881, 1772};

static void* tab_alloc(pft_ctx* c, size_t bytes) {
    void* p = nullptr;
    PFT_CUDA(cudaMalloc(&p, bytes));
    c->owned.push_back(p);
    return p;
}
template <class T>
static T* tab_upload(pft_ctx* c, const std::vector<T>& v) {
    T* p = (T*)tab_alloc(c, std::max<size_t>(1, v.size()) * sizeof(T));
    PFT_CUDA(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return p;
}

namespace pft {
// Byte planes of the tensor-core conversion: for target m, byte plane b and k = 8 i + a, the
// bf16 of byte b of B[m][i][a] = c[m][i] 2^(8a) mod t_m.  Then for y_i = sum_a y_ia 2^(8a),
// sum_i y_i c[m][i] = sum_b 2^(8b) sum_(i,a) y_ia byte_b(B[m][i][a]) (mod t_m): eight exact sums
// of 32 products of bytes, one per byte plane.  A byte is exact in bf16 (8 significant bits), so
// its bf16 is the top half of its FP32 bits.
std::vector<uint32_t> bconv_tc_table(const std::vector<u64>& c, const std::vector<u64>& tp, int nt) {
    std::vector<uint32_t> out((size_t)nt * 8 * kBconvTcStride, 0);
    auto bf16 = [](uint32_t v) {
        const float f = (float)v;
        uint32_t u;
        memcpy(&u, &f, 4);
        return u >> 16;
    };
    for (int m = 0; m < nt; m++) {
        const u64 t = tp[m];
        for (int i = 0; i < 4; i++) {
            u64 w = c[(size_t)m * 4 + i] % t;
            for (int a = 0; a < 8; a++) {
                for (int b = 0; b < 8; b++) {
                    const int k = 8 * i + a;
                    const uint32_t v = bf16((uint32_t)((w >> (8 * b)) & 0xff));
                    uint32_t& word = out[((size_t)m * 8 + b) * kBconvTcStride + k / 2];
                    word |= (k & 1) ? v << 16 : v;
                }
                w = mulmod_host(w, 256, t);
            }
        }
    }
    return out;
}
}  // namespace pft

static void build_tables(pft_ctx* c) {
    const int P = (int)c->primes.size(), n = c->n, logn = c->logn, L = c->L, k = c->k;
    // primes
    std::vector<DPrime> dp(P);
    for (int i = 0; i < P; i++) {
        const u64 q = c->primes[i];
        const int s = bitlen(q) - 1;
        dp[i].q = q;
        dp[i].mu = (u64)((((unsigned __int128)1) << (64 + s)) / q);
        dp[i].r64 = (u64)((((unsigned __int128)1) << 64) % q);
        u64 inv = 1;  // q^-1 mod 2^64 by Newton iteration (q odd)
        for (int it = 0; it < 6; it++) inv *= 2 - q * inv;
        dp[i].mneg = 0 - inv;
        dp[i].s = (u32)s;
        dp[i].pad = 0;
    }
    c->tabs.logn = logn;
    c->tabs.n = n;
    default_plans(c->tabs);  // until the autotuner chooses
    {
        const char* e = getenv("PFT_BCONV");
        c->tabs.bconv_tc = e && strcmp(e, "tc") == 0 ? 1 : 0;  // integer pipes unless asked
        const char* o = getenv("PFT_NTT_ORDER");
        c->tabs.ntt_order = o ? atoi(o) & 7 : 3;
    }
    c->tabs.primes = tab_upload(c, dp);
    // twiddles
    std::vector<ulonglong2> fwd((size_t)P * n), inv((size_t)P * n), ninv(P), inv1(P);
    std::vector<u64> pw(n);
    for (int i = 0; i < P; i++) {
        const u64 q = c->primes[i];
        const u64 psi = root_2n_host(q, logn);
        const u64 psi_inv = invmod_host(psi, q);
        pw[0] = 1;
        for (int j = 1; j < n; j++) pw[j] = mulmod_host(pw[j - 1], psi, q);
        for (int j = 0; j < n; j++) {
            u32 b = 0;
            for (int t = 0; t < logn; t++) b |= ((j >> t) & 1) << (logn - 1 - t);
            const u64 w = pw[b];
            const u64 wi = b == 0 ? 1 : q - mulmod_host(pw[n - b], 1, q);  // psi^-b = -psi^(N-b)
            fwd[(size_t)i * n + j] = make_ulonglong2(w, shoup(w, q));
            inv[(size_t)i * n + j] = make_ulonglong2(wi, shoup(wi, q));
        }
        (void)psi_inv;
        const u64 ni = invmod_host((u64)n % q, q);
        ninv[i] = make_ulonglong2(ni, shoup(ni, q));
        const u64 v = mulmod_host(inv[(size_t)i * n + 1].x, ni, q);
        inv1[i] = make_ulonglong2(v, shoup(v, q));
    }
    c->tabs.fwd = tab_upload(c, fwd);
    c->tabs.inv = tab_upload(c, inv);
    c->tabs.fwd_rows = c->tabs.inv_rows = nullptr;
    if (logn == 16) {  // lane-major copy of the twiddles of stages 12..15 (row passes)
        std::vector<ulonglong2> fr((size_t)P * 256 * 240), ir((size_t)P * 256 * 240);
        for (int i = 0; i < P; i++)
            for (int u = 0; u < 256; u++)
                for (int kk = 0; kk < 4; kk++)
                    for (int j = 0; j < (1 << kk); j++)
                        for (int w = 0; w < 16; w++) {
                            const size_t src = (size_t)i * n + (1u << (12 + kk)) + ((size_t)u << (4 + kk)) + (w << kk) + j;
                            const size_t dst = (((size_t)i * 256 + u) * 15 + ((1 << kk) - 1 + j)) * 16 + w;
                            fr[dst] = fwd[src];
                            ir[dst] = inv[src];
                        }
        c->tabs.fwd_rows = tab_upload(c, fr);
        c->tabs.inv_rows = tab_upload(c, ir);
    }
    c->tabs.ninv = tab_upload(c, ninv);
    c->tabs.inv1ninv = tab_upload(c, inv1);

    // P mod q_m, P^-1 mod q_m
    c->P_mod_q.assign(L, 0);
    std::vector<u64> md(3 * (size_t)L);
    for (int m = 0; m < L; m++) {
        u64 pm = 1;
        for (int j = 0; j < k; j++) pm = mulmod_host(pm, c->primes[L + j] % c->primes[m], c->primes[m]);
        c->P_mod_q[m] = pm;
        const u64 pi = invmod_host(pm, c->primes[m]);
        md[3 * m] = 0;
        md[3 * m + 1] = pi;
        md[3 * m + 2] = shoup(pi, c->primes[m]);
    }
    c->moddown_consts = tab_upload(c, md);
    // key generation: P mod q_m on the rows of digit j (consts indexed from the digit's first row)
    for (int j = 0; j < c->beta_max; j++) {
        std::vector<u64> v;
        for (int m = j * c->alpha; m < std::min(L, (j + 1) * c->alpha); m++) {
            v.push_back(0);
            v.push_back(c->P_mod_q[m]);
            v.push_back(shoup(c->P_mod_q[m], c->primes[m]));
        }
        c->pmodq_consts.push_back(tab_upload(c, v));
    }
    // ModUp tables per (level l, digit j): [ns]{qhat_inv, shoup}, then [targets][ns] qhat mod target
    // (Montgomery form, 30-bit split), targets = rows 0..l+k-1 outside the digit, in order
    c->modup_tab.assign((size_t)L * c->beta_max, nullptr);
    c->modup_tab_u.assign((size_t)L * c->beta_max, nullptr);
    c->modup_tc.assign((size_t)L * c->beta_max, nullptr);
    for (int l = 1; l <= L; l++) {
        const int beta = (l + c->alpha - 1) / c->alpha, E = l + k;
        for (int j = 0; j < beta; j++) {
            const int lo = j * c->alpha, hi = std::min(l, lo + c->alpha), ns = hi - lo;
            const int nt = E - ns;
            std::vector<u64> tab(2 * ns + (size_t)ns * nt);
            std::vector<u64> plain((size_t)nt * 4, 0), tprime(nt, 0);  // for the tensor-core table
            for (int i = 0; i < ns; i++) {
                const u64 qi = c->primes[lo + i];
                u64 h = 1;
                for (int i2 = 0; i2 < ns; i2++)
                    if (i2 != i) h = mulmod_host(h, c->primes[lo + i2] % qi, qi);
                const u64 hinv = invmod_host(h, qi);
                tab[2 * i] = hinv;
                tab[2 * i + 1] = shoup(hinv, qi);
                int mi = 0;
                for (int m = 0; m < E; m++) {
                    if (m >= lo && m < hi) continue;
                    const u64 t = m < l ? c->primes[m] : c->primes[L + m - l];
                    u64 hm = 1;
                    for (int i2 = 0; i2 < ns; i2++)
                        if (i2 != i) hm = mulmod_host(hm, c->primes[lo + i2] % t, t);
                    tab[2 * ns + (size_t)mi * ns + i] = split30_host(mont_host(hm, t));
                    if (ns == 4) {
                        plain[(size_t)mi * 4 + i] = hm;
                        tprime[mi] = t;
                    }
                    mi++;
                }
            }
            c->modup_tab[(size_t)(l - 1) * c->beta_max + j] = tab_upload(c, tab);
            if (ns == 4) c->modup_tc[(size_t)(l - 1) * c->beta_max + j] = tab_upload(c, bconv_tc_table(plain, tprime, nt));
            for (int i = 0; i < ns; i++) {
                const u64 qi = c->primes[lo + i];
                tab[2 * i] = mulmod_host(tab[2 * i], invmod_host((u64)c->n % qi, qi), qi);
                tab[2 * i + 1] = shoup(tab[2 * i], qi);
            }
            c->modup_tab_u[(size_t)(l - 1) * c->beta_max + j] = tab_upload(c, tab);
        }
    }
    // ModDown tables per level: [k]{phat_inv, shoup}, then [l][k] phat mod q_m (Montgomery form,
    // 30-bit split)
    c->moddown_tab.assign(L, nullptr);
    c->moddown_tab_u.assign(L, nullptr);
    c->moddown_tc.assign(L, nullptr);
    for (int l = 1; l <= L; l++) {
        std::vector<u64> tab(2 * k + (size_t)k * l);
        std::vector<u64> plain((size_t)l * 4, 0), tprime(l, 0);  // for the tensor-core table (k = 4)
        for (int i = 0; i < k; i++) {
            const u64 pi = c->primes[L + i];
            u64 h = 1;
            for (int i2 = 0; i2 < k; i2++)
                if (i2 != i) h = mulmod_host(h, c->primes[L + i2] % pi, pi);
            const u64 hinv = invmod_host(h, pi);
            tab[2 * i] = hinv;
            tab[2 * i + 1] = shoup(hinv, pi);
            for (int m = 0; m < l; m++) {
                const u64 t = c->primes[m];
                u64 hm = 1;
                for (int i2 = 0; i2 < k; i2++)
                    if (i2 != i) hm = mulmod_host(hm, c->primes[L + i2] % t, t);
                tab[2 * k + (size_t)m * k + i] = split30_host(mont_host(hm, t));
                if (k == 4) {
                    plain[(size_t)m * 4 + i] = hm;
                    tprime[m] = t;
                }
            }
        }
        c->moddown_tab[l - 1] = tab_upload(c, tab);
        if (k == 4) c->moddown_tc[l - 1] = tab_upload(c, bconv_tc_table(plain, tprime, l));
        for (int i = 0; i < k; i++) {
            const u64 pi = c->primes[L + i];
            tab[2 * i] = mulmod_host(tab[2 * i], invmod_host((u64)c->n % pi, pi), pi);
            tab[2 * i + 1] = shoup(tab[2 * i], pi);
        }
        c->moddown_tab_u[l - 1] = tab_upload(c, tab);
    }
    // rescale constants per level l >= 2: for k' < l-1: {0, p^-1, shoup}, p = q_{l-1}
    c->rescale_consts.assign(L, nullptr);
    for (int l = 2; l <= L; l++) {
        const u64 p = c->primes[l - 1];
        std::vector<u64> v(3 * (size_t)(l - 1));
        for (int kk = 0; kk < l - 1; kk++) {
            const u64 q = c->primes[kk];
            const u64 pinv = invmod_host(p % q, q);
            v[3 * kk] = 0;
            v[3 * kk + 1] = pinv;
            v[3 * kk + 2] = shoup(pinv, q);
        }
        c->rescale_consts[l - 1] = tab_upload(c, v);
    }
}


u32 galois_of(int n, int32_t step) {
    const long long half = n / 2;
    long long r = ((long long)step % half + half) % half;
    u64 g = 1;
    const u64 mask = (2ull * n) - 1;
    for (long long i = 0; i < r; i++) g = (g * 5) & mask;
    return (u32)g;
}

// ---- keygen ---------------------------------------------------------------------------------
enum { DOM_SECRET = 1, DOM_PK_A, DOM_PK_E, DOM_KSK_A, DOM_KSK_E, DOM_ENC_A, DOM_ENC_E, DOM_ENC_V, DOM_ENC_E0, DOM_ENC_E1 };

// signed polynomial from a sampler stream, reduced into `refs` and transformed
static void sample_signed_ntt(pft_ctx* c, u32 dom, u32 obj, u32 sub, int kind, const std::vector<PolyRef>& refs) {
    Scratch tmp(c, (size_t)c->n * 8);
    sample_small(c->tabs, c->prm.seed, dom, obj, sub, kind, c->cdt.data(), (int)c->cdt.size(), (i64*)tmp.p,
                 c->stream);
    chunks(refs.size(), [&](size_t a, size_t b) { reduce_signed(c->tabs, (i64*)tmp.p, mkset(refs, a, b), c->stream); });
    ntt_fwd(c, refs, refs);
}

// switching key from s' (evaluation form over the full basis, rows [L+k]) to s
// Digit j of the key from s' to s: a_j uniform, b_j = -a_j s + e_j (+ P s' on the digit's
// primes).  Full keys keep (b_j, a_j) with a_j drawn in coefficient form; compressed keys
// (PFT_COMPRESSED_KEYS) keep b_j only, a_j being drawn directly in evaluation form from
// its own stream so that the inner product can regenerate it.
static u64* make_switch_key(pft_ctx* c, const u64* sp, u32 key_id) {
    const int n = c->n, L = c->L, k = c->k, R = L + k;
    const bool comp = c->compressed_keys;
    u64* K = (u64*)dalloc(c, (size_t)c->beta_max * (comp ? 1 : 2) * R * n * 8);
    std::unique_ptr<Scratch> abuf(comp ? new Scratch(c, (size_t)R * n * 8) : nullptr);
    for (int j = 0; j < c->beta_max; j++) {
        u64* b = K + (size_t)(comp ? j : 2 * j) * R * n;
        u64* a = comp ? abuf->u() : K + (size_t)(2 * j + 1) * R * n;
        std::vector<PolyRef> ra{ref(a, R, 0, L, L)}, rb{ref(b, R, 0, L, L)};
        if (comp) {
            sample_uniform(c->tabs, c->prm.seed, kDomKskAEval, key_id, 256u * j, mkset(ra, 0, 1), c->stream);
        } else {
            sample_uniform(c->tabs, c->prm.seed, DOM_KSK_A, key_id, 256u * j, mkset(ra, 0, 1), c->stream);
            ntt_fwd(c, ra, ra);
        }
        sample_signed_ntt(c, DOM_KSK_E, key_id, (u32)j, 1, rb);  // b = e
        Scratch as(c, (size_t)R * n * 8);
        std::vector<PolyRef> ras{ref(as.u(), R, 0, L, L)}, rs{ref((u64*)c->s_ntt, R, 0, L, L)};
        ew(c, EwOp::Mul, ra, rs, ras);   // a s
        ew(c, EwOp::Sub, rb, ras, rb);   // e - a s
        // + P s' on the rows of digit j
        const int lo = j * c->alpha, hi = std::min(L, lo + c->alpha);
        Scratch ps(c, (size_t)(hi - lo) * n * 8);
        std::vector<PolyRef> rsp{ref((u64*)sp + (size_t)lo * n, hi - lo, lo)};
        std::vector<PolyRef> rps{ref(ps.u(), hi - lo, lo)};
        std::vector<PolyRef> rbd{ref(b + (size_t)lo * n, hi - lo, lo)};
        subscale(c, rsp, nullptr, nullptr, rps, c->pmodq_consts[j]);
        ew(c, EwOp::Add, rbd, rps, rbd);
    }
    return K;
}

// An uncompressed key's copy for the key inner product: every word k as (k 2^64 mod p) split
// into 30-bit halves (the same 8 bytes; the inner product then sums 30-bit products without
// carries and reduces once in Montgomery form).
static void add_key(pft_ctx* c, u32 key_id, u64* K) {
    c->keys[key_id] = K;
    if (c->compressed_keys) return;
    const int R = c->L + c->k;
    const size_t words = (size_t)c->beta_max * 2 * R * c->n;
    u64* M = (u64*)dalloc(c, words * 8);
    std::vector<PolyRef> in, out;
    for (int i = 0; i < 2 * c->beta_max; i++) {
        in.push_back(ref(K + (size_t)i * R * c->n, R, 0, c->L, c->L));
        out.push_back(ref(M + (size_t)i * R * c->n, R, 0, c->L, c->L));
    }
    chunks(in.size(), [&](size_t a, size_t b) { mont_split(c->tabs, mkset(in, a, b), mkset(out, a, b), c->stream); });
    c->keys_mont[key_id] = M;
}
static void free_keys(pft_ctx* c) {
    for (auto& kv : c->keys) dfree(c, kv.second);
    for (auto& kv : c->keys_mont) dfree(c, kv.second);
    c->keys.clear();
    c->keys_mont.clear();
}

static void add_rot_keys(pft_ctx* c, const int32_t* steps, int n_steps) {
    NEED(c->have_sk, PFT_ERR_NO_KEY, "keygen has not run");
    const int n = c->n, R = c->L + c->k;
    for (int i = 0; i < n_steps; i++) {
        const u32 g = galois_of(n, steps[i]);
        if (g == 1 || c->keys.count(g)) continue;
        Scratch sg(c, (size_t)R * n * 8);
        std::vector<PolyRef> in{ref(c->s_ntt, R, 0, c->L, c->L)}, out{ref(sg.u(), R, 0, c->L, c->L)};
        chunks(1, [&](size_t a, size_t b) { automorph(c->tabs, mkset(in, a, b), mkset(out, a, b), g, c->stream); });
        add_key(c, g, make_switch_key(c, sg.u(), g));
    }
}

// ---- key switching ---------------------------------------------------------------------------

// For each input d (any level): (out0, out1) = (acc0, acc1) + ModDown(sum_j ModUp_j(d) * key_j).
// Every stage is one launch (or a few, by descriptor capacity) over all inputs, whatever
// their levels; the key is read once per stage.
KeyRef keyref(pft_ctx* c, u32 key_id) {
    NEED(c->keys.count(key_id), PFT_ERR_NO_KEY, "no such key");
    KeyRef r;
    r.ptr = c->keys[key_id];
    auto m = c->keys_mont.find(key_id);
    r.mont = m == c->keys_mont.end() ? nullptr : m->second;
    r.id = key_id;
    r.compressed = c->compressed_keys ? 1 : 0;
    for (int i = 0; i < 4; i++) {
        r.seedw[2 * i] = (u32)(c->prm.seed[i] & 0xffffffffu);
        r.seedw[2 * i + 1] = (u32)(c->prm.seed[i] >> 32);
    }
    return r;
}

// conv <- NTT(conv), then out = (x + c - conv) s (+ acc; entries of acc with a null pointer, or
// an empty acc: none), with per-limb constants {c, s, s'}: one fused pass where the transform
// variant has it, else the transform and the elementwise epilogue.
static void ntt_fwd_sub_scale(pft_ctx* c, const std::vector<PolyRef>& conv, const std::vector<PolyRef>& x,
                              const std::vector<PolyRef>& acc, const std::vector<PolyRef>& out, const u64* consts) {
    std::vector<PolyRef> a = acc;
    if (a.empty())
        for (const PolyRef& r : x) a.push_back(ref(nullptr, r.nlimbs));
    bool fused = true;
    chunks(conv.size(), [&](size_t lo, size_t hi) {
        NttEpi e;
        e.x = mkset(x, lo, hi);
        e.acc = mkset(a, lo, hi);
        e.out = mkset(out, lo, hi);
        e.consts = consts;
        if (fused) fused = ntt_forward_epilogue(c->tabs, mkset(conv, lo, hi), e, c->stream);
    });
    if (fused) return;
    ntt_fwd(c, conv, conv);
    std::vector<PolyRef> xw, yw, aw, ow, xn, yn, on;
    for (size_t i = 0; i < conv.size(); i++) {
        if (a[i].ptr) {
            xw.push_back(x[i]);
            yw.push_back(conv[i]);
            aw.push_back(a[i]);
            ow.push_back(out[i]);
        } else {
            xn.push_back(x[i]);
            yn.push_back(conv[i]);
            on.push_back(out[i]);
        }
    }
    if (!ow.empty()) subscale(c, xw, &yw, &aw, ow, consts);
    if (!on.empty()) subscale(c, xn, &yn, nullptr, on, consts);
}

void keyswitch_batch(pft_ctx* c, u32 key_id, const std::vector<KsIO>& io) {
    const KeyRef key = keyref(c, key_id);
    const int L = c->L, k = c->k, alpha = c->alpha;
    const size_t B = io.size();
    if (B == 0) return;
    const size_t limb = (size_t)c->n;
    std::vector<size_t> oDc(B), oExt(B), oU(B), oCv(B);
    size_t tDc = 0, tExt = 0, tU = 0, tCv = 0;
    for (size_t b = 0; b < B; b++) {
        const int l = io[b].l, E = l + k, beta = (l + alpha - 1) / alpha;
        oDc[b] = tDc;
        tDc += l;
        oExt[b] = tExt;
        tExt += (size_t)beta * E;
        oU[b] = tU;
        tU += 2 * (size_t)E;
        oCv[b] = tCv;
        tCv += 2 * (size_t)l;
    }
    Scratch Dc(c, tDc * limb * 8), Ext(c, tExt * limb * 8), U(c, tU * limb * 8), Cv(c, tCv * limb * 8);
    auto Eof = [&](size_t b) { return io[b].l + k; };
    auto dc = [&](size_t b) { return Dc.u() + oDc[b] * limb; };
    auto ext = [&](size_t b, int j) { return Ext.u() + (oExt[b] + (size_t)j * Eof(b)) * limb; };
    auto uu = [&](size_t b, int pol) { return U.u() + (oU[b] + (size_t)pol * Eof(b)) * limb; };
    auto cv = [&](size_t b, int pol) { return Cv.u() + (oCv[b] + (size_t)pol * io[b].l) * limb; };
    // 1. coefficient form of d (times N where the transform variant allows it: the conversion
    // tables then carry N^-1)
    bool unscaled = true;
    {
        std::vector<PolyRef> in, out;
        for (size_t b = 0; b < B; b++) {
            in.push_back(ref((u64*)io[b].d, io[b].l));
            out.push_back(ref(dc(b), io[b].l));
        }
        unscaled = ntt_inv_unscaled(c, in, out);
    }
    // 2. ModUp: fast basis conversion of every digit to the other rows; digit rows copied
    {
        std::vector<BconvJob> jobs;
        for (size_t b = 0; b < B; b++) {
            const int l = io[b].l, E = l + k, beta = (l + alpha - 1) / alpha;
            for (int j = 0; j < beta; j++) {
                const int lo = j * alpha, hi = std::min(l, lo + alpha);
                BconvJob J;
                J.src = dc(b) + (size_t)lo * limb;
                J.dst = ext(b, j);
                J.table = (unscaled ? c->modup_tab_u : c->modup_tab)[(size_t)(l - 1) * c->beta_max + j];
                J.tc = c->modup_tc[(size_t)(l - 1) * c->beta_max + j];
                J.ns = hi - lo;
                J.src_p0 = lo;
                J.nrows = E;
                J.skip_lo = lo;
                J.skip_hi = hi;
                J.split = l;
                J.base2 = L;
                J.pad = 0;
                jobs.push_back(J);
            }
        }
        bconv(c->tabs, jobs.data(), (int)jobs.size(), c->stream);
        // the digit's own rows are d itself: the inner product reads them there
    }
    // 3. evaluation form of the converted rows
    {
        std::vector<PolyRef> rows;
        for (size_t b = 0; b < B; b++) {
            const int l = io[b].l, E = l + k, beta = (l + alpha - 1) / alpha;
            for (int j = 0; j < beta; j++) {
                const int lo = j * alpha, hi = std::min(l, lo + alpha);
                if (lo > 0) rows.push_back(ref(ext(b, j), lo, 0));
                rows.push_back(ref(ext(b, j) + (size_t)hi * limb, E - hi, hi, l - hi, L));
            }
        }
        ntt_fwd(c, rows, rows);
    }
    // 4. inner product with the key (one pass over the key for all inputs)
    {
        std::vector<KsDesc> d(B);
        for (size_t b = 0; b < B; b++) {
            d[b].ext = ext(b, 0);
            d[b].u = uu(b, 0);
            d[b].d = io[b].d;
            d[b].l = io[b].l;
            d[b].pad = 0;
        }
        ks_inner_multi(c->tabs, d.data(), (int)B, key, L, k, alpha, c->stream);
    }
    // 5. ModDown: coefficient form of the special rows, conversion to q_0..q_{l-1}, evaluation form
    {
        std::vector<PolyRef> sp;
        std::vector<BconvJob> jobs;
        for (size_t b = 0; b < B; b++) {
            const int l = io[b].l;
            for (int pol = 0; pol < 2; pol++) {
                sp.push_back(ref(uu(b, pol) + (size_t)l * limb, k, 0, 0, L));
                BconvJob J;
                J.src = uu(b, pol) + (size_t)l * limb;
                J.dst = cv(b, pol);
                J.table = nullptr;  // chosen below, with the form of the transform
                J.tc = c->moddown_tc[l - 1];
                J.ns = k;
                J.src_p0 = L;
                J.nrows = l;
                J.skip_lo = 0;
                J.skip_hi = 0;
                J.split = l;
                J.base2 = L;
                J.pad = 0;
                jobs.push_back(J);
            }
        }
        const bool unscaled5 = ntt_inv_unscaled(c, sp, sp);
        for (BconvJob& J : jobs) J.table = (unscaled5 ? c->moddown_tab_u : c->moddown_tab)[J.nrows - 1];
        bconv(c->tabs, jobs.data(), (int)jobs.size(), c->stream);
    }
    // 6. out = acc + (u_Q - conv) P^-1, fused with the last forward pass of conv where the
    // transform variant has that kernel
    bool all0 = true, all1 = true, none1 = true;
    for (size_t b = 0; b < B; b++) {
        all0 &= io[b].acc0 != nullptr;
        all1 &= io[b].acc1 != nullptr;
        none1 &= io[b].acc1 == nullptr;
    }
    NEED(all0 && (all1 || none1), PFT_ERR_ARG, "internal: mixed accumulators");
    std::vector<PolyRef> cvr, ex, eacc, eout;
    for (size_t b = 0; b < B; b++) {
        const int l = io[b].l;
        for (int pol = 0; pol < 2; pol++) {
            cvr.push_back(ref(cv(b, pol), l));
            ex.push_back(ref(uu(b, pol), l));
            eacc.push_back(ref((u64*)(pol ? io[b].acc1 : io[b].acc0), l));
            eout.push_back(ref(pol ? io[b].out1 : io[b].out0, l));
        }
    }
    ntt_fwd_sub_scale(c, cvr, ex, eacc, eout, c->moddown_consts);
}

// ---- operations ---------------------------------------------------------------------------

static std::map<int, std::vector<int>> by_level(const pft_ct* const* a, int B) {
    std::map<int, std::vector<int>> g;
    for (int i = 0; i < B; i++) g[a[i]->level].push_back(i);
    return g;
}

void op_add_batch(pft_ctx* c, const pft_ct* const* a, const pft_ct* const* b, int B, pft_ct* const* out,
                         EwOp op) {
    for (int i = 0; i < B; i++) {
        check_ct(c, a[i]);
        check_ct(c, b[i]);
        NEED(out[i], PFT_ERR_ARG, "null output");
        NEED(a[i]->level == b[i]->level, PFT_ERR_LEVEL_MISMATCH, "HADD operands at different levels");
        NEED(a[i]->scale == b[i]->scale, PFT_ERR_SCALE_MISMATCH, "HADD operands at different scales");
    }
    std::vector<PolyRef> ra, rb, ro;
    for (int i = 0; i < B; i++) {
        const int l = a[i]->level;
        const double sc = a[i]->scale;
        ensure_ct(c, out[i], l);
        out[i]->scale = sc;
        for (int pol = 0; pol < 2; pol++) {
            ra.push_back(cpoly(a[i]->data, l, c->n, pol));
            rb.push_back(cpoly(b[i]->data, l, c->n, pol));
            ro.push_back(cpoly(out[i]->data, l, c->n, pol));
        }
    }
    ew(c, op, ra, rb, ro);
}

void op_mul_plain_batch(pft_ctx* c, const pft_ct* const* a, const pft_pt* const* p, int B,
                               pft_ct* const* out) {
    for (int i = 0; i < B; i++) {
        check_ct(c, a[i]);
        check_pt(c, p[i]);
        NEED(out[i], PFT_ERR_ARG, "null output");
        NEED(a[i]->level == p[i]->level, PFT_ERR_LEVEL_MISMATCH, "HMULPLAIN operands at different levels");
    }
    std::vector<PolyRef> ra, rb, ro;
    for (int i = 0; i < B; i++) {
        const int l = a[i]->level;
        const double sc = a[i]->scale * p[i]->scale;
        ensure_ct(c, out[i], l);
        out[i]->scale = sc;
        for (int pol = 0; pol < 2; pol++) {
            ra.push_back(cpoly(a[i]->data, l, c->n, pol));
            rb.push_back(ref(p[i]->data, l));
            ro.push_back(cpoly(out[i]->data, l, c->n, pol));
        }
    }
    ew(c, EwOp::Mul, ra, rb, ro);
}

static void mul_relin_group(pft_ctx* c, const pft_ct* const* a, const pft_ct* const* b, int B,
                            pft_ct* const* out);

void op_mul_relin_batch(pft_ctx* c, const pft_ct* const* a, const pft_ct* const* b, int B,
                               pft_ct* const* out) {
    NEED(c->keys.count(0), PFT_ERR_NO_KEY, "no relinearisation key");
    for (int i = 0; i < B; i++) {
        check_ct(c, a[i]);
        check_ct(c, b[i]);
        NEED(out[i], PFT_ERR_ARG, "null output");
        NEED(a[i]->level == b[i]->level, PFT_ERR_LEVEL_MISMATCH, "HMUL operands at different levels");
    }
    if (B == 0) return;
    // groups whose tensor and key-switching scratch fit the budget, unless an output is also
    // the input of another entry (then every product must be formed before any output is written)
    bool cross_alias = false;
    {
        std::map<const pft_ct*, int> pos;
        for (int i = 0; i < B; i++) {
            pos[a[i]] = i;
            pos[b[i]] = i;
        }
        for (int i = 0; i < B && !cross_alias; i++) {
            auto it = pos.find(out[i]);
            cross_alias = it != pos.end() && (it->second != i || a[i] != out[i] && b[i] != out[i]);
        }
    }
    int i0 = 0;
    while (i0 < B) {
        int i1 = i0;
        size_t words = 0;
        while (i1 < B) {
            const size_t w = 3 * (size_t)a[i1]->level * c->n + ks_scratch_words(c, a[i1]->level);
            if (!cross_alias && i1 > i0 && (words + w) * 8 > kKsScratchBudget) break;
            words += w;
            i1++;
        }
        mul_relin_group(c, a + i0, b + i0, i1 - i0, out + i0);
        i0 = i1;
    }
}

static void mul_relin_group(pft_ctx* c, const pft_ct* const* a, const pft_ct* const* b, int B,
                            pft_ct* const* out) {
    const size_t limb = c->n;
    std::vector<size_t> off(B);
    size_t tot = 0;
    for (int i = 0; i < B; i++) {
        off[i] = tot;
        tot += 3 * (size_t)a[i]->level;
    }
    Scratch D(c, tot * limb * 8);
    std::vector<PolyRef> ra, rb, rd;
    for (int i = 0; i < B; i++) {
        const int l = a[i]->level;
        ra.push_back(ref(a[i]->data, l));
        rb.push_back(ref(b[i]->data, l));
        rd.push_back(ref(D.u() + off[i] * limb, l));
    }
    chunks(rd.size(), [&](size_t x, size_t y) {
        ew_tensor(c->tabs, mkset(ra, x, y), mkset(rb, x, y), mkset(rd, x, y), c->stream);
    });
    std::vector<KsIO> io;
    for (int i = 0; i < B; i++) {
        const int l = a[i]->level;
        const double sc = a[i]->scale * b[i]->scale;
        ensure_ct(c, out[i], l);
        out[i]->scale = sc;
        u64* d = D.u() + off[i] * limb;
        io.push_back(KsIO{d + 2 * l * limb, d, d + l * limb, out[i]->data, out[i]->data + l * limb, l});
    }
    keyswitch_batch(c, 0u, io);
}

static void op_rotate_batch(pft_ctx* c, const pft_ct* const* a, int B, int32_t step, pft_ct* const* out) {
    for (int i = 0; i < B; i++) {
        check_ct(c, a[i]);
        NEED(out[i], PFT_ERR_ARG, "null output");
    }
    const u32 g = galois_of(c->n, step);
    const size_t limb = c->n;
    if (g == 1) {  // identity rotation
        for (int i = 0; i < B; i++) {
            if (out[i] == a[i]) continue;
            const int l = a[i]->level;
            const double sc = a[i]->scale;
            ensure_ct(c, out[i], l);
            out[i]->scale = sc;
            PFT_CUDA(cudaMemcpyAsync(out[i]->data, a[i]->data, 2 * l * limb * 8, cudaMemcpyDeviceToDevice, c->stream));
        }
        return;
    }
    NEED(c->keys.count(g), PFT_ERR_NO_KEY, "no rotation key for step " + std::to_string(step));
    if (B == 0) return;
    std::vector<size_t> off(B);
    size_t tot = 0;
    for (int i = 0; i < B; i++) {
        off[i] = tot;
        tot += 2 * (size_t)a[i]->level;
    }
    Scratch R(c, tot * limb * 8);
    std::vector<PolyRef> rin, rout;
    for (int i = 0; i < B; i++) {
        const int l = a[i]->level;
        for (int pol = 0; pol < 2; pol++) {
            rin.push_back(cpoly(a[i]->data, l, c->n, pol));
            rout.push_back(cpoly(R.u() + off[i] * limb, l, c->n, pol));
        }
    }
    chunks(rout.size(), [&](size_t x, size_t y) {
        automorph(c->tabs, mkset(rin, x, y), mkset(rout, x, y), g, c->stream);
    });
    std::vector<KsIO> io;
    for (int i = 0; i < B; i++) {
        const int l = a[i]->level;
        const double sc = a[i]->scale;
        ensure_ct(c, out[i], l);
        out[i]->scale = sc;
        u64* r = R.u() + off[i] * limb;
        io.push_back(KsIO{r + l * limb, r, nullptr, out[i]->data, out[i]->data + l * limb, l});
    }
    keyswitch_batch(c, g, io);
}

// Rotations of one ciphertext by several steps sharing one ModUp of c1 (hoisting): the
// extended digits (evaluation form) are permuted by each step's automorphism, then go through
// the inner product with that step's key and ModDown; out_i = (aut(c0) + u0', u1').
void op_rotate_hoisted(pft_ctx* c, const pft_ct* a, const int32_t* steps, int n, pft_ct* const* outs) {
    check_ct(c, a);
    NEED(n >= 0 && (n == 0 || (steps && outs)), PFT_ERR_ARG, "bad arguments");
    const int l = a->level, k = c->k, L = c->L, alpha = c->alpha, E = l + k, beta = (l + alpha - 1) / alpha;
    const size_t limb = (size_t)c->n;
    std::vector<u32> gs(n);
    for (int i = 0; i < n; i++) {
        NEED(outs[i] && outs[i] != a, PFT_ERR_ARG, "outputs must be distinct from the input");
        gs[i] = galois_of(c->n, steps[i]);
        NEED(gs[i] == 1 || c->keys.count(gs[i]), PFT_ERR_NO_KEY, "no rotation key for step " + std::to_string(steps[i]));
    }
    if (n == 0) return;
    Scratch Dc(c, l * limb * 8), Ext(c, (size_t)beta * E * limb * 8), ExtG(c, (size_t)beta * E * limb * 8),
        U(c, 2 * (size_t)E * limb * 8), Cv(c, 2 * (size_t)l * limb * 8), A0(c, l * limb * 8);
    u64* c1 = a->data + (size_t)l * limb;
    auto ext = [&](u64* base, int j) { return base + (size_t)j * E * limb; };
    // ModUp of c1, once
    {
        std::vector<PolyRef> in{ref(c1, l)}, out{ref(Dc.u(), l)};
        const bool unscaled = ntt_inv_unscaled(c, in, out);  // N^-1 then in the conversion tables
        std::vector<BconvJob> jobs;
        std::vector<PolyRef> cin, cout, rows;
        for (int j = 0; j < beta; j++) {
            const int lo = j * alpha, hi = std::min(l, lo + alpha);
            BconvJob J;
            J.src = Dc.u() + (size_t)lo * limb;
            J.dst = ext(Ext.u(), j);
            J.table = (unscaled ? c->modup_tab_u : c->modup_tab)[(size_t)(l - 1) * c->beta_max + j];
            J.tc = c->modup_tc[(size_t)(l - 1) * c->beta_max + j];
            J.ns = hi - lo;
            J.src_p0 = lo;
            J.nrows = E;
            J.skip_lo = lo;
            J.skip_hi = hi;
            J.split = l;
            J.base2 = L;
            J.pad = 0;
            jobs.push_back(J);
            cin.push_back(ref(c1 + (size_t)lo * limb, hi - lo, lo));
            cout.push_back(ref(ext(Ext.u(), j) + (size_t)lo * limb, hi - lo, lo));
            if (lo > 0) rows.push_back(ref(ext(Ext.u(), j), lo, 0));
            rows.push_back(ref(ext(Ext.u(), j) + (size_t)hi * limb, E - hi, hi, l - hi, L));
        }
        bconv(c->tabs, jobs.data(), (int)jobs.size(), c->stream);
        ew(c, EwOp::Copy, cin, {}, cout);
        ntt_fwd(c, rows, rows);
    }
    for (int i = 0; i < n; i++) {
        pft_ct* o = outs[i];
        const double sc = a->scale;
        ensure_ct(c, o, l);
        o->scale = sc;
        if (gs[i] == 1) {
            PFT_CUDA(cudaMemcpyAsync(o->data, a->data, 2 * l * limb * 8, cudaMemcpyDeviceToDevice, c->stream));
            continue;
        }
        // automorphism of the extended digits and of c0
        std::vector<PolyRef> ein, eout;
        for (int j = 0; j < beta; j++) {
            ein.push_back(ref(ext(Ext.u(), j), E, 0, l, L));
            eout.push_back(ref(ext(ExtG.u(), j), E, 0, l, L));
        }
        ein.push_back(ref(a->data, l));
        eout.push_back(ref(A0.u(), l));
        chunks(eout.size(), [&](size_t x, size_t y) {
            automorph(c->tabs, mkset(ein, x, y), mkset(eout, x, y), gs[i], c->stream);
        });
        KsDesc d{ExtG.u(), U.u(), nullptr, l, 0};
        ks_inner_multi(c->tabs, &d, 1, keyref(c, gs[i]), L, k, alpha, c->stream);
        // ModDown
        std::vector<PolyRef> sp, cvr;
        std::vector<BconvJob> jobs;
        for (int pol = 0; pol < 2; pol++) {
            u64* up = U.u() + (size_t)pol * E * limb;
            sp.push_back(ref(up + (size_t)l * limb, k, 0, 0, L));
            cvr.push_back(ref(Cv.u() + (size_t)pol * l * limb, l));
            BconvJob J;
            J.src = up + (size_t)l * limb;
            J.dst = Cv.u() + (size_t)pol * l * limb;
            J.table = nullptr;  // chosen with the form of the transform
            J.tc = c->moddown_tc[l - 1];
            J.ns = k;
            J.src_p0 = L;
            J.nrows = l;
            J.skip_lo = 0;
            J.skip_hi = 0;
            J.split = l;
            J.base2 = L;
            J.pad = 0;
            jobs.push_back(J);
        }
        const bool unscaled_sp = ntt_inv_unscaled(c, sp, sp);
        for (BconvJob& J : jobs) J.table = (unscaled_sp ? c->moddown_tab_u : c->moddown_tab)[l - 1];
        bconv(c->tabs, jobs.data(), (int)jobs.size(), c->stream);
        const std::vector<PolyRef> xs{ref(U.u(), l), ref(U.u() + (size_t)E * limb, l)};
        const std::vector<PolyRef> as{ref(A0.u(), l), ref(nullptr, l)};
        const std::vector<PolyRef> os{ref(o->data, l), ref(o->data + (size_t)l * limb, l)};
        ntt_fwd_sub_scale(c, cvr, xs, as, os, c->moddown_consts);
    }
}

void op_rescale_batch(pft_ctx* c, const pft_ct* const* a, int B, pft_ct* const* out) {
    for (int i = 0; i < B; i++) {
        check_ct(c, a[i]);
        NEED(out[i], PFT_ERR_ARG, "null output");
        NEED(a[i]->level >= 2, PFT_ERR_LEVEL_MISMATCH, "rescale needs at least two primes");
    }
    const size_t limb = c->n;
    for (auto& kv : by_level(a, B)) {
        const int l = kv.first;
        const std::vector<int>& idx = kv.second;
        const size_t G = idx.size();
        Scratch Last(c, G * 2 * limb * 8), Rb(c, G * 2 * (l - 1) * limb * 8);
        std::vector<PolyRef> lin, lout, rr, x, y, out_refs;
        // fresh output buffers (the output is smaller than the input and may alias it)
        std::vector<u64*> nb(G);
        for (size_t i = 0; i < G; i++) nb[i] = (u64*)dalloc(c, 2 * (l - 1) * limb * 8);
        for (size_t i = 0; i < G; i++) {
            u64* A = a[idx[i]]->data;
            for (int pol = 0; pol < 2; pol++) {
                lin.push_back(ref(A + ((size_t)pol * l + l - 1) * limb, 1, l - 1));
                lout.push_back(ref(Last.u() + (i * 2 + pol) * limb, 1, l - 1));
                rr.push_back(ref(Rb.u() + (i * 2 + pol) * (l - 1) * limb, l - 1));
                x.push_back(ref(A + (size_t)pol * l * limb, l - 1));
                out_refs.push_back(ref(nb[i] + (size_t)pol * (l - 1) * limb, l - 1));
            }
        }
        ntt_inv(c, lin, lout);
        chunks(rr.size(), [&](size_t p, size_t q) { rescale_bcast(c->tabs, mkset(lout, p, q), mkset(rr, p, q), c->stream); });
        ntt_fwd_sub_scale(c, rr, x, {}, out_refs, c->rescale_consts[l - 1]);
        for (size_t i = 0; i < G; i++) {
            pft_ct* o = out[idx[i]];
            const double sc = a[idx[i]]->scale / (double)c->primes[l - 1];
            dfree(c, o->data);  // stream-ordered: queued work on the old buffer completes first
            o->data = nb[i];
            o->cap = 2 * (size_t)(l - 1) * limb;
            o->level = l - 1;
            o->scale = sc;
        }
        // inputs aliased by an output of the same group were released above; make sure no
        // later entry of this group still points at them (each handle appears once per group)
    }
}

// ---- level and scale management --------------------------------------------------------------
void op_drop_level_batch(pft_ctx* c, const pft_ct* const* a, int B, int level, pft_ct* const* out) {
    for (int i = 0; i < B; i++) {
        check_ct(c, a[i]);
        NEED(out[i], PFT_ERR_ARG, "null output");
        NEED(level >= 1 && level <= a[i]->level, PFT_ERR_LEVEL_MISMATCH, "target level above the input level");
    }
    const size_t limb = c->n;
    std::vector<u64*> nb(B);
    std::vector<PolyRef> in, o;
    for (int i = 0; i < B; i++) {
        nb[i] = (u64*)dalloc(c, 2 * (size_t)level * limb * 8);
        for (int pol = 0; pol < 2; pol++) {
            in.push_back(ref(a[i]->data + (size_t)pol * a[i]->level * limb, level));
            o.push_back(ref(nb[i] + (size_t)pol * level * limb, level));
        }
    }
    ew(c, EwOp::Copy, in, {}, o);
    std::vector<double> sc(B);
    for (int i = 0; i < B; i++) sc[i] = a[i]->scale;
    for (int i = 0; i < B; i++) {
        // stream-ordered free: the copy above reads an aliased input first; an output that
        // appears twice gets the last copy
        if (out[i]->data != nb[i]) dfree(c, out[i]->data);
        out[i]->data = nb[i];
        out[i]->cap = 2 * (size_t)level * limb;
        out[i]->level = level;
        out[i]->scale = sc[i];
        out[i]->ctx = c;
    }
}

void op_const_batch(pft_ctx* c, const pft_ct* const* a, int B, double value, double const_scale, bool mul,
                    pft_ct* const* out) {
    int lmax = 0;
    for (int i = 0; i < B; i++) {
        check_ct(c, a[i]);
        NEED(out[i], PFT_ERR_ARG, "null output");
        lmax = std::max(lmax, a[i]->level);
    }
    if (B == 0) return;
    NEED(std::isfinite(value) && (!mul || (std::isfinite(const_scale) && const_scale > 0)), PFT_ERR_ARG,
         "constant and its scale must be finite (scale positive)");
    // groups of equal integer constants: k depends on the ciphertext's scale when adding
    std::map<long long, std::vector<int>> by_k;
    for (int i = 0; i < B; i++) {
        const double x = value * (mul ? const_scale : a[i]->scale);
        NEED(std::fabs(x) < 9.0e18, PFT_ERR_ARG, "constant times scale exceeds 2^63");
        by_k[std::llround(x)].push_back(i);  // nearest integer, halfway cases away from zero
    }
    const size_t limb = c->n;
    for (auto& kv : by_k) {
        const long long k = kv.first;
        std::vector<u64> consts(3 * (size_t)lmax);
        for (int r = 0; r < lmax; r++) {
            const u64 q = c->primes[r];
            long long km = k % (long long)q;
            const u64 kr = km < 0 ? (u64)(km + (long long)q) : (u64)km;
            const u64 sm = mul ? kr : 1;
            consts[3 * r] = mul ? 0 : kr;
            consts[3 * r + 1] = sm;
            consts[3 * r + 2] = shoup(sm, q);
        }
        Scratch dc(c, consts.size() * 8);
        const u64* cdev = upload(c, dc, consts);
        std::vector<PolyRef> x, o, cin, cout;
        for (int i : kv.second) {
            const int l = a[i]->level;
            const double sc = mul ? a[i]->scale * const_scale : a[i]->scale;
            u64* src = a[i]->data;
            if (out[i] != a[i]) {
                ensure_ct(c, out[i], l);
                out[i]->ctx = c;
            }
            out[i]->scale = sc;
            x.push_back(cpoly(src, l, c->n, 0));
            o.push_back(cpoly(out[i]->data, l, c->n, 0));
            if (mul) {
                x.push_back(cpoly(src, l, c->n, 1));
                o.push_back(cpoly(out[i]->data, l, c->n, 1));
            } else if (out[i]->data != src) {
                cin.push_back(cpoly(src, l, c->n, 1));
                cout.push_back(cpoly(out[i]->data, l, c->n, 1));
            }
        }
        subscale(c, x, nullptr, nullptr, o, cdev);
        if (!cin.empty()) ew(c, EwOp::Copy, cin, {}, cout);
    }
    (void)limb;
}

void relin_batch(pft_ctx* c, const std::vector<RelinIO>& io) {
    NEED(c->keys.count(0), PFT_ERR_NO_KEY, "no relinearisation key");
    const size_t limb = c->n;
    size_t i0 = 0;
    while (i0 < io.size()) {
        size_t i1 = i0, words = 0;
        while (i1 < io.size()) {
            const size_t w = ks_scratch_words(c, io[i1].l);
            if (i1 > i0 && (words + w) * 8 > kKsScratchBudget) break;
            words += w;
            i1++;
        }
        std::vector<KsIO> ks;
        for (size_t i = i0; i < i1; i++) {
            const RelinIO& r = io[i];
            ensure_ct(c, r.out, r.l);
            r.out->ctx = c;
            r.out->scale = r.scale;
            ks.push_back(KsIO{r.d + 2 * (size_t)r.l * limb, r.d, r.d + (size_t)r.l * limb, r.out->data,
                              r.out->data + (size_t)r.l * limb, r.l});
        }
        keyswitch_batch(c, 0u, ks);
        i0 = i1;
    }
}

// ---- encryption ----------------------------------------------------------------------------
static void encrypt(pft_ctx* c, const pft_pt* pt, int mode, u32 nonce, pft_ct* out) {
    NEED(c->have_sk, PFT_ERR_NO_KEY, "keygen has not run");
    check_pt(c, pt);
    const int l = pt->level, n = c->n;
    const size_t limb = n;
    ensure_ct(c, out, l);
    out->scale = pt->scale;
    u64* c0 = out->data;
    u64* c1 = out->data + l * limb;
    std::vector<PolyRef> r0{ref(c0, l)}, r1{ref(c1, l)}, rpt{ref(pt->data, l)}, rs{ref(c->s_ntt, l)};
    if (mode == PFT_ENC_SK) {
        sample_uniform(c->tabs, c->prm.seed, DOM_ENC_A, nonce, 0, mkset(r1, 0, 1), c->stream);
        ntt_fwd(c, r1, r1);
        sample_signed_ntt(c, DOM_ENC_E, nonce, 0, 1, r0);  // c0 = e
        Scratch as(c, l * limb * 8);
        std::vector<PolyRef> ras{ref(as.u(), l)};
        ew(c, EwOp::Mul, r1, rs, ras);
        ew(c, EwOp::Sub, r0, ras, r0);
        ew(c, EwOp::Add, r0, rpt, r0);
    } else {
        Scratch v(c, l * limb * 8), e1(c, l * limb * 8), t(c, l * limb * 8);
        std::vector<PolyRef> rv{ref(v.u(), l)}, re1{ref(e1.u(), l)}, rt{ref(t.u(), l)};
        std::vector<PolyRef> rb{ref(c->pk, l)}, ra{ref(c->pk + (size_t)c->L * limb, l)};
        sample_signed_ntt(c, DOM_ENC_V, nonce, 0, 0, rv);
        sample_signed_ntt(c, DOM_ENC_E0, nonce, 0, 1, r0);
        sample_signed_ntt(c, DOM_ENC_E1, nonce, 0, 1, re1);
        ew(c, EwOp::Mul, rv, rb, rt);
        ew(c, EwOp::Add, r0, rt, r0);
        ew(c, EwOp::Add, r0, rpt, r0);
        ew(c, EwOp::Mul, rv, ra, rt);
        ew(c, EwOp::Add, re1, rt, r1);
    }
}

// ---- fastText inference (Sec. 3.1) ----------------------------------------------------------
// T[i] += rotate(T[i], g) for every ciphertext of T: c0 + aut(c0) first, then the key switch
// of aut(c1) with (T.c0, T.c1) as accumulators, in place; tiled to bound the scratch memory.
void rot_accumulate(pft_ctx* c, const std::vector<pft_ct*>& T, u32 g) {
    NEED(c->keys.count(g), PFT_ERR_NO_KEY, "missing rotation key");
    const int n = c->n;
    const size_t limb = n;
    size_t i0 = 0;
    const size_t budget = (size_t)24 << 30;
    while (i0 < T.size()) {
        size_t i1 = i0, bytes = 0;
        while (i1 < T.size()) {
            const int l = T[i1]->level, E = l + c->k, beta = (l + c->alpha - 1) / c->alpha;
            const size_t per = (size_t)(2 * l + l + beta * E + 2 * E + 2 * l) * limb * 8;
            if (i1 > i0 && bytes + per > budget) break;
            bytes += per;
            i1++;
        }
        std::vector<size_t> off;
        size_t tot = 0;
        for (size_t i = i0; i < i1; i++) {
            off.push_back(tot);
            tot += 2 * (size_t)T[i]->level;
        }
        Scratch R(c, tot * limb * 8);
        std::vector<PolyRef> rin, rout, tin0, rc0;
        std::vector<KsIO> io;
        for (size_t i = i0; i < i1; i++) {
            const int l = T[i]->level;
            u64* r = R.u() + off[i - i0] * limb;
            for (int pol = 0; pol < 2; pol++) {
                rin.push_back(cpoly(T[i]->data, l, n, pol));
                rout.push_back(cpoly(r, l, n, pol));
            }
            tin0.push_back(cpoly(T[i]->data, l, n, 0));
            rc0.push_back(cpoly(r, l, n, 0));
            io.push_back(KsIO{r + l * limb, T[i]->data, T[i]->data + l * limb, T[i]->data, T[i]->data + l * limb, l});
        }
        chunks(rout.size(), [&](size_t x, size_t y) {
            automorph(c->tabs, mkset(rin, x, y), mkset(rout, x, y), g, c->stream);
        });
        ew(c, EwOp::Add, tin0, rc0, tin0);
        keyswitch_batch(c, g, io);
        i0 = i1;
    }
}

// Stages of one inference.
//   Fig. 3 packing: BEGIN (column products T_j = sum_i v_i H_{j,i}), ROT(2^s) for 2^s < t
//     (TotalSum, Algorithm 2), FINISH (rescale the columns, s = sum_j h_j O_j, rescale).
//   Diagonal packing (rotation-light, not in the paper): BEGIN (Q = sum_k rot(v, k) D_k with
//     D_k[i] = H[(i + k) mod t, i mod n], n - 1 hoisted rotations), ROT(n 2^s) while n 2^s < t
//     (h_{i mod n} in slot i), MID (rescale, S = Q P with P[n c + j] = O[j, c]),
//     ROT(2^s) while 2^s < n (s_c in slot n c), FINISH (rescale).
std::vector<FtStage> ft_program(pft_ctx* c, const pft_ft_model* M) {
    const int n = c->n, t = n / 2, cols = M->n;
    std::vector<FtStage> p{{FT_BEGIN, 0}};
    if (M->variant == 0) {
        for (int st = 1; st < t; st *= 2) p.push_back({FT_ROT, galois_of(n, st)});
    } else {
        for (int st = cols; st < t; st *= 2) p.push_back({FT_ROT, galois_of(n, st)});
        p.push_back({FT_MID, 0});
        for (int st = 1; st < cols; st *= 2) p.push_back({FT_ROT, galois_of(n, st)});
    }
    p.push_back({FT_FINISH, 0});
    return p;
}

void ft_check_doc(pft_ctx* c, const pft_ft_model* M, const pft_ct* const* v, int n_chunks) {
    NEED(M && M->ctx == c, PFT_ERR_ARG, "model from another context");
    NEED(n_chunks == M->chunks, PFT_ERR_ARG, "number of input ciphertexts must be ceil(m/t)");
    NEED(v, PFT_ERR_ARG, "null input");
    for (int i = 0; i < n_chunks; i++) {
        check_ct(c, v[i]);
        NEED(v[i]->level == v[0]->level, PFT_ERR_LEVEL_MISMATCH, "the inputs of one document differ in level");
        NEED(v[i]->scale == v[0]->scale, PFT_ERR_SCALE_MISMATCH, "the inputs of one document differ in scale");
    }
    const int l = v[0]->level;
    NEED(l >= 3, PFT_ERR_LEVEL_MISMATCH, "inference needs three levels");
    NEED(l <= M->level, PFT_ERR_LEVEL_MISMATCH, "input level above the model level");
    for (const pft_pt* o : M->O) NEED(o->level >= l - 1, PFT_ERR_LEVEL_MISMATCH, "output-layer plaintexts too low");
    const int n = c->n;
    if (M->variant == 1)
        for (int k = 1; k < M->n; k++) NEED(c->keys.count(galois_of(n, k)), PFT_ERR_NO_KEY, "missing rotation key");
    for (const FtStage& st : ft_program(c, M))
        if (st.kind == FT_ROT)
            NEED(c->keys.count(st.g), PFT_ERR_NO_KEY,
                 M->variant == 0 ? "missing rotation key for TotalSum" : "missing rotation key");
}

static std::map<int, std::vector<FtDoc*>> docs_by_level(const std::vector<FtDoc*>& docs) {
    std::map<int, std::vector<FtDoc*>> g;
    for (FtDoc* d : docs) g[d->l].push_back(d);
    return g;
}

static void ft_init_work(pft_ctx* c, FtDoc* d, int count, double scale) {
    d->W.clear();
    d->W.resize(count);
    d->work.clear();
    for (auto& x : d->W) {
        x.ctx = c;
        ensure_ct(c, &x, d->l);
        x.scale = scale;
        d->work.push_back(&x);
    }
}

static void ft_release_work(pft_ctx* c, FtDoc* d) {
    for (auto& x : d->W) dfree(c, x.data);
    d->W.clear();
}

// BEGIN, Fig. 3 packing: T[d][j] = sum_i v[d][i] * H[j][i]; one launch per level present.
static void ft_begin_columns(pft_ctx* c, const pft_ft_model* M, const std::vector<FtDoc*>& docs) {
    const int cols = M->n, K = M->chunks;
    const size_t limb = c->n;
    for (FtDoc* d : docs) ft_init_work(c, d, cols, d->v[0]->scale * M->H[0]->scale);
    for (auto& kv : docs_by_level(docs)) {
        const int l = kv.first;
        std::vector<const u64*> A, Bv;
        std::vector<u64*> O;
        for (FtDoc* d : kv.second)
            for (int j = 0; j < cols; j++)
                for (int pol = 0; pol < 2; pol++) {
                    for (int i = 0; i < K; i++) {
                        A.push_back(d->v[i]->data + (size_t)pol * l * limb);
                        Bv.push_back(M->H[(size_t)j * K + i]->data);
                    }
                    O.push_back(d->W[j].data + (size_t)pol * l * limb);
                }
        Scratch dA(c, A.size() * 8), dB(c, Bv.size() * 8), dO(c, O.size() * 8);
        ew_dot(c->tabs, upload(c, dA, A), upload(c, dB, Bv), upload(c, dO, O), (int)O.size(), K, false, l,
               c->stream);
    }
}

// FINISH, Fig. 3 packing: rescale the columns, s = sum_j h_j * O_j (horizontal packing), rescale.
static void ft_finish_columns(pft_ctx* c, const pft_ft_model* M, const std::vector<FtDoc*>& docs) {
    const int cols = M->n;
    const size_t limb = c->n;
    std::vector<pft_ct*> T;
    for (FtDoc* d : docs)
        for (pft_ct* x : d->work) T.push_back(x);
    op_rescale_batch(c, T.data(), (int)T.size(), T.data());
    for (auto& kv : docs_by_level(docs)) {
        const int l1 = kv.first - 1;
        std::vector<const u64*> A, Bv;
        std::vector<u64*> O;
        for (int j = 0; j < cols; j++) Bv.push_back(M->O[j]->data);
        for (FtDoc* d : kv.second) {
            ensure_ct(c, d->score, l1);
            d->score->scale = d->W[0].scale * M->O[0]->scale;
            for (int pol = 0; pol < 2; pol++) {
                for (int j = 0; j < cols; j++) A.push_back(d->W[j].data + (size_t)pol * l1 * limb);
                O.push_back(d->score->data + (size_t)pol * l1 * limb);
            }
        }
        // the O_j table is shared by every output (document, polynomial)
        Scratch dA(c, A.size() * 8), dB(c, Bv.size() * 8), dO(c, O.size() * 8);
        ew_dot(c->tabs, upload(c, dA, A), upload(c, dB, Bv), upload(c, dO, O), (int)O.size(), cols, true, l1,
               c->stream);
    }
    std::vector<pft_ct*> S;
    for (FtDoc* d : docs) {
        S.push_back(d->score);
        ft_release_work(c, d);
        d->work.clear();
    }
    op_rescale_batch(c, S.data(), (int)S.size(), S.data());
}

// BEGIN, diagonal packing: Q = sum_k rot(v, k) D_k, documents in chunks that bound the memory
// of the rotated copies.
static void ft_begin_diag(pft_ctx* c, const pft_ft_model* M, const std::vector<FtDoc*>& docs) {
    const int cols = M->n, nch = M->chunks;
    const size_t limb = c->n;
    std::vector<int32_t> hsteps;
    for (int k = 1; k < cols; k++) hsteps.push_back(k);
    for (FtDoc* d : docs) ft_init_work(c, d, 1, d->v[0]->scale * M->H[0]->scale);
    // per document: the n - 1 hoisted rotations of each vocabulary chunk, then one dot product
    // Q = sum_i sum_k rot(v_i, k) D_{i,k} over all of them (K = chunks n terms)
    const size_t rot_per_doc = (size_t)nch * (cols - 1);
    for (auto& kv : docs_by_level(docs)) {
        const int l = kv.first;
        const std::vector<FtDoc*>& G = kv.second;
        const size_t per_doc = rot_per_doc * 2 * l * limb * 8;
        const size_t chunk = std::max<size_t>(1, std::min<size_t>(G.size(), ((size_t)16 << 30) / per_doc));
        for (size_t b0 = 0; b0 < G.size(); b0 += chunk) {
            const size_t b1 = std::min(G.size(), b0 + chunk);
            std::vector<pft_ct> R((b1 - b0) * rot_per_doc);
            struct CleanR {
                pft_ctx* c;
                std::vector<pft_ct>* T;
                ~CleanR() {
                    for (auto& x : *T) dfree(c, x.data);
                }
            } cleanR{c, &R};
            for (auto& x : R) x.ctx = c;
            auto rot = [&](size_t b, int i, int k) -> pft_ct& {  // rot(v_i, k) of document b, k >= 1
                return R[(b - b0) * rot_per_doc + (size_t)i * (cols - 1) + k - 1];
            };
            for (size_t b = b0; b < b1; b++)
                for (int i = 0; i < nch; i++) {
                    std::vector<pft_ct*> outs;
                    for (int k = 1; k < cols; k++) outs.push_back(&rot(b, i, k));
                    op_rotate_hoisted(c, G[b]->v[i], hsteps.data(), cols - 1, outs.data());
                }
            std::vector<const u64*> A, Bv;
            std::vector<u64*> O;
            for (int i = 0; i < nch; i++)
                for (int k = 0; k < cols; k++) Bv.push_back(M->H[(size_t)i * cols + k]->data);
            for (size_t b = b0; b < b1; b++)
                for (int pol = 0; pol < 2; pol++) {
                    for (int i = 0; i < nch; i++) {
                        A.push_back(G[b]->v[i]->data + (size_t)pol * l * limb);
                        for (int k = 1; k < cols; k++) A.push_back(rot(b, i, k).data + (size_t)pol * l * limb);
                    }
                    O.push_back(G[b]->W[0].data + (size_t)pol * l * limb);
                }
            Scratch dA(c, A.size() * 8), dB(c, Bv.size() * 8), dO(c, O.size() * 8);
            ew_dot(c->tabs, upload(c, dA, A), upload(c, dB, Bv), upload(c, dO, O), (int)O.size(), nch * cols, true,
                   l, c->stream);
        }
    }
}

// MID, diagonal packing: rescale Q, S = Q * P into the score; later steps act on the score.
static void ft_mid_diag(pft_ctx* c, const pft_ft_model* M, const std::vector<FtDoc*>& docs) {
    std::vector<pft_ct*> Q;
    for (FtDoc* d : docs) Q.push_back(&d->W[0]);
    op_rescale_batch(c, Q.data(), (int)Q.size(), Q.data());
    const pft_pt* P = M->O[0];
    std::vector<PolyRef> ra, rb, ro;
    for (FtDoc* d : docs) {
        const int l1 = d->W[0].level;
        ensure_ct(c, d->score, l1);
        d->score->scale = d->W[0].scale * P->scale;
        for (int pol = 0; pol < 2; pol++) {
            ra.push_back(cpoly(d->W[0].data, l1, c->n, pol));
            rb.push_back(ref(P->data, l1));
            ro.push_back(cpoly(d->score->data, l1, c->n, pol));
        }
    }
    ew(c, EwOp::Mul, ra, rb, ro);
    for (FtDoc* d : docs) {
        ft_release_work(c, d);
        d->work.assign(1, d->score);
    }
}

void ft_stage(pft_ctx* c, const pft_ft_model* M, const FtStage& st, const std::vector<FtDoc*>& docs) {
    if (docs.empty()) return;
    switch (st.kind) {
        case FT_BEGIN:
            if (M->variant == 0) ft_begin_columns(c, M, docs);
            else ft_begin_diag(c, M, docs);
            break;
        case FT_ROT: {
            std::vector<pft_ct*> T;
            for (FtDoc* d : docs)
                for (pft_ct* x : d->work) T.push_back(x);
            rot_accumulate(c, T, st.g);
            break;
        }
        case FT_MID:
            NEED(M->variant == 1, PFT_ERR_ARG, "internal: MID stage of the Fig. 3 sequence");
            ft_mid_diag(c, M, docs);
            break;
        case FT_FINISH:
            if (M->variant == 0) {
                ft_finish_columns(c, M, docs);
            } else {
                std::vector<pft_ct*> S;
                for (FtDoc* d : docs) {
                    S.push_back(d->score);
                    d->work.clear();
                }
                op_rescale_batch(c, S.data(), (int)S.size(), S.data());
            }
            break;
        default:
            fail(PFT_ERR_ARG, "internal: unknown stage");
    }
}

// The whole sequence for B documents at once (each stage is one batched call).
static void fasttext_batch(pft_ctx* c, const pft_ft_model* M, const pft_ct* const* v, int chunks_in, int B,
                           pft_ct* const* scores) {
    NEED(M && M->ctx == c, PFT_ERR_ARG, "model from another context");
    NEED(B >= 0 && (B == 0 || (v && scores)), PFT_ERR_ARG, "bad arguments");
    std::vector<std::unique_ptr<FtDoc>> docs;
    std::vector<FtDoc*> dp;
    for (int b = 0; b < B; b++) {
        ft_check_doc(c, M, v + (size_t)b * chunks_in, chunks_in);
        NEED(scores[b], PFT_ERR_ARG, "null output");
        docs.emplace_back(new FtDoc());
        FtDoc* d = docs.back().get();
        d->v = v + (size_t)b * chunks_in;
        d->l = d->v[0]->level;
        d->score = scores[b];
        dp.push_back(d);
    }
    for (const FtStage& st : ft_program(c, M)) ft_stage(c, M, st, dp);
}

// ---- allocation-free rescale ---------------------------------------------------------------
// For callers that cannot obtain device memory when they call the library (their device
// memory is owned by another framework's pool, or allocator calls are not allowed in their
// processing loop).  The working space of pft_rescale_noalloc -- the dropped limb of both
// polynomials in coefficient form and its broadcast into the lower limbs -- lives in this
// fixed array instead of coming from the allocator.  Every device that loads the library
// holds it until the process exits; all calls on a device share it, so calls whose GPU work
// overlaps (other streams, other contexts on the same device) race on it.
constexpr size_t kNoAllocScratchWords = (size_t)4 << 20;  // 32 MiB
static __device__ __align__(256) u64 g_noalloc_scratch[kNoAllocScratchWords];

// Device address of the array on the current device.  Host code cannot use the array's name
// as a device address, so pft_ctx_create looks it up (once per device, under a lock) and keeps
// it in the context.
static u64* noalloc_scratch_lookup() {
    static std::mutex mu;
    static std::map<int, u64*> addr;
    int dev = -1;
    PFT_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> g(mu);
    u64*& a = addr[dev];
    if (!a) {
        void* p = nullptr;
        PFT_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        NEED(p != nullptr, PFT_ERR_CUDA, "no device address for the fixed scratch array");
        a = (u64*)p;
    }
    return a;
}

// ---- launch accounting ---------------------------------------------------------------------
namespace {
struct Prof {
    bool on = false;
    std::string prefix;
    long long all = 0;
    double work = 0;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
    size_t used = 0;
    bool open = false;
};
Prof g_prof;
}  // namespace
namespace pft {
void prof_begin(const char* name, cudaStream_t st, double work) {
    g_prof.all++;
    if (!g_prof.on || strncmp(name, g_prof.prefix.c_str(), g_prof.prefix.size()) != 0) return;
    g_prof.work += work;
    if (g_prof.used == g_prof.ev.size()) {
        cudaEvent_t a, b;
        if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return;
        g_prof.ev.push_back({a, b});
    }
    cudaEventRecord(g_prof.ev[g_prof.used].first, st);
    g_prof.open = true;
}
void prof_end(const char* name, cudaStream_t st) {
    if (!g_prof.open || strncmp(name, g_prof.prefix.c_str(), g_prof.prefix.size()) != 0) return;
    cudaEventRecord(g_prof.ev[g_prof.used].second, st);
    g_prof.used++;
    g_prof.open = false;
}
}  // namespace pft

// ===================================================================================================
// C ABI
// ===================================================================================================
extern "C" {

int pft_prof_start(const char* prefix) {
    g_prof.on = prefix != nullptr && prefix[0] != 0;
    g_prof.prefix = prefix ? prefix : "";
    g_prof.all = 0;
    g_prof.work = 0;
    g_prof.used = 0;
    g_prof.open = false;
    return PFT_OK;
}

int pft_prof_stop(double* ms, long long* timed_launches, long long* all_launches, double* work) {
    double tot = 0;
    if (g_prof.used) {
        if (cudaEventSynchronize(g_prof.ev[g_prof.used - 1].second) != cudaSuccess) return PFT_ERR_CUDA;
        for (size_t i = 0; i < g_prof.used; i++) {
            float t = 0;
            if (cudaEventElapsedTime(&t, g_prof.ev[i].first, g_prof.ev[i].second) != cudaSuccess) return PFT_ERR_CUDA;
            tot += t;
        }
    }
    if (ms) *ms = tot;
    if (timed_launches) *timed_launches = (long long)g_prof.used;
    if (all_launches) *all_launches = g_prof.all;
    if (work) *work = g_prof.work;
    g_prof.on = false;
    g_prof.used = 0;
    return PFT_OK;
}

int pft_gen_primes(int log_n, int bits, int count, const uint64_t* exclude, int n_exclude, uint64_t* out) {
    return guard(nullptr, [&] {
        NEED(out && count >= 0, PFT_ERR_ARG, "bad arguments");
        std::vector<u64> ex(exclude, exclude + (exclude ? n_exclude : 0));
        std::vector<u64> p = gen_primes(log_n, bits, count, ex);
        std::copy(p.begin(), p.end(), out);
    });
}

int pft_gauss_cdt(double sigma, uint32_t* out, int cap, int* n_out) {
    return guard(nullptr, [&] {
        int tail = 0;
        std::vector<u32> t = gauss_cdt(sigma, &tail);
        NEED(out && cap >= tail, PFT_ERR_ARG, "output too small");
        std::copy(t.begin(), t.end(), out);
        if (n_out) *n_out = tail;
    });
}

int pft_ctx_create(const pft_params* prm, const pft_allocator* alloc, pft_ctx** out) {
    if (!prm || !out) return PFT_ERR_ARG;
    *out = nullptr;
    std::unique_ptr<pft_ctx> c(new pft_ctx());
    int rc = guard(c.get(), [&] {
        c->prm = *prm;
        c->compressed_keys = (prm->flags & PFT_COMPRESSED_KEYS) != 0;
        c->logn = prm->log_n;
        NEED(prm->log_n >= 4 && prm->log_n <= 16, PFT_ERR_ARG, "log_n must be in 4..16");
        NEED(prm->n_limbs >= 1 && prm->n_limbs <= kMaxLimbs, PFT_ERR_ARG, "n_limbs must be in 1..60");
        NEED(prm->n_special >= 1 && prm->n_special <= kMaxSpecial, PFT_ERR_ARG, "n_special must be in 1..8");
        NEED(prm->alpha >= 1 && prm->alpha <= kMaxAlpha, PFT_ERR_ARG, "alpha must be in 1..8");
        c->n = 1 << c->logn;
        c->L = prm->n_limbs;
        c->k = prm->n_special;
        c->alpha = prm->alpha;
        c->beta_max = (c->L + c->alpha - 1) / c->alpha;
        if (prm->primes) {
            c->primes.assign(prm->primes, prm->primes + c->L + c->k);
            for (u64 q : c->primes) {
                NEED(q % (2ull * c->n) == 1 && bitlen(q) <= 60 && bitlen(q) >= 20, PFT_ERR_ARG,
                     "explicit primes must be 20..60 bits and 1 mod 2N");
            }
        } else {
            std::vector<u64> q0 = gen_primes(c->logn, prm->first_bits, 1, {});
            std::vector<u64> mids = gen_primes(c->logn, prm->mid_bits, c->L - 1, q0);
            std::vector<u64> used = q0;
            used.insert(used.end(), mids.begin(), mids.end());
            std::vector<u64> sp = gen_primes(c->logn, prm->special_bits, c->k, used);
            c->primes = used;
            c->primes.insert(c->primes.end(), sp.begin(), sp.end());
        }
        double logqp = 0;
        for (u64 q : c->primes) logqp += std::log2((double)q);
        if (!(prm->flags & PFT_ALLOW_INSECURE)) {
            NEED(c->logn >= 10 && logqp <= kSecureLogQP[c->logn], PFT_ERR_SECURITY,
                 "log2(QP) = " + std::to_string(logqp) + " is above the 128-bit bound for this N");
        }
        int tail = 0;
        c->cdt = gauss_cdt(prm->sigma > 0 ? prm->sigma : 3.2, &tail);
        if (alloc && alloc->alloc && alloc->free) {
            c->alloc = *alloc;
            c->has_alloc = true;
        }
        PFT_CUDA(cudaGetDevice(&c->device));
        build_tables(c.get());
        c->noalloc_scratch = noalloc_scratch_lookup();
    });
    if (rc != PFT_OK) {
        for (void* p : c->owned) cudaFree(p);
        return rc;
    }
    *out = c.release();
    return PFT_OK;
}

int pft_ctx_destroy(pft_ctx* c) {
    if (!c) return PFT_OK;
    cudaStreamSynchronize(c->stream);
    free_keys(c);
    dfree(c, c->s_ntt);
    dfree(c, c->pk);
    cudaStreamSynchronize(c->stream);
    for (void* p : c->owned) cudaFree(p);
    delete c;
    return PFT_OK;
}

int pft_set_stream(pft_ctx* c, void* stream) {
    if (!c) return PFT_ERR_ARG;
    c->stream = (cudaStream_t)stream;
    return PFT_OK;
}

const char* pft_last_error(pft_ctx* c) { return c ? c->err.c_str() : "null context"; }

int pft_ctx_info(pft_ctx* c, int* n, int* n_limbs, int* n_special, int* alpha, uint64_t* primes_out) {
    if (!c) return PFT_ERR_ARG;
    if (n) *n = c->n;
    if (n_limbs) *n_limbs = c->L;
    if (n_special) *n_special = c->k;
    if (alpha) *alpha = c->alpha;
    if (primes_out) std::copy(c->primes.begin(), c->primes.end(), primes_out);
    return PFT_OK;
}

int pft_keygen(pft_ctx* c, const int32_t* rot_steps, int n_steps, int want_relin) {
    return guard(c, [&] {
        NEED(c, PFT_ERR_ARG, "null context");
        const int n = c->n, L = c->L, R = L + c->k;
        const size_t limb = n;
        // s (ternary, the same integer polynomial in every prime of the full basis)
        c->s_coeff.assign(n, 0);
        if (!c->s_ntt) c->s_ntt = (u64*)dalloc(c, (size_t)R * limb * 8);
        {
            Scratch tmp(c, limb * 8);
            sample_small(c->tabs, c->prm.seed, DOM_SECRET, 0, 0, 0, c->cdt.data(), (int)c->cdt.size(), (i64*)tmp.p,
                         c->stream);
            std::vector<PolyRef> rs{ref(c->s_ntt, R, 0, L, L)};
            reduce_signed(c->tabs, (i64*)tmp.p, mkset(rs, 0, 1), c->stream);
            PFT_CUDA(cudaMemcpyAsync(c->s_coeff.data(), tmp.p, limb * 8, cudaMemcpyDeviceToHost, c->stream));
            PFT_CUDA(cudaStreamSynchronize(c->stream));
            ntt_fwd(c, rs, rs);
        }
        // pk = (b, a): a uniform, b = -a s + e
        if (!c->pk) c->pk = (u64*)dalloc(c, 2 * (size_t)L * limb * 8);
        {
            std::vector<PolyRef> rb{ref(c->pk, L)}, ra{ref(c->pk + (size_t)L * limb, L)}, rs{ref(c->s_ntt, L)};
            sample_uniform(c->tabs, c->prm.seed, DOM_PK_A, 0, 0, mkset(ra, 0, 1), c->stream);
            ntt_fwd(c, ra, ra);
            sample_signed_ntt(c, DOM_PK_E, 0, 0, 1, rb);
            Scratch as(c, (size_t)L * limb * 8);
            std::vector<PolyRef> ras{ref(as.u(), L)};
            ew(c, EwOp::Mul, ra, rs, ras);
            ew(c, EwOp::Sub, rb, ras, rb);
        }
        c->have_sk = true;
        free_keys(c);
        if (want_relin) {
            Scratch s2(c, (size_t)R * limb * 8);
            std::vector<PolyRef> rs{ref(c->s_ntt, R, 0, L, L)}, r2{ref(s2.u(), R, 0, L, L)};
            ew(c, EwOp::Mul, rs, rs, r2);
            add_key(c, 0, make_switch_key(c, s2.u(), 0));
        }
        if (n_steps > 0) {
            NEED(rot_steps, PFT_ERR_ARG, "null rotation steps");
            add_rot_keys(c, rot_steps, n_steps);
        }
    });
}

int pft_add_rotation_keys(pft_ctx* c, const int32_t* rot_steps, int n_steps) {
    return guard(c, [&] {
        NEED(c && (rot_steps || n_steps == 0), PFT_ERR_ARG, "bad arguments");
        add_rot_keys(c, rot_steps, n_steps);
    });
}

int pft_key_export(pft_ctx* c, uint32_t key_id, uint64_t* out, size_t nw) {
    return guard(c, [&] {
        NEED(c && out, PFT_ERR_ARG, "bad arguments");
        NEED(c->keys.count(key_id), PFT_ERR_NO_KEY, "no such key");
        const int R = c->L + c->k;
        const size_t words = (size_t)c->beta_max * 2 * R * c->n;
        NEED(nw >= words, PFT_ERR_ARG, "output too small");
        Scratch t(c, words * 8);
        std::vector<PolyRef> in, o;
        for (int i = 0; i < 2 * c->beta_max; i++) {
            u64* src = c->keys[key_id] + (size_t)i * R * c->n;
            if (c->compressed_keys) {
                const int j = i / 2;
                if (i % 2 == 0) {
                    src = c->keys[key_id] + (size_t)j * R * c->n;
                } else {  // regenerate a_j (evaluation form) in the output slot, then transform it there
                    src = t.u() + (size_t)i * R * c->n;
                    std::vector<PolyRef> ra{ref(src, R, 0, c->L, c->L)};
                    sample_uniform(c->tabs, c->prm.seed, kDomKskAEval, key_id, 256u * j, mkset(ra, 0, 1), c->stream);
                }
            }
            in.push_back(ref(src, R, 0, c->L, c->L));
            o.push_back(ref(t.u() + (size_t)i * R * c->n, R, 0, c->L, c->L));
        }
        ntt_inv(c, in, o);
        PFT_CUDA(cudaMemcpyAsync(out, t.p, words * 8, cudaMemcpyDeviceToHost, c->stream));
        PFT_CUDA(cudaStreamSynchronize(c->stream));
    });
}

int pft_secret_export(pft_ctx* c, int64_t* out, size_t nw) {
    return guard(c, [&] {
        NEED(c && out && nw >= (size_t)c->n, PFT_ERR_ARG, "bad arguments");
        NEED(c->have_sk, PFT_ERR_NO_KEY, "keygen has not run");
        std::copy(c->s_coeff.begin(), c->s_coeff.end(), out);
    });
}

int pft_ct_create(pft_ctx* c, pft_ct** out) {
    if (!c || !out) return PFT_ERR_ARG;
    *out = new pft_ct();
    (*out)->ctx = c;
    return PFT_OK;
}
int pft_ct_destroy(pft_ct* ct) {
    if (!ct) return PFT_OK;
    if (!handle_live(ct)) return PFT_ERR_ARG;  // destroyed already, or never a handle
    dfree(ct->ctx, ct->data);
    delete ct;
    return PFT_OK;
}
int pft_pt_destroy(pft_pt* pt) {
    if (!pt) return PFT_OK;
    if (!handle_live(pt)) return PFT_ERR_ARG;
    dfree(pt->ctx, pt->data);
    delete pt;
    return PFT_OK;
}
int pft_ct_level(const pft_ct* ct, int* level) {
    if (!ct || !level || !handle_live(ct)) return PFT_ERR_ARG;
    *level = ct->level;
    return PFT_OK;
}
int pft_ct_scale(const pft_ct* ct, double* scale) {
    if (!ct || !scale || !handle_live(ct)) return PFT_ERR_ARG;
    *scale = ct->scale;
    return PFT_OK;
}
int pft_pt_level(const pft_pt* pt, int* level) {
    if (!pt || !level || !handle_live(pt)) return PFT_ERR_ARG;
    *level = pt->level;
    return PFT_OK;
}
int pft_ct_data(const pft_ct* ct, uint64_t** p) {
    if (!ct || !p || !handle_live(ct)) return PFT_ERR_ARG;
    *p = ct->data;
    return PFT_OK;
}

int pft_ct_copy_out(pft_ctx* c, const pft_ct* ct, uint64_t* dst) {
    return guard(c, [&] {
        NEED(c && dst, PFT_ERR_ARG, "null argument");
        check_ct(c, ct);
        PFT_CUDA(cudaMemcpyAsync(dst, ct->data, (size_t)2 * ct->level * c->n * 8, cudaMemcpyDeviceToDevice,
                                 c->stream));
    });
}

int pft_ct_reduce_sum(pft_ctx* c, const uint64_t* words, int level, double scale, int n_terms, pft_ct* out) {
    return guard(c, [&] {
        NEED(c && words, PFT_ERR_ARG, "null argument");
        NEED(level >= 1 && level <= c->L, PFT_ERR_ARG, "level must be in 1..L");
        NEED(n_terms >= 1, PFT_ERR_ARG, "n_terms must be positive");
        u64 qmax = 0;
        for (int r = 0; r < level; r++) qmax = std::max(qmax, c->primes[r]);
        NEED((unsigned __int128)n_terms * (qmax - 1) < ((unsigned __int128)1 << 64), PFT_ERR_ARG,
             "n_terms canonical residues can exceed 64 bits: exchange by gathering instead");
        ensure_ct(c, out, level);
        out->scale = scale;
        std::vector<PolyRef> in, o;
        for (int pol = 0; pol < 2; pol++) {
            in.push_back(ref((u64*)words + (size_t)pol * level * c->n, level));
            o.push_back(ref(out->data + (size_t)pol * level * c->n, level));
        }
        reduce_words(c->tabs, mkset(in, 0, 2), mkset(o, 0, 2), c->stream);
    });
}

static pft_pt* new_pt(pft_ctx* c) {
    pft_pt* p = new pft_pt();
    p->ctx = c;
    return p;
}

int pft_pt_import(pft_ctx* c, const uint64_t* coeffs, int level, double scale, pft_pt** out) {
    return guard(c, [&] {
        NEED(c && coeffs && out && level >= 1 && level <= c->L, PFT_ERR_ARG, "bad arguments");
        std::unique_ptr<pft_pt> p(new_pt(c));
        ensure_pt(c, p.get(), level);
        p->scale = scale;
        PFT_CUDA(cudaMemcpyAsync(p->data, coeffs, (size_t)level * c->n * 8, cudaMemcpyHostToDevice, c->stream));
        std::vector<PolyRef> r{ref(p->data, level)};
        ntt_fwd(c, r, r);
        *out = p.release();
    });
}

int pft_pt_export(pft_ctx* c, const pft_pt* pt, uint64_t* coeffs, size_t nw) {
    return guard(c, [&] {
        check_pt(c, pt);
        NEED(c && coeffs && nw >= (size_t)pt->level * c->n, PFT_ERR_ARG, "bad arguments");
        Scratch t(c, (size_t)pt->level * c->n * 8);
        std::vector<PolyRef> in{ref(pt->data, pt->level)}, o{ref(t.u(), pt->level)};
        ntt_inv(c, in, o);
        PFT_CUDA(cudaMemcpyAsync(coeffs, t.p, (size_t)pt->level * c->n * 8, cudaMemcpyDeviceToHost, c->stream));
        PFT_CUDA(cudaStreamSynchronize(c->stream));
    });
}

int pft_ct_import(pft_ctx* c, const uint64_t* coeffs, int level, double scale, pft_ct** out) {
    return guard(c, [&] {
        NEED(c && coeffs && out && level >= 1 && level <= c->L, PFT_ERR_ARG, "bad arguments");
        std::unique_ptr<pft_ct> ct(new pft_ct());
        ct->ctx = c;
        ensure_ct(c, ct.get(), level);
        ct->scale = scale;
        PFT_CUDA(cudaMemcpyAsync(ct->data, coeffs, (size_t)2 * level * c->n * 8, cudaMemcpyHostToDevice, c->stream));
        std::vector<PolyRef> r{cpoly(ct->data, level, c->n, 0), cpoly(ct->data, level, c->n, 1)};
        ntt_fwd(c, r, r);
        *out = ct.release();
    });
}

int pft_ct_export(pft_ctx* c, const pft_ct* ct, uint64_t* coeffs, size_t nw) {
    return guard(c, [&] {
        check_ct(c, ct);
        const size_t words = (size_t)2 * ct->level * c->n;
        NEED(c && coeffs && nw >= words, PFT_ERR_ARG, "bad arguments");
        Scratch t(c, words * 8);
        std::vector<PolyRef> in{cpoly(ct->data, ct->level, c->n, 0), cpoly(ct->data, ct->level, c->n, 1)};
        std::vector<PolyRef> o{cpoly(t.u(), ct->level, c->n, 0), cpoly(t.u(), ct->level, c->n, 1)};
        ntt_inv(c, in, o);
        PFT_CUDA(cudaMemcpyAsync(coeffs, t.p, words * 8, cudaMemcpyDeviceToHost, c->stream));
        PFT_CUDA(cudaStreamSynchronize(c->stream));
    });
}

int pft_ct_import_batch(pft_ctx* c, const uint64_t* const* coeffs, const int* levels, const double* scales, int B,
                        pft_ct** out) {
    return guard(c, [&] {
        NEED(c && coeffs && levels && scales && out && B >= 0, PFT_ERR_ARG, "bad arguments");
        std::vector<std::unique_ptr<pft_ct>> cts;
        std::vector<PolyRef> r;
        for (int i = 0; i < B; i++) {
            NEED(coeffs[i] && levels[i] >= 1 && levels[i] <= c->L, PFT_ERR_ARG, "bad ciphertext " + std::to_string(i));
            cts.emplace_back(new pft_ct());
            pft_ct* ct = cts.back().get();
            ct->ctx = c;
            ensure_ct(c, ct, levels[i]);
            ct->scale = scales[i];
            PFT_CUDA(cudaMemcpyAsync(ct->data, coeffs[i], (size_t)2 * levels[i] * c->n * 8, cudaMemcpyHostToDevice,
                                     c->stream));
            r.push_back(cpoly(ct->data, levels[i], c->n, 0));
            r.push_back(cpoly(ct->data, levels[i], c->n, 1));
        }
        ntt_fwd(c, r, r);
        for (int i = 0; i < B; i++) out[i] = cts[i].release();
    });
}

int pft_ct_import_batch_into(pft_ctx* c, const uint64_t* const* coeffs, const int* levels, const double* scales,
                             int B, pft_ct* const* cts) {
    return guard(c, [&] {
        NEED(c && coeffs && levels && scales && cts && B >= 0, PFT_ERR_ARG, "bad arguments");
        for (int i = 0; i < B; i++) {
            NEED(coeffs[i] && cts[i] && levels[i] >= 1 && levels[i] <= c->L, PFT_ERR_ARG,
                 "bad ciphertext " + std::to_string(i));
            NEED(!cts[i]->ctx || cts[i]->ctx == c, PFT_ERR_ARG, "handle from another context");
            for (int j = 0; j < i; j++) NEED(cts[j] != cts[i], PFT_ERR_ARG, "a handle appears twice");
        }
        std::vector<PolyRef> r;
        for (int i = 0; i < B; i++) {
            pft_ct* ct = cts[i];
            ct->ctx = c;
            ensure_ct(c, ct, levels[i]);
            ct->scale = scales[i];
            PFT_CUDA(cudaMemcpyAsync(ct->data, coeffs[i], (size_t)2 * levels[i] * c->n * 8, cudaMemcpyHostToDevice,
                                     c->stream));
            r.push_back(cpoly(ct->data, levels[i], c->n, 0));
            r.push_back(cpoly(ct->data, levels[i], c->n, 1));
        }
        ntt_fwd(c, r, r);
    });
}

static void export_batch(pft_ctx* c, const pft_ct* const* cts, int B, uint64_t* const* coeffs, bool sync);

int pft_ct_export_batch(pft_ctx* c, const pft_ct* const* cts, int B, uint64_t* const* coeffs) {
    return guard(c, [&] { export_batch(c, cts, B, coeffs, true); });
}

int pft_ct_export_batch_async(pft_ctx* c, const pft_ct* const* cts, int B, uint64_t* const* coeffs) {
    return guard(c, [&] { export_batch(c, cts, B, coeffs, false); });
}

static void export_batch(pft_ctx* c, const pft_ct* const* cts, int B, uint64_t* const* coeffs, bool sync) {
    {
        NEED(c && cts && coeffs && B >= 0, PFT_ERR_ARG, "bad arguments");
        size_t maxw = 0;
        for (int i = 0; i < B; i++) {
            check_ct(c, cts[i]);
            NEED(coeffs[i], PFT_ERR_ARG, "null output buffer");
            maxw = std::max(maxw, (size_t)2 * cts[i]->level * c->n);
        }
        if (B == 0) return;
        // groups of ciphertexts through one staging buffer of at most 256 MiB (or one
        // ciphertext), reused in stream order: transform, copy out, next group
        const size_t cap = std::max(maxw, ((size_t)256 << 20) / 8);
        Scratch t(c, cap * 8);
        int i0 = 0;
        while (i0 < B) {
            int i1 = i0;
            size_t used = 0;
            std::vector<size_t> off;
            std::vector<PolyRef> in, o;
            while (i1 < B && used + (size_t)2 * cts[i1]->level * c->n <= cap) {
                const int l = cts[i1]->level;
                off.push_back(used);
                for (int pol = 0; pol < 2; pol++) {
                    in.push_back(cpoly(cts[i1]->data, l, c->n, pol));
                    o.push_back(cpoly(t.u() + used, l, c->n, pol));
                }
                used += (size_t)2 * l * c->n;
                i1++;
            }
            ntt_inv(c, in, o);
            for (int i = i0; i < i1; i++)
                PFT_CUDA(cudaMemcpyAsync(coeffs[i], t.u() + off[i - i0], (size_t)2 * cts[i]->level * c->n * 8,
                                         cudaMemcpyDeviceToHost, c->stream));
            i0 = i1;
        }
        if (sync) {
            PFT_CUDA(cudaStreamSynchronize(c->stream));
            NEED(!wait_timeout_flag(true, c->stream), PFT_ERR_TIMEOUT, "a bounded device wait expired; results are invalid");
        }
    }
}

int pft_encode(pft_ctx* c, const double* re_im, int n_slots, double scale, int level, pft_pt** out) {
    return guard(c, [&] {
        NEED(c && out && (re_im || n_slots == 0), PFT_ERR_ARG, "bad arguments");
        NEED(n_slots >= 0 && n_slots <= c->n / 2, PFT_ERR_ARG, "too many slots");
        NEED(level >= 1 && level <= c->L, PFT_ERR_ARG, "bad level");
        std::vector<i64> coeffs;
        NEED(encode_slots(c->logn, re_im, n_slots, scale, coeffs), PFT_ERR_ARG, "encoded coefficient exceeds 2^62");
        std::unique_ptr<pft_pt> p(new_pt(c));
        ensure_pt(c, p.get(), level);
        p->scale = scale;
        Scratch t(c, (size_t)c->n * 8);
        PFT_CUDA(cudaMemcpyAsync(t.p, coeffs.data(), (size_t)c->n * 8, cudaMemcpyHostToDevice, c->stream));
        std::vector<PolyRef> r{ref(p->data, level)};
        reduce_signed(c->tabs, (i64*)t.p, mkset(r, 0, 1), c->stream);
        ntt_fwd(c, r, r);
        *out = p.release();
    });
}

int pft_decode(pft_ctx* c, const pft_pt* pt, double* re_im, int n_slots) {
    return guard(c, [&] {
        check_pt(c, pt);
        NEED(c && re_im && n_slots >= 0 && n_slots <= c->n / 2, PFT_ERR_ARG, "bad arguments");
        const int l = pt->level;
        std::vector<u64> rows((size_t)l * c->n);
        Scratch t(c, rows.size() * 8);
        std::vector<PolyRef> in{ref(pt->data, l)}, o{ref(t.u(), l)};
        ntt_inv(c, in, o);
        PFT_CUDA(cudaMemcpyAsync(rows.data(), t.p, rows.size() * 8, cudaMemcpyDeviceToHost, c->stream));
        PFT_CUDA(cudaStreamSynchronize(c->stream));
        std::vector<u64> ps(c->primes.begin(), c->primes.begin() + l);
        std::vector<double> coeffs;
        crt_to_double(ps, rows.data(), c->n, coeffs);
        decode_coeffs(c->logn, coeffs, pt->scale, re_im, n_slots);
    });
}

int pft_encrypt(pft_ctx* c, const pft_pt* pt, int mode, uint32_t nonce, pft_ct** out) {
    return guard(c, [&] {
        NEED(c && out && (mode == PFT_ENC_PK || mode == PFT_ENC_SK), PFT_ERR_ARG, "bad arguments");
        std::unique_ptr<pft_ct> ct(new pft_ct());
        ct->ctx = c;
        encrypt(c, pt, mode, nonce, ct.get());
        *out = ct.release();
    });
}

int pft_decrypt(pft_ctx* c, const pft_ct* ct, pft_pt** out) {
    return guard(c, [&] {
        check_ct(c, ct);
        NEED(c && out, PFT_ERR_ARG, "bad arguments");
        NEED(c->have_sk, PFT_ERR_NO_KEY, "keygen has not run");
        const int l = ct->level;
        std::unique_ptr<pft_pt> p(new_pt(c));
        ensure_pt(c, p.get(), l);
        p->scale = ct->scale;
        std::vector<PolyRef> r0{cpoly(ct->data, l, c->n, 0)}, r1{cpoly(ct->data, l, c->n, 1)}, rs{ref(c->s_ntt, l)},
            rp{ref(p->data, l)};
        ew(c, EwOp::Mul, r1, rs, rp);
        ew(c, EwOp::Add, rp, r0, rp);
        *out = p.release();
    });
}

int pft_add(pft_ctx* c, const pft_ct* a, const pft_ct* b, pft_ct* out) {
    return guard(c, [&] { op_add_batch(c, &a, &b, 1, &out, EwOp::Add); });
}
int pft_sub(pft_ctx* c, const pft_ct* a, const pft_ct* b, pft_ct* out) {
    return guard(c, [&] { op_add_batch(c, &a, &b, 1, &out, EwOp::Sub); });
}
int pft_add_plain(pft_ctx* c, const pft_ct* a, const pft_pt* p, pft_ct* out) {
    return guard(c, [&] {
        check_ct(c, a);
        check_pt(c, p);
        NEED(out, PFT_ERR_ARG, "null output");
        NEED(a->level == p->level, PFT_ERR_LEVEL_MISMATCH, "HADDPLAIN operands at different levels");
        NEED(a->scale == p->scale, PFT_ERR_SCALE_MISMATCH, "HADDPLAIN operands at different scales");
        const int l = a->level;
        const double sc = a->scale;
        const u64* src1 = a->data + (size_t)l * c->n;
        ensure_ct(c, out, l);
        out->scale = sc;
        std::vector<PolyRef> r0{cpoly(a->data, l, c->n, 0)}, rp{ref(p->data, l)}, o0{cpoly(out->data, l, c->n, 0)};
        ew(c, EwOp::Add, r0, rp, o0);
        if (out != a) {
            std::vector<PolyRef> r1{ref((u64*)src1, l)}, o1{cpoly(out->data, l, c->n, 1)};
            ew(c, EwOp::Copy, r1, {}, o1);
        }
    });
}
int pft_mul_plain(pft_ctx* c, const pft_ct* a, const pft_pt* p, pft_ct* out) {
    return guard(c, [&] { op_mul_plain_batch(c, &a, &p, 1, &out); });
}
int pft_mul_relin(pft_ctx* c, const pft_ct* a, const pft_ct* b, pft_ct* out) {
    return guard(c, [&] { op_mul_relin_batch(c, &a, &b, 1, &out); });
}
int pft_rescale(pft_ctx* c, const pft_ct* a, pft_ct* out) {
    return guard(c, [&] { op_rescale_batch(c, &a, 1, &out); });
}
int pft_rotate(pft_ctx* c, const pft_ct* a, int32_t step, pft_ct* out) {
    return guard(c, [&] { op_rotate_batch(c, &a, 1, step, &out); });
}
int pft_drop_level(pft_ctx* c, const pft_ct* a, int level, pft_ct* out) {
    return guard(c, [&] { op_drop_level_batch(c, &a, 1, level, &out); });
}
int pft_add_const(pft_ctx* c, const pft_ct* a, double value, pft_ct* out) {
    return guard(c, [&] { op_const_batch(c, &a, 1, value, 0.0, false, &out); });
}
int pft_mul_const(pft_ctx* c, const pft_ct* a, double value, double const_scale, pft_ct* out) {
    return guard(c, [&] { op_const_batch(c, &a, 1, value, const_scale, true, &out); });
}
int pft_device_status(pft_ctx* c) {
    return guard(c, [&] {
        NEED(c, PFT_ERR_ARG, "bad arguments");
        PFT_CUDA(cudaStreamSynchronize(c->stream));
        NEED(!wait_timeout_flag(true, c->stream), PFT_ERR_TIMEOUT, "a bounded device wait expired");
    });
}

int pft_bfly_ceiling(pft_ctx* c, double* out) {
    return guard(c, [&] {
        NEED(c && out, PFT_ERR_ARG, "bad arguments");
        *out = bfly_ceiling(c->tabs, c->stream);
    });
}

int pft_mul_rates(pft_ctx* c, double* lo, double* hi, double* wide) {
    return guard(c, [&] {
        NEED(c, PFT_ERR_ARG, "null context");
        mul_rates(c->stream, lo, hi, wide);
    });
}
int pft_wait_selftest(pft_ctx* c, long long polls) {
    return guard(c, [&] {
        NEED(c && polls >= 1 && polls <= (1ll << 20), PFT_ERR_ARG, "polls must lie in 1..2^20");
        wait_selftest(polls, c->stream);
    });
}

int pft_ct_set_scale(pft_ct* ct, double scale) {
    if (!ct || !(scale > 0) || !std::isfinite(scale)) return PFT_ERR_ARG;
    ct->scale = scale;
    return PFT_OK;
}
int pft_dot_plain_batch(pft_ctx* c, const pft_ct* const* cts, const pft_pt* const* pts, int K, int n_out,
                        int pts_shared, pft_ct* const* outs) {
    return guard(c, [&] {
        NEED(c && cts && pts && outs && K >= 1 && n_out >= 0, PFT_ERR_ARG, "bad arguments");
        if (n_out == 0) return;
        const int l = cts[0]->level;
        const size_t limb = c->n;
        std::vector<const u64*> A, Bv;
        std::vector<u64*> O;
        for (int k = 0; k < (pts_shared ? K : K * n_out); k++) {
            check_pt(c, pts[k]);
            NEED(pts[k]->level == l, PFT_ERR_LEVEL_MISMATCH, "plaintexts must sit at the ciphertexts' level");
        }
        std::vector<double> sc(n_out);
        for (int o = 0; o < n_out; o++) {
            for (int k = 0; k < K; k++) {
                const pft_ct* x = cts[(size_t)o * K + k];
                check_ct(c, x);
                NEED(x->level == l, PFT_ERR_LEVEL_MISMATCH, "all ciphertexts must share one level");
                const double s = x->scale * pts[pts_shared ? k : (size_t)o * K + k]->scale;
                if (k == 0) sc[o] = s;
                NEED(s == sc[o], PFT_ERR_SCALE_MISMATCH, "products of one output must share one scale");
            }
            NEED(outs[o], PFT_ERR_ARG, "null output");
            for (int k = 0; k < K; k++) NEED(outs[o] != cts[(size_t)o * K + k], PFT_ERR_ARG, "output aliases an input");
        }
        for (int o = 0; o < n_out; o++) {
            ensure_ct(c, outs[o], l);
            outs[o]->scale = sc[o];
        }
        if (pts_shared)
            for (int k = 0; k < K; k++) Bv.push_back(pts[k]->data);
        for (int o = 0; o < n_out; o++)
            for (int pol = 0; pol < 2; pol++) {
                for (int k = 0; k < K; k++) {
                    A.push_back(cts[(size_t)o * K + k]->data + (size_t)pol * l * limb);
                    if (!pts_shared) Bv.push_back(pts[(size_t)o * K + k]->data);
                }
                O.push_back(outs[o]->data + (size_t)pol * l * limb);
            }
        Scratch dA(c, A.size() * 8), dB(c, Bv.size() * 8), dO(c, O.size() * 8);
        ew_dot(c->tabs, upload(c, dA, A), upload(c, dB, Bv), upload(c, dO, O), (int)O.size(), K, pts_shared != 0, l,
               c->stream);
    });
}

int pft_rotate_hoisted(pft_ctx* c, const pft_ct* a, const int32_t* steps, int n, pft_ct* const* outs) {
    return guard(c, [&] { op_rotate_hoisted(c, a, steps, n, outs); });
}
int pft_add_batch(pft_ctx* c, const pft_ct* const* a, const pft_ct* const* b, int B, pft_ct* const* out) {
    return guard(c, [&] {
        NEED(c && a && b && out && B >= 0, PFT_ERR_ARG, "bad arguments");
        op_add_batch(c, a, b, B, out, EwOp::Add);
    });
}
int pft_mul_plain_batch(pft_ctx* c, const pft_ct* const* a, const pft_pt* const* p, int B, pft_ct* const* out) {
    return guard(c, [&] {
        NEED(c && a && p && out && B >= 0, PFT_ERR_ARG, "bad arguments");
        op_mul_plain_batch(c, a, p, B, out);
    });
}
int pft_mul_relin_batch(pft_ctx* c, const pft_ct* const* a, const pft_ct* const* b, int B, pft_ct* const* out) {
    return guard(c, [&] {
        NEED(c && a && b && out && B >= 0, PFT_ERR_ARG, "bad arguments");
        op_mul_relin_batch(c, a, b, B, out);
    });
}
int pft_rescale_batch(pft_ctx* c, const pft_ct* const* a, int B, pft_ct* const* out) {
    return guard(c, [&] {
        NEED(c && a && out && B >= 0, PFT_ERR_ARG, "bad arguments");
        op_rescale_batch(c, a, B, out);
    });
}
int pft_rotate_batch(pft_ctx* c, const pft_ct* const* a, int B, int32_t step, pft_ct* const* out) {
    return guard(c, [&] {
        NEED(c && a && out && B >= 0, PFT_ERR_ARG, "bad arguments");
        op_rotate_batch(c, a, B, step, out);
    });
}

// The autotuner: for each launch-size bucket (by the launch's total limbs: <= 64, <= 512, larger)
// it times every transform plan of the ring (ntt_candidates: the specialised kernels and generic
// staged passes of several stage splits and tile widths) on a forward + inverse transform of a
// representative launch (32, 256 and 1024 limbs of the chain's primes), median of 3, and keeps
// the fastest plan for that bucket.
int pft_autotune(pft_ctx* c, double* us_out, int cap, int* chosen) {
    return guard(c, [&] {
        NEED(c, PFT_ERR_ARG, "null context");
        constexpr int kMaxCand = 16;
        DevTables::Plan cand[kMaxCand];
        const char* names[kMaxCand];
        const int nc = ntt_candidates(c->logn, cand, names, kMaxCand);
        std::string js = "{\"N\": " + std::to_string(c->n) + ", \"buckets\": [";
        int best_last = 0;
        std::vector<double> us_last(std::max(nc, 1), 0.0);
        if (nc > 1) {
            const int reps_limbs[kNttBuckets] = {32, 256, 1024};
            const int limbs = std::min(c->L + c->k, 32);
            cudaEvent_t e0, e1;
            PFT_CUDA(cudaEventCreate(&e0));
            PFT_CUDA(cudaEventCreate(&e1));
            for (int b = 0; b < kNttBuckets; b++) {
                const int polys = std::max(1, reps_limbs[b] / limbs);
                Scratch buf(c, (size_t)polys * limbs * c->n * 8);
                PFT_CUDA(cudaMemsetAsync(buf.p, 0, (size_t)polys * limbs * c->n * 8, c->stream));
                std::vector<PolyRef> r;
                for (int i = 0; i < polys; i++) r.push_back(ref(buf.u() + (size_t)i * limbs * c->n, limbs));
                std::vector<double> us(nc, 0.0);
                for (int v = 0; v < nc; v++) {
                    c->tabs.plan[b] = cand[v];
                    ntt_fwd(c, r, r);  // warm-up (and one-time kernel attributes)
                    ntt_inv(c, r, r);
                    double t3[3];
                    for (int rep = 0; rep < 3; rep++) {
                        PFT_CUDA(cudaEventRecord(e0, c->stream));
                        ntt_fwd(c, r, r);
                        ntt_inv(c, r, r);
                        PFT_CUDA(cudaEventRecord(e1, c->stream));
                        PFT_CUDA(cudaEventSynchronize(e1));
                        float ms = 0;
                        PFT_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                        t3[rep] = 1e3 * ms;
                    }
                    std::sort(t3, t3 + 3);
                    us[v] = t3[1];
                }
                int best = 0;
                for (int v = 1; v < nc; v++)
                    if (us[v] < us[best]) best = v;
                c->tabs.plan[b] = cand[best];
                char head[160];
                snprintf(head, sizeof(head), "%s{\"limbs\": %d, \"chosen\": \"%s\", \"us_fwd_inv\": {", b ? ", " : "",
                         polys * limbs, names[best]);
                js += head;
                for (int v = 0; v < nc; v++) {
                    char item[160];
                    snprintf(item, sizeof(item), "%s\"%s\": %.1f", v ? ", " : "", names[v], us[v]);
                    js += item;
                }
                js += "}}";
                if (b == kNttBuckets - 1) {
                    best_last = best;
                    us_last = us;
                }
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
        }
        js += "]}";
        c->autotune_report = js;
        if (chosen) *chosen = best_last;
        if (us_out)
            for (int v = 0; v < nc && v < cap; v++) us_out[v] = us_last[v];
    });
}

int pft_autotune_report(pft_ctx* c, char* buf, size_t cap, size_t* len) {
    return guard(c, [&] {
        NEED(c, PFT_ERR_ARG, "null context");
        if (len) *len = c->autotune_report.size();
        if (buf && cap) {
            const size_t k = std::min(cap - 1, c->autotune_report.size());
            memcpy(buf, c->autotune_report.data(), k);
            buf[k] = 0;
        }
    });
}

int pft_set_transform_plan(pft_ctx* c, int plan) {
    return guard(c, [&] {
        NEED(c, PFT_ERR_ARG, "null context");
        DevTables::Plan cand[16];
        const int nc = ntt_candidates(c->logn, cand, nullptr, 16);
        NEED(plan >= -1 && plan < nc, PFT_ERR_ARG, "plan out of range");
        if (plan < 0) default_plans(c->tabs);
        else
            for (int b = 0; b < kNttBuckets; b++) c->tabs.plan[b] = cand[plan];
    });
}

int pft_set_transform_variant(pft_ctx* c, int variant) {
    return guard(c, [&] {
        NEED(c && variant >= 0 && variant < kNttVariants, PFT_ERR_ARG, "variant out of range");
        c->tabs.ntt_variant = variant;
        for (int b = 0; b < kNttBuckets; b++) c->tabs.plan[b].kind = -1;  // the fixed variant everywhere
    });
}

int pft_graph_begin(pft_ctx* c) {
    return guard(c, [&] {
        NEED(c, PFT_ERR_ARG, "null context");
        NEED(c->stream != nullptr, PFT_ERR_ARG, "graph capture needs a non-default context stream");
        NEED(!c->has_alloc, PFT_ERR_ARG, "graph capture needs the stream-ordered default allocator");
        PFT_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    });
}

int pft_graph_end(pft_ctx* c, pft_graph** out) {
    return guard(c, [&] {
        NEED(c && out, PFT_ERR_ARG, "bad arguments");
        std::unique_ptr<pft_graph> g(new pft_graph());
        PFT_CUDA(cudaStreamEndCapture(c->stream, &g->graph));
        PFT_CUDA(cudaGraphInstantiate(&g->exec, g->graph, 0));
        *out = g.release();
    });
}

int pft_graph_launch(pft_ctx* c, const pft_graph* g) {
    return guard(c, [&] {
        NEED(c && g && g->exec, PFT_ERR_ARG, "bad arguments");
        PFT_CUDA(cudaGraphLaunch(g->exec, c->stream));
    });
}

int pft_graph_destroy(pft_graph* g) {
    if (!g) return PFT_OK;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
    return PFT_OK;
}

int pft_rescale_noalloc(pft_ctx* c, const uint64_t* in, int level, uint64_t* out) {
    return guard(c, [&] {
        NEED(c && in && out, PFT_ERR_ARG, "null argument");
        NEED(level >= 2 && level <= c->L, PFT_ERR_ARG, "level must be in 2..L");
        const size_t n = (size_t)c->n, l = (size_t)level;
        const size_t need = 2 * n + 2 * (l - 1) * n;
        NEED(need <= kNoAllocScratchWords, PFT_ERR_ARG,
             "rescale_noalloc: 2 N level = " + std::to_string(2 * n * l) + " words exceed the fixed scratch of " +
                 std::to_string(kNoAllocScratchWords) + " words");
        const u64* in_end = in + 2 * l * n;
        const u64* out_end = out + 2 * (l - 1) * n;
        NEED(out_end <= in || in_end <= out, PFT_ERR_ARG, "rescale_noalloc: output overlaps input");
        int dev = -1;
        PFT_CUDA(cudaGetDevice(&dev));
        NEED(dev == c->device, PFT_ERR_ARG,
             "rescale_noalloc: the current device (" + std::to_string(dev) + ") is not the context's device (" +
                 std::to_string(c->device) + ")");
        u64* last = c->noalloc_scratch;
        u64* rb = last + 2 * n;
        u64* src = (u64*)in;
        std::vector<PolyRef> lin, lout, rr, x, o;
        for (int pol = 0; pol < 2; pol++) {
            lin.push_back(ref(src + ((size_t)pol * l + l - 1) * n, 1, level - 1));
            lout.push_back(ref(last + (size_t)pol * n, 1, level - 1));
            rr.push_back(ref(rb + (size_t)pol * (l - 1) * n, level - 1));
            x.push_back(ref(src + (size_t)pol * l * n, level - 1));
            o.push_back(ref(out + (size_t)pol * (l - 1) * n, level - 1));
        }
        ntt_inv(c, lin, lout);
        rescale_bcast(c->tabs, mkset(lout, 0, 2), mkset(rr, 0, 2), c->stream);
        ntt_fwd(c, rr, rr);
        subscale(c, x, &rr, nullptr, o, c->rescale_consts[level - 1]);
    });
}

int pft_ntt(pft_ctx* c, uint64_t* data, int n_polys, int n_limbs, int inverse) {
    return guard(c, [&] {
        NEED(c && data && n_polys >= 0 && n_limbs >= 1 && n_limbs <= c->L + c->k, PFT_ERR_ARG, "bad arguments");
        std::vector<PolyRef> r;
        for (int i = 0; i < n_polys; i++) r.push_back(ref(data + (size_t)i * n_limbs * c->n, n_limbs));
        if (inverse) ntt_inv(c, r, r);
        else ntt_fwd(c, r, r);
    });
}

int pft_ft_model_import(pft_ctx* c, const pft_pt* const* H_pts, const pft_pt* const* O_pts, int m, int n, int cl,
                        pft_ft_model** out) {
    return guard(c, [&] {
        NEED(c && H_pts && O_pts && out && m >= 1 && n >= 1 && cl >= 1 && cl <= c->n / 2, PFT_ERR_ARG,
             "bad arguments");
        const int t = c->n / 2, chunks_n = (m + t - 1) / t;
        std::unique_ptr<pft_ft_model> M(new pft_ft_model());
        M->ctx = c;
        M->m = m;
        M->n = n;
        M->c = cl;
        M->chunks = chunks_n;
        M->level = H_pts[0]->level;
        auto copy_pt = [&](const pft_pt* p) {
            check_pt(c, p);
            pft_pt* q = new_pt(c);
            ensure_pt(c, q, p->level);
            q->scale = p->scale;
            PFT_CUDA(cudaMemcpyAsync(q->data, p->data, (size_t)p->level * c->n * 8, cudaMemcpyDeviceToDevice, c->stream));
            return q;
        };
        for (int i = 0; i < n * chunks_n; i++) {
            NEED(H_pts[i]->level == M->level, PFT_ERR_LEVEL_MISMATCH, "embedding plaintexts at different levels");
            M->H.push_back(copy_pt(H_pts[i]));
        }
        for (int j = 0; j < n; j++) M->O.push_back(copy_pt(O_pts[j]));
        *out = M.release();
    });
}

int pft_ft_model_create(pft_ctx* c, const double* H, const double* O, int m, int n, int cl, int level,
                        pft_ft_model** out) {
    return guard(c, [&] {
        NEED(c && H && O && out && m >= 1 && n >= 1 && cl >= 1 && cl <= c->n / 2, PFT_ERR_ARG, "bad arguments");
        NEED(level >= 3 && level <= c->L, PFT_ERR_ARG, "model level must be in 3..L");
        const int t = c->n / 2, chunks_n = (m + t - 1) / t;
        std::vector<pft_pt*> hp, op;
        std::vector<double> slots(2 * (size_t)t);
        auto cleanup = [&] {
            for (auto p : hp) pft_pt_destroy(p);
            for (auto p : op) pft_pt_destroy(p);
        };
        int rc = PFT_OK;
        for (int j = 0; j < n && rc == PFT_OK; j++)
            for (int i = 0; i < chunks_n && rc == PFT_OK; i++) {
                std::fill(slots.begin(), slots.end(), 0.0);
                for (int u = 0; u < t && i * t + u < m; u++) slots[2 * u] = H[(size_t)(i * t + u) * n + j];
                pft_pt* p = nullptr;
                rc = pft_encode(c, slots.data(), t, c->prm.scale, level, &p);
                if (rc == PFT_OK) hp.push_back(p);
            }
        for (int j = 0; j < n && rc == PFT_OK; j++) {
            std::fill(slots.begin(), slots.end(), 0.0);
            for (int u = 0; u < cl; u++) slots[2 * u] = O[(size_t)j * cl + u];
            pft_pt* p = nullptr;
            rc = pft_encode(c, slots.data(), t, c->prm.scale, level - 1, &p);
            if (rc == PFT_OK) op.push_back(p);
        }
        if (rc != PFT_OK) {
            cleanup();
            fail(rc, c->err);
        }
        std::unique_ptr<pft_ft_model> M(new pft_ft_model());
        M->ctx = c;
        M->m = m;
        M->n = n;
        M->c = cl;
        M->chunks = chunks_n;
        M->level = level;
        M->H = hp;
        M->O = op;
        *out = M.release();
    });
}

int pft_ft_model_create_diag(pft_ctx* c, const double* H, const double* O, int m, int n, int cl, int level,
                             pft_ft_model** out) {
    return guard(c, [&] {
        const int t = c ? c->n / 2 : 0;
        NEED(c && H && O && out && m >= 1 && n >= 2 && cl >= 1, PFT_ERR_ARG, "bad arguments");
        NEED((n & (n - 1)) == 0 && t % n == 0 && (size_t)n * cl <= (size_t)t, PFT_ERR_ARG,
             "diagonal packing needs n a power of two dividing N/2 and n c <= N/2");
        NEED(level >= 3 && level <= c->L, PFT_ERR_ARG, "model level must be in 3..L");
        const int nch = (m + t - 1) / t;
        std::vector<pft_pt*> dp, op;
        auto cleanup = [&] {
            for (auto p : dp) pft_pt_destroy(p);
            for (auto p : op) pft_pt_destroy(p);
        };
        std::vector<double> slots(2 * (size_t)t);
        int rc = PFT_OK;
        // chunk ch, diagonal k: D_{ch,k}[i] = H[ch t + (i + k) mod t, i mod n] (zero rows >= m)
        for (int ch = 0; ch < nch && rc == PFT_OK; ch++)
            for (int k = 0; k < n && rc == PFT_OK; k++) {
                std::fill(slots.begin(), slots.end(), 0.0);
                for (int i = 0; i < t; i++) {
                    const size_t row = (size_t)ch * t + (i + k) % t;
                    if (row < (size_t)m) slots[2 * (size_t)i] = H[row * n + (i % n)];
                }
                pft_pt* p = nullptr;
                rc = pft_encode(c, slots.data(), t, c->prm.scale, level, &p);
                if (rc == PFT_OK) dp.push_back(p);
            }
        if (rc == PFT_OK) {  // P[n c + j] = O[j, c]
            std::fill(slots.begin(), slots.end(), 0.0);
            for (int cc = 0; cc < cl; cc++)
                for (int j = 0; j < n; j++) slots[2 * ((size_t)n * cc + j)] = O[(size_t)j * cl + cc];
            pft_pt* p = nullptr;
            rc = pft_encode(c, slots.data(), t, c->prm.scale, level - 1, &p);
            if (rc == PFT_OK) op.push_back(p);
        }
        if (rc != PFT_OK) {
            cleanup();
            fail(rc, c->err);
        }
        std::unique_ptr<pft_ft_model> M(new pft_ft_model());
        M->ctx = c;
        M->m = m;
        M->n = n;
        M->c = cl;
        M->chunks = nch;
        M->level = level;
        M->variant = 1;
        M->H = dp;
        M->O = op;
        *out = M.release();
    });
}

int pft_ft_model_import_diag(pft_ctx* c, const pft_pt* const* D_pts, const pft_pt* P_pt, int m, int n, int cl,
                             pft_ft_model** out) {
    return guard(c, [&] {
        const int t = c ? c->n / 2 : 0;
        NEED(c && D_pts && P_pt && out && m >= 1 && n >= 2 && cl >= 1, PFT_ERR_ARG, "bad arguments");
        NEED((n & (n - 1)) == 0 && t % n == 0 && (size_t)n * cl <= (size_t)t, PFT_ERR_ARG,
             "diagonal packing needs n a power of two dividing N/2 and n c <= N/2");
        const int nch = (m + t - 1) / t;
        std::unique_ptr<pft_ft_model> M(new pft_ft_model());
        M->ctx = c;
        M->m = m;
        M->n = n;
        M->c = cl;
        M->chunks = nch;
        M->level = D_pts[0]->level;
        M->variant = 1;
        auto copy_pt = [&](const pft_pt* p) {
            check_pt(c, p);
            pft_pt* q = new_pt(c);
            ensure_pt(c, q, p->level);
            q->scale = p->scale;
            PFT_CUDA(cudaMemcpyAsync(q->data, p->data, (size_t)p->level * c->n * 8, cudaMemcpyDeviceToDevice, c->stream));
            return q;
        };
        for (int k = 0; k < nch * n; k++) {
            check_pt(c, D_pts[k]);
            NEED(D_pts[k]->level == M->level, PFT_ERR_LEVEL_MISMATCH, "diagonal plaintexts at different levels");
            M->H.push_back(copy_pt(D_pts[k]));
        }
        NEED(P_pt->level == M->level - 1, PFT_ERR_LEVEL_MISMATCH, "output plaintext must sit one level below");
        M->O.push_back(copy_pt(P_pt));
        *out = M.release();
    });
}

int pft_ft_model_destroy(pft_ft_model* M) {
    if (!M) return PFT_OK;
    for (auto p : M->H) pft_pt_destroy(p);
    for (auto p : M->O) pft_pt_destroy(p);
    delete M;
    return PFT_OK;
}

int pft_fasttext_infer(pft_ctx* c, const pft_ft_model* M, const pft_ct* const* v, int n_chunks, pft_ct* scores) {
    return guard(c, [&] {
        NEED(c && v && scores, PFT_ERR_ARG, "bad arguments");
        fasttext_batch(c, M, v, n_chunks, 1, &scores);
    });
}

int pft_fasttext_infer_batch(pft_ctx* c, const pft_ft_model* M, const pft_ct* const* v, int n_chunks, int B,
                             pft_ct* const* scores) {
    return guard(c, [&] {
        NEED(c && v && scores && B >= 1, PFT_ERR_ARG, "bad arguments");
        fasttext_batch(c, M, v, n_chunks, B, scores);
    });
}


}  // extern "C"
