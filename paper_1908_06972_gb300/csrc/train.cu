// Encrypted minibatch training of fastText (Sec. 4.2, Algorithm 5) on one GPU.
//
// Layout (the inference packing of Fig. 3 with encrypted weights): H_j holds column j of H
// over the vocabulary slots (m <= t), O_j holds row j of O in slots 0..c-1, v_b is document
// b, and the client sends w_b = y_b - 1/4 on the c class slots: the constant term of the
// softmax polynomial is folded into the labels, so the server never needs a slot mask.
// Softmax is the paper's minimax polynomial P(s) = s^2/8 + s/2 + 1/4; the loss is the
// degree-3 polynomial sum_c [s^3/24 + s^2/4 + s/4 - y s] whose gradient in s is P(s) - y.
// Levels relative to the model level l0:
//   forward   h_bj = Rescale(TotalSum(Relin(v_b x H_j)))                 l0-1
//             s_b  = Rescale(Relin(sum_j h_bj x O_j))                    l0-2
//             U_b  = Rescale(Relin(u_b x u_b)), u_b = s_b + 2            l0-3
//             g_b  = U_b read at 8x its scale - 1/2 - w_b  = P(s_b) - y_b
//   backward  dO_j = Rescale(Relin(sum_b h_bj x g_b))                    l0-4
//             e_bj = Rescale(TotalSum(Relin(g_b x O_j)))                 l0-4
//             dH_j = Rescale(Relin(sum_b v_b x e_bj))                    l0-5
//   update    O_j <- O_j - eta dO_j (l0-5), H_j <- H_j - eta dH_j (l0-6); each product by
//             eta is taken at the constant scale that returns, after one rescale, the
//             model's own scale, so the model keeps its scales from step to step.
// Operands of a higher level enter products through their leading limbs; sums of tensor
// products are relinearised once.  Each stage is one batched call over every (document,
// column) pair of a tile of documents; tiles bound the working memory.
#include <algorithm>
#include <cmath>
#include <cstdlib>

#include "evaluator.h"

struct pft_ft_enc_model {
    pft_ctx* ctx = nullptr;
    int m = 0, n = 0, c = 0;
    int variant = 0;            // 0: Fig. 3 layout; 1: diagonal layout (rotation-light)
    int lift = 0;               // variant 1: the documents are multiplied by 2^lift before rotating
    std::vector<pft_ct> H, O;   // variant 1: H = the diagonals D_k, O = {P}
    pft_pt mask;                // variant 1: 1 in the score slots n c
    ~pft_ft_enc_model() {
        for (auto& x : H) dfree(ctx, x.data);
        for (auto& x : O) dfree(ctx, x.data);
        dfree(ctx, mask.data);
    }
};

struct pft_ft_tape {
    pft_ctx* ctx = nullptr;
    const pft_ft_enc_model* M = nullptr;
    int B = 0, l0 = 0;
    std::vector<const pft_ct*> v;  // the caller's documents (kept alive by the caller)
    std::vector<pft_ct> h;         // [B][n], level l0-1 (diagonal layout: [B], the replicated h_b)
    std::vector<pft_ct> s;         // [B], level l0-2 (the scores; diagonal layout: masked, l0-3)
    std::vector<pft_ct> g;         // [B], level l0-3 (diagonal layout: spread over blocks, l0-4)
    std::vector<pft_ct> r;         // diagonal layout: [B][n] lifted documents and their rotations, level l0
    ~pft_ft_tape() {
        for (auto* vec : {&h, &s, &g, &r})
            for (auto& x : *vec) dfree(ctx, x.data);
    }
};

namespace {

void free_cts(pft_ctx* c, std::vector<pft_ct>& v, size_t a, size_t b) {
    for (size_t i = a; i < b; i++) {
        dfree(c, v[i].data);
        v[i].data = nullptr;
        v[i].cap = 0;
    }
}

// polynomial base of a ciphertext operand (limb r of polynomial pol at + r N)
const u64* pbase(const pft_ct* x, int pol, int n) { return x->data + (size_t)pol * x->level * n; }

// outs[o] (+)= sum_k a_ok (x) b_ok at level l, K terms for every output, operands at level >= l.
void tensor_dot(pft_ctx* c, const std::vector<std::vector<std::pair<const pft_ct*, const pft_ct*>>>& terms, int l,
                const std::vector<u64*>& outs, bool accumulate) {
    const size_t n_out = outs.size();
    if (n_out == 0) return;
    const int K = (int)terms[0].size();
    const int n = c->n;
    size_t o0 = 0;
    while (o0 < n_out) {
        const size_t o1 = std::min(n_out, o0 + 65535);
        std::vector<const u64*> A, Bv;
        std::vector<u64*> O;
        for (size_t o = o0; o < o1; o++) {
            NEED((int)terms[o].size() == K, PFT_ERR_ARG, "internal: uneven tensor sums");
            for (auto& pr : terms[o]) {
                NEED(pr.first->level >= l && pr.second->level >= l, PFT_ERR_LEVEL_MISMATCH,
                     "internal: operand below the product level");
                A.push_back(pbase(pr.first, 0, n));
                A.push_back(pbase(pr.first, 1, n));
                Bv.push_back(pbase(pr.second, 0, n));
                Bv.push_back(pbase(pr.second, 1, n));
            }
            for (int i = 0; i < 3; i++) O.push_back(outs[o] + (size_t)i * l * n);
        }
        Scratch dA(c, A.size() * 8), dB(c, Bv.size() * 8), dO(c, O.size() * 8);
        ew_tensor_dot(c->tabs, upload(c, dA, A), upload(c, dB, Bv), upload(c, dO, O), (int)(o1 - o0), K, l,
                      accumulate, c->stream);
        o0 = o1;
    }
}

// Documents per tile: the working set of a tile (columns, their tensor products and
// backward copies) within the key-switching budget; PFT_TRAIN_TILE overrides it.
int tile_docs(const pft_ctx* c, const pft_ft_enc_model* M, int l0) {
    if (const char* e = std::getenv("PFT_TRAIN_TILE")) {
        const int v = std::atoi(e);
        if (v > 0) return v;
    }
    const size_t per_doc = M->variant == 0 ? (size_t)M->n * 7 * l0 * c->n * 8 : (size_t)(M->n + 7) * 2 * l0 * c->n * 8;
    return (int)std::max<size_t>(1, kKsScratchBudget / per_doc);
}

void check_model(const pft_ft_enc_model* M, pft_ctx* c) {
    NEED(M && M->ctx == c, PFT_ERR_ARG, "model from another context");
}

// forward of documents [b0, b1): h, s, g of the tape
void fwd_tile(pft_ctx* c, pft_ft_tape& T, const pft_ct* const* w, int b0, int b1) {
    const pft_ft_enc_model* M = T.M;
    const int n = M->n, l0 = T.l0, N = c->n, t = N / 2;
    const size_t cnt = (size_t)(b1 - b0) * n;
    // h_bj = Rescale(TotalSum(Relin(v_b x H_j)))
    std::vector<const pft_ct*> A, Bv;
    std::vector<pft_ct*> hx;
    for (int b = b0; b < b1; b++)
        for (int j = 0; j < n; j++) {
            pft_ct& x = T.h[(size_t)b * n + j];
            x.ctx = c;
            A.push_back(T.v[b]);
            Bv.push_back(&M->H[j]);
            hx.push_back(&x);
        }
    op_mul_relin_batch(c, A.data(), Bv.data(), (int)cnt, hx.data());
    for (int st = 1; st < t; st *= 2) rot_accumulate(c, hx, galois_of(N, st));
    op_rescale_batch(c, hx.data(), (int)cnt, hx.data());
    // s_b = Rescale(Relin(sum_j h_bj x O_j))
    const int l1 = l0 - 1;
    {
        Scratch S(c, (size_t)(b1 - b0) * 3 * l1 * N * 8);
        std::vector<std::vector<std::pair<const pft_ct*, const pft_ct*>>> terms(b1 - b0);
        std::vector<u64*> outs;
        std::vector<RelinIO> rio;
        std::vector<pft_ct*> sx;
        for (int b = b0; b < b1; b++) {
            for (int j = 0; j < n; j++) terms[b - b0].push_back({&T.h[(size_t)b * n + j], &M->O[j]});
            u64* buf = S.u() + (size_t)(b - b0) * 3 * l1 * N;
            outs.push_back(buf);
            pft_ct& sb = T.s[b];
            sb.ctx = c;
            rio.push_back(RelinIO{buf, l1, T.h[(size_t)b * n].scale * M->O[0].scale, &sb});
            sx.push_back(&sb);
        }
        tensor_dot(c, terms, l1, outs, false);
        relin_batch(c, rio);
        op_rescale_batch(c, sx.data(), (int)sx.size(), sx.data());
    }
    // g_b = [Rescale(Relin(u x u)), u = s + 2] read at 8x its scale, - 1/2, - w_b
    std::vector<pft_ct> u(b1 - b0);
    std::vector<pft_ct*> ux;
    std::vector<const pft_ct*> sc, ws;
    std::vector<pft_ct*> gx;
    struct Free {
        pft_ctx* c;
        std::vector<pft_ct>* u;
        ~Free() { free_cts(c, *u, 0, u->size()); }
    } fr{c, &u};
    for (int b = b0; b < b1; b++) {
        u[b - b0].ctx = c;
        ux.push_back(&u[b - b0]);
        sc.push_back(&T.s[b]);
        ws.push_back(w[b]);
        T.g[b].ctx = c;
        gx.push_back(&T.g[b]);
    }
    op_const_batch(c, sc.data(), (int)sc.size(), 2.0, 0.0, false, ux.data());
    op_mul_relin_batch(c, ux.data(), ux.data(), (int)ux.size(), ux.data());
    op_rescale_batch(c, ux.data(), (int)ux.size(), ux.data());
    for (pft_ct* x : ux) x->scale = 8.0 * x->scale;
    op_const_batch(c, ux.data(), (int)ux.size(), -0.5, 0.0, false, ux.data());
    for (size_t i = 0; i < ws.size(); i++) {
        check_ct(c, ws[i]);
        NEED(ws[i]->level == ux[i]->level, PFT_ERR_LEVEL_MISMATCH,
             "labels must be encrypted at the level pft_fasttext_train_spec gives");
        NEED(ws[i]->scale == ux[i]->scale, PFT_ERR_SCALE_MISMATCH,
             "labels must be encrypted at the scale pft_fasttext_train_spec gives");
    }
    op_add_batch(c, ux.data(), ws.data(), (int)ux.size(), gx.data(), EwOp::Sub);
}

struct Accum {
    pft_ctx* c;
    u64* O = nullptr;  // n x [3][l0-3][N]
    u64* H = nullptr;  // n x [3][l0-4][N]
    double scO = 0, scH = 0;
    ~Accum() {
        dfree(c, O);
        dfree(c, H);
    }
};

// backward of documents [b0, b1) into the accumulators
void bwd_tile(pft_ctx* c, pft_ft_tape& T, int b0, int b1, Accum& acc, bool first) {
    const pft_ft_enc_model* M = T.M;
    const int n = M->n, l0 = T.l0, N = c->n, t = N / 2;
    const int lg = l0 - 3, le = l0 - 4;
    // dO_j += sum_b h_bj x g_b
    {
        std::vector<std::vector<std::pair<const pft_ct*, const pft_ct*>>> terms(n);
        std::vector<u64*> outs;
        for (int j = 0; j < n; j++) {
            for (int b = b0; b < b1; b++) terms[j].push_back({&T.h[(size_t)b * n + j], &T.g[b]});
            outs.push_back(acc.O + (size_t)j * 3 * lg * N);
        }
        tensor_dot(c, terms, lg, outs, !first);
        acc.scO = T.h[(size_t)b0 * n].scale * T.g[b0].scale;
    }
    // e_bj = Rescale(TotalSum(Relin(g_b x O_j)))
    const size_t cnt = (size_t)(b1 - b0) * n;
    std::vector<pft_ct> E(cnt);
    struct Free {
        pft_ctx* c;
        std::vector<pft_ct>* e;
        ~Free() { free_cts(c, *e, 0, e->size()); }
    } fr{c, &E};
    std::vector<pft_ct*> ex;
    for (auto& x : E) {
        x.ctx = c;
        ex.push_back(&x);
    }
    {
        Scratch D(c, cnt * 3 * lg * N * 8);
        std::vector<std::vector<std::pair<const pft_ct*, const pft_ct*>>> terms(cnt);
        std::vector<u64*> outs;
        std::vector<RelinIO> rio;
        for (int b = b0; b < b1; b++)
            for (int j = 0; j < n; j++) {
                const size_t i = (size_t)(b - b0) * n + j;
                terms[i].push_back({&T.g[b], &M->O[j]});
                outs.push_back(D.u() + i * 3 * lg * N);
                rio.push_back(RelinIO{outs.back(), lg, T.g[b].scale * M->O[j].scale, &E[i]});
            }
        tensor_dot(c, terms, lg, outs, false);
        relin_batch(c, rio);
    }
    for (int st = 1; st < t; st *= 2) rot_accumulate(c, ex, galois_of(N, st));
    op_rescale_batch(c, ex.data(), (int)cnt, ex.data());
    // dH_j += sum_b v_b x e_bj
    {
        std::vector<std::vector<std::pair<const pft_ct*, const pft_ct*>>> terms(n);
        std::vector<u64*> outs;
        for (int j = 0; j < n; j++) {
            for (int b = b0; b < b1; b++) terms[j].push_back({T.v[b], &E[(size_t)(b - b0) * n + j]});
            outs.push_back(acc.H + (size_t)j * 3 * le * N);
        }
        tensor_dot(c, terms, le, outs, !first);
        acc.scH = T.v[b0]->scale * E[0].scale;
    }
}

// accumulator shapes: Fig. 3 layout n dO sums at l0-3 and n dH sums at l0-4; diagonal layout
// one dP sum at l0-4 and n dD sums at l0-5
struct AccShape {
    int nO, lO, nH, lH;
};
AccShape acc_shape(const pft_ft_enc_model* M, int l0) {
    return M->variant == 0 ? AccShape{M->n, l0 - 3, M->n, l0 - 4} : AccShape{1, l0 - 4, M->n, l0 - 5};
}

void alloc_accum(pft_ctx* c, const pft_ft_enc_model* M, int l0, Accum& acc) {
    const AccShape a = acc_shape(M, l0);
    acc.O = (u64*)dalloc(c, (size_t)a.nO * 3 * a.lO * c->n * 8);
    acc.H = (u64*)dalloc(c, (size_t)a.nH * 3 * a.lH * c->n * 8);
}

// gradients from the accumulators (relinearised, then rescaled once)
void finalize(pft_ctx* c, const pft_ft_enc_model* M, int l0, const Accum& acc, pft_ct* const* gH,
              pft_ct* const* gO) {
    const AccShape a = acc_shape(M, l0);
    const int N = c->n;
    std::vector<RelinIO> rio;
    std::vector<pft_ct*> all;
    for (int j = 0; j < a.nO; j++) {
        gO[j]->ctx = c;
        rio.push_back(RelinIO{acc.O + (size_t)j * 3 * a.lO * N, a.lO, acc.scO, gO[j]});
        all.push_back(gO[j]);
    }
    for (int j = 0; j < a.nH; j++) {
        gH[j]->ctx = c;
        rio.push_back(RelinIO{acc.H + (size_t)j * 3 * a.lH * N, a.lH, acc.scH, gH[j]});
        all.push_back(gH[j]);
    }
    relin_batch(c, rio);
    op_rescale_batch(c, all.data(), (int)all.size(), all.data());
}

int n_grad_O(const pft_ft_enc_model* M) { return M->variant == 0 ? M->n : 1; }

// X_j <- X_j - eta dX_j for the n ciphertexts of one weight matrix
void sgd(pft_ctx* c, std::vector<pft_ct>& X, const pft_ct* const* dX, int n, double eta) {
    const int l = dX[0]->level;
    const double sc = dX[0]->scale, target = X[0].scale;
    for (int j = 0; j < n; j++) {
        check_ct(c, dX[j]);
        NEED(dX[j]->level == l && dX[j]->scale == sc, PFT_ERR_SCALE_MISMATCH, "gradients differ in level or scale");
    }
    NEED(l >= 2, PFT_ERR_LEVEL_MISMATCH, "no level left for the update");
    const double c_sc = target * (double)c->primes[l - 1] / sc;
    std::vector<pft_ct> a(n);
    struct Free {
        pft_ctx* c;
        std::vector<pft_ct>* a;
        ~Free() { free_cts(c, *a, 0, a->size()); }
    } fr{c, &a};
    std::vector<pft_ct*> ax, xx;
    for (int j = 0; j < n; j++) {
        a[j].ctx = c;
        ax.push_back(&a[j]);
        xx.push_back(&X[j]);
    }
    op_const_batch(c, dX, n, eta, c_sc, true, ax.data());
    op_rescale_batch(c, ax.data(), n, ax.data());
    for (pft_ct* x : ax) x->scale = target;
    NEED(X[0].level >= a[0].level, PFT_ERR_LEVEL_MISMATCH, "model below the update level");
    op_drop_level_batch(c, xx.data(), n, a[0].level, xx.data());
    op_add_batch(c, xx.data(), ax.data(), n, xx.data(), EwOp::Sub);
}

// ---- diagonal layout (rotation-light; not in the paper) ---------------------------------------
// D_k[i] = H[(i + k) mod t, i mod n] at level l0, P[n c + j] = O[j, c] at l0 - 1, a plaintext
// mask with 1 in the score slots n c; labels w_b = y_b - 1/4 over block c (slots n c .. n c + n - 1).
//   lift     v'_b = 2^K v_b (exact integer product; K = 0: v_b itself)
//   forward  R_bk = rot(v'_b, k) (hoisted), Hb = Rescale(rotsum_{n 2^s}(Relin(sum_k R_bk x D_k))) l0-1
//            Sb = Rescale(rotsum_{2^s < n}(Relin(Hb x P)))  (s_b[c] in slot n c)                   l0-2
//            Sm = Rescale(rotsum_{-2^s}(Sb * mask))  (s_b[c] over block c)                          l0-3
//            Gb = [Rescale(Relin(u x u)), u = Sm + 2] / 8 - 1/2 - w_b                               l0-4
//   backward dP = Rescale(Relin(sum_b Hb x Gb))                                                   l0-5
//            Eb = Rescale(rotsum_{n 2^s}(Relin(Gb x P)))  (e_b[i mod n] in slot i)                l0-5
//            dD_k = Rescale(Relin(sum_b R_bk x Eb))  (the diagonals of dH)                        l0-6
//   update   D_k -> l0-7, P -> l0-8 (one level below the diagonals)
// The document rotations are the only key switches at the input scale; the sums over the
// vocabulary collect their rounding noise, which the lift divides by 2^K.  Spreading the masked
// scores before their rescale keeps the rescale noise of neighbouring slots out of Gb.
void rot_sum(pft_ctx* c, std::vector<pft_ct*>& T, int first, int below, int sign) {
    for (int st = first; st < below; st *= 2) rot_accumulate(c, T, galois_of(c->n, sign * st));
}

// R_bk of the tape: k = 0 the (lifted) document, else its rotation by k
const pft_ct* doc_rot(const pft_ft_tape& T, int b, int k) {
    return k == 0 && T.M->lift == 0 ? T.v[b] : &T.r[(size_t)b * T.M->n + k];
}

void fwd_tile_diag(pft_ctx* c, pft_ft_tape& T, const pft_ct* const* w, int b0, int b1) {
    const pft_ft_enc_model* M = T.M;
    const int n = M->n, l0 = T.l0, N = c->n, t = N / 2;
    const int nb = b1 - b0;
    // v'_b = 2^K v_b, then R_bk = rot(v'_b, k), k = 1..n-1, sharing one ModUp per document
    if (M->lift > 0) {
        std::vector<const pft_ct*> vin;
        std::vector<pft_ct*> vout;
        for (int b = b0; b < b1; b++) {
            vin.push_back(T.v[b]);
            vout.push_back(&T.r[(size_t)b * n]);
        }
        op_const_batch(c, vin.data(), nb, 1.0, std::ldexp(1.0, M->lift), true, vout.data());
    }
    auto rk = [&](int b, int k) -> const pft_ct* { return doc_rot(T, b, k); };
    std::vector<int32_t> hs;
    for (int k = 1; k < n; k++) hs.push_back(k);
    for (int b = b0; b < b1; b++) {
        std::vector<pft_ct*> outs;
        for (int k = 1; k < n; k++) outs.push_back(&T.r[(size_t)b * n + k]);
        if (n > 1) op_rotate_hoisted(c, rk(b, 0), hs.data(), n - 1, outs.data());
    }
    // Hb
    std::vector<pft_ct*> hx;
    {
        Scratch S(c, (size_t)nb * 3 * l0 * N * 8);
        std::vector<std::vector<std::pair<const pft_ct*, const pft_ct*>>> terms(nb);
        std::vector<u64*> outs;
        std::vector<RelinIO> rio;
        for (int b = b0; b < b1; b++) {
            for (int k = 0; k < n; k++) terms[b - b0].push_back({rk(b, k), &M->H[k]});
            outs.push_back(S.u() + (size_t)(b - b0) * 3 * l0 * N);
            T.h[b].ctx = c;
            rio.push_back(RelinIO{outs.back(), l0, rk(b, 0)->scale * M->H[0].scale, &T.h[b]});
            hx.push_back(&T.h[b]);
        }
        tensor_dot(c, terms, l0, outs, false);
        relin_batch(c, rio);
    }
    rot_sum(c, hx, n, t, 1);
    op_rescale_batch(c, hx.data(), nb, hx.data());
    // Sb, then the mask
    const int l1 = l0 - 1;
    std::vector<pft_ct*> sx;
    {
        Scratch S(c, (size_t)nb * 3 * l1 * N * 8);
        std::vector<std::vector<std::pair<const pft_ct*, const pft_ct*>>> terms(nb);
        std::vector<u64*> outs;
        std::vector<RelinIO> rio;
        for (int b = b0; b < b1; b++) {
            terms[b - b0].push_back({&T.h[b], &M->O[0]});
            outs.push_back(S.u() + (size_t)(b - b0) * 3 * l1 * N);
            T.s[b].ctx = c;
            rio.push_back(RelinIO{outs.back(), l1, T.h[b].scale * M->O[0].scale, &T.s[b]});
            sx.push_back(&T.s[b]);
        }
        tensor_dot(c, terms, l1, outs, false);
        relin_batch(c, rio);
    }
    rot_sum(c, sx, 1, n, 1);
    op_rescale_batch(c, sx.data(), nb, sx.data());
    {
        std::vector<PolyRef> ra, rb, ro;
        for (pft_ct* x : sx) {
            const int l = x->level;
            for (int pol = 0; pol < 2; pol++) {
                ra.push_back(cpoly(x->data, l, N, pol));
                rb.push_back(ref(M->mask.data, l));
                ro.push_back(cpoly(x->data, l, N, pol));
            }
            x->scale = x->scale * M->mask.scale;
        }
        ew(c, EwOp::Mul, ra, rb, ro);
    }
    rot_sum(c, sx, 1, n, -1);
    op_rescale_batch(c, sx.data(), nb, sx.data());
    // Gb, as g_b in the Fig. 3 layout (here over the class blocks)
    std::vector<pft_ct> u(nb);
    struct Free {
        pft_ctx* c;
        std::vector<pft_ct>* u;
        ~Free() { free_cts(c, *u, 0, u->size()); }
    } fr{c, &u};
    std::vector<pft_ct*> ux, gx;
    std::vector<const pft_ct*> sc, ws;
    for (int b = b0; b < b1; b++) {
        u[b - b0].ctx = c;
        ux.push_back(&u[b - b0]);
        sc.push_back(&T.s[b]);
        ws.push_back(w[b]);
        T.g[b].ctx = c;
        gx.push_back(&T.g[b]);
    }
    op_const_batch(c, sc.data(), nb, 2.0, 0.0, false, ux.data());
    op_mul_relin_batch(c, ux.data(), ux.data(), nb, ux.data());
    op_rescale_batch(c, ux.data(), nb, ux.data());
    for (pft_ct* x : ux) x->scale = 8.0 * x->scale;
    op_const_batch(c, ux.data(), nb, -0.5, 0.0, false, ux.data());
    for (int i = 0; i < nb; i++) {
        check_ct(c, ws[i]);
        NEED(ws[i]->level == ux[i]->level, PFT_ERR_LEVEL_MISMATCH,
             "labels must be encrypted at the level pft_fasttext_train_spec gives");
        NEED(ws[i]->scale == ux[i]->scale, PFT_ERR_SCALE_MISMATCH,
             "labels must be encrypted at the scale pft_fasttext_train_spec gives");
    }
    op_add_batch(c, ux.data(), ws.data(), nb, gx.data(), EwOp::Sub);
}

void bwd_tile_diag(pft_ctx* c, pft_ft_tape& T, int b0, int b1, Accum& acc, bool first) {
    const pft_ft_enc_model* M = T.M;
    const int n = M->n, l0 = T.l0, N = c->n, t = N / 2;
    const int nb = b1 - b0, lg = l0 - 4, le = l0 - 5;
    // dP += sum_b Hb x Gb
    {
        std::vector<std::vector<std::pair<const pft_ct*, const pft_ct*>>> terms(1);
        for (int b = b0; b < b1; b++) terms[0].push_back({&T.h[b], &T.g[b]});
        tensor_dot(c, terms, lg, {acc.O}, !first);
        acc.scO = T.h[b0].scale * T.g[b0].scale;
    }
    // Eb = Rescale(rotsum_{n 2^s}(Relin(Gb x P)))
    std::vector<pft_ct> E(nb);
    struct Free {
        pft_ctx* c;
        std::vector<pft_ct>* e;
        ~Free() { free_cts(c, *e, 0, e->size()); }
    } fr{c, &E};
    std::vector<pft_ct*> ex;
    for (auto& x : E) {
        x.ctx = c;
        ex.push_back(&x);
    }
    {
        Scratch D(c, (size_t)nb * 3 * lg * N * 8);
        std::vector<std::vector<std::pair<const pft_ct*, const pft_ct*>>> terms(nb);
        std::vector<u64*> outs;
        std::vector<RelinIO> rio;
        for (int b = b0; b < b1; b++) {
            terms[b - b0].push_back({&T.g[b], &M->O[0]});
            outs.push_back(D.u() + (size_t)(b - b0) * 3 * lg * N);
            rio.push_back(RelinIO{outs.back(), lg, T.g[b].scale * M->O[0].scale, &E[b - b0]});
        }
        tensor_dot(c, terms, lg, outs, false);
        relin_batch(c, rio);
    }
    rot_sum(c, ex, n, t, 1);
    op_rescale_batch(c, ex.data(), nb, ex.data());
    // dD_k += sum_b R_bk x Eb
    {
        std::vector<std::vector<std::pair<const pft_ct*, const pft_ct*>>> terms(n);
        std::vector<u64*> outs;
        for (int k = 0; k < n; k++) {
            for (int b = b0; b < b1; b++) terms[k].push_back({doc_rot(T, b, k), &E[b - b0]});
            outs.push_back(acc.H + (size_t)k * 3 * le * N);
        }
        tensor_dot(c, terms, le, outs, !first);
        acc.scH = doc_rot(T, b0, 0)->scale * E[0].scale;
    }
}

// levels a call needs: forward and backward / with the update
int levels_needed(const pft_ft_enc_model* M, bool update) {
    return M->variant == 0 ? (update ? 7 : 6) : (update ? 9 : 7);
}

void check_batch(pft_ctx* c, const pft_ft_enc_model* M, const pft_ct* const* docs, const pft_ct* const* labels,
                 int B, bool with_update) {
    check_model(M, c);
    NEED(B >= 1 && docs && labels, PFT_ERR_ARG, "bad arguments");
    const int l0 = M->H[0].level;
    const int min_level = levels_needed(M, with_update);
    NEED(l0 >= min_level, PFT_ERR_LEVEL_MISMATCH,
         "the model has " + std::to_string(l0) + " levels left, this call needs " + std::to_string(min_level));
    NEED(c->keys.count(0), PFT_ERR_NO_KEY, "no relinearisation key");
    const int t = c->n / 2;
    std::vector<int> steps;
    if (M->variant == 0) {
        for (int st = 1; st < t; st *= 2) steps.push_back(st);
    } else {
        for (int k = 1; k < M->n; k++) steps.push_back(k);
        for (int st = M->n; st < t; st *= 2) steps.push_back(st);
        for (int st = 1; st < M->n; st *= 2) steps.push_back(-st);
    }
    for (int st : steps)
        NEED(c->keys.count(galois_of(c->n, st)), PFT_ERR_NO_KEY, "missing rotation key for step " + std::to_string(st));
    for (int b = 0; b < B; b++) {
        check_ct(c, docs[b]);
        check_ct(c, labels[b]);
        NEED(docs[b]->level == l0, PFT_ERR_LEVEL_MISMATCH, "documents must sit at the model level");
        NEED(docs[b]->scale == docs[0]->scale, PFT_ERR_SCALE_MISMATCH, "documents differ in scale");
    }
}

void init_tape(pft_ctx* c, const pft_ft_enc_model* M, const pft_ct* const* docs, int B, pft_ft_tape& T) {
    T.ctx = c;
    T.M = M;
    T.B = B;
    T.l0 = M->H[0].level;
    T.v.assign(docs, docs + B);
    T.h.resize(M->variant == 0 ? (size_t)B * M->n : (size_t)B);
    T.s.resize(B);
    T.g.resize(B);
    if (M->variant == 1) T.r.resize((size_t)B * M->n);
    for (auto* vec : {&T.h, &T.s, &T.g, &T.r})
        for (auto& x : *vec) x.ctx = c;
}

void copy_ct(pft_ctx* c, const pft_ct& src, pft_ct* out) {
    NEED(out, PFT_ERR_ARG, "null output");
    ensure_ct(c, out, src.level);
    out->ctx = c;
    out->scale = src.scale;
    PFT_CUDA(cudaMemcpyAsync(out->data, src.data, (size_t)2 * src.level * c->n * 8, cudaMemcpyDeviceToDevice,
                             c->stream));
}

// SGD: Fig. 3 layout O then H; diagonal layout the diagonals, then P, which is dropped one level
// below the diagonals' new level
void update(pft_ctx* c, pft_ft_enc_model* M, const pft_ct* const* gH, const pft_ct* const* gO, double eta) {
    sgd(c, M->H, gH, M->n, eta);
    if (M->variant == 0) {
        sgd(c, M->O, gO, M->n, eta);
    } else {
        sgd(c, M->O, gO, 1, eta);
        pft_ct* p = &M->O[0];
        op_drop_level_batch(c, &p, 1, M->H[0].level - 1, &p);
    }
}

}  // namespace

extern "C" {

int pft_ft_enc_model_create(pft_ctx* c, const pft_ct* const* H, const pft_ct* const* O, int m, int n, int cl,
                            pft_ft_enc_model** out) {
    return guard(c, [&] {
        NEED(c && H && O && out && n >= 1 && cl >= 1 && m >= 1, PFT_ERR_ARG, "bad arguments");
        NEED(m <= c->n / 2 && cl <= c->n / 2, PFT_ERR_ARG, "the vocabulary and the classes must fit one ciphertext");
        std::unique_ptr<pft_ft_enc_model> M(new pft_ft_enc_model());
        M->ctx = c;
        M->m = m;
        M->n = n;
        M->c = cl;
        for (int j = 0; j < n; j++) {
            check_ct(c, H[j]);
            check_ct(c, O[j]);
            NEED(H[j]->level == H[0]->level && H[j]->scale == H[0]->scale, PFT_ERR_LEVEL_MISMATCH,
                 "embedding ciphertexts differ in level or scale");
            NEED(O[j]->level == H[0]->level - 1 && O[j]->scale == O[0]->scale, PFT_ERR_LEVEL_MISMATCH,
                 "output-layer ciphertexts must sit one level below the embedding, at one scale");
        }
        M->H.resize(n);
        M->O.resize(n);
        for (int j = 0; j < n; j++) {
            M->H[j].ctx = c;
            M->O[j].ctx = c;
            copy_ct(c, *H[j], &M->H[j]);
            copy_ct(c, *O[j], &M->O[j]);
        }
        *out = M.release();
    });
}

int pft_ft_enc_model_create_diag(pft_ctx* c, const pft_ct* const* D, const pft_ct* P, const pft_pt* mask, int m,
                                 int n, int cl, int lift_bits, pft_ft_enc_model** out) {
    return guard(c, [&] {
        NEED(c && D && P && mask && out && n >= 1 && cl >= 1 && m >= 1, PFT_ERR_ARG, "bad arguments");
        NEED(lift_bits >= 0 && lift_bits <= 30, PFT_ERR_ARG, "lift_bits must lie in 0..30");
        const int t = c->n / 2;
        NEED(m <= t && (n & (n - 1)) == 0 && t % n == 0 && (size_t)n * cl <= (size_t)t, PFT_ERR_ARG,
             "the diagonal layout needs m <= t, n a power of two dividing t and n c <= t");
        check_ct(c, P);
        check_pt(c, mask);
        std::unique_ptr<pft_ft_enc_model> M(new pft_ft_enc_model());
        M->ctx = c;
        M->m = m;
        M->n = n;
        M->c = cl;
        M->variant = 1;
        M->lift = lift_bits;
        for (int k = 0; k < n; k++) {
            check_ct(c, D[k]);
            NEED(D[k]->level == D[0]->level && D[k]->scale == D[0]->scale, PFT_ERR_LEVEL_MISMATCH,
                 "diagonal ciphertexts differ in level or scale");
        }
        NEED(P->level == D[0]->level - 1, PFT_ERR_LEVEL_MISMATCH, "the output layer must sit one level below");
        NEED(mask->level >= D[0]->level - 2, PFT_ERR_LEVEL_MISMATCH, "the mask must reach the score level");
        M->H.resize(n);
        M->O.resize(1);
        for (int k = 0; k < n; k++) {
            M->H[k].ctx = c;
            copy_ct(c, *D[k], &M->H[k]);
        }
        M->O[0].ctx = c;
        copy_ct(c, *P, &M->O[0]);
        M->mask.ctx = c;
        ensure_pt(c, &M->mask, mask->level);
        M->mask.scale = mask->scale;
        PFT_CUDA(cudaMemcpyAsync(M->mask.data, mask->data, (size_t)mask->level * c->n * 8, cudaMemcpyDeviceToDevice,
                                 c->stream));
        *out = M.release();
    });
}

int pft_ft_enc_model_get(pft_ctx* c, const pft_ft_enc_model* M, int which, int j, pft_ct* out) {
    return guard(c, [&] {
        check_model(M, c);
        NEED((which == 0 && j >= 0 && j < M->n) || (which == 1 && j >= 0 && j < n_grad_O(M)), PFT_ERR_ARG,
             "no such weight ciphertext");
        copy_ct(c, which == 0 ? M->H[j] : M->O[j], out);
    });
}

int pft_ft_enc_model_levels(const pft_ft_enc_model* M, int* level_H, int* level_O) {
    if (!M || !level_H || !level_O) return PFT_ERR_ARG;
    *level_H = M->H[0].level;
    *level_O = M->O[0].level;
    return PFT_OK;
}

int pft_ft_enc_model_destroy(pft_ft_enc_model* M) {
    delete M;
    return PFT_OK;
}

int pft_fasttext_train_spec(pft_ctx* c, const pft_ft_enc_model* M, double input_scale, int* doc_level,
                            int* label_level, double* label_scale) {
    return guard(c, [&] {
        check_model(M, c);
        NEED(doc_level && label_level && label_scale && input_scale > 0, PFT_ERR_ARG, "bad arguments");
        const int l0 = M->H[0].level;
        NEED(l0 >= (M->variant == 0 ? 4 : 5), PFT_ERR_LEVEL_MISMATCH, "the model has too few levels left");
        const double sh = std::ldexp(input_scale, M->lift) * M->H[0].scale / (double)c->primes[l0 - 1];
        const double ss = sh * M->O[0].scale / (double)c->primes[l0 - 2];
        if (M->variant == 0) {
            const double su = ss * ss / (double)c->primes[l0 - 3];
            *label_level = l0 - 3;
            *label_scale = 8.0 * su;
        } else {  // one more level: the mask of the score slots
            const double sm = ss * M->mask.scale / (double)c->primes[l0 - 3];
            const double su = sm * sm / (double)c->primes[l0 - 4];
            *label_level = l0 - 4;
            *label_scale = 8.0 * su;
        }
        *doc_level = l0;
    });
}

int pft_fasttext_train_forward(pft_ctx* c, const pft_ft_enc_model* M, const pft_ct* const* docs,
                               const pft_ct* const* labels, int B, pft_ft_tape** out) {
    return guard(c, [&] {
        NEED(out, PFT_ERR_ARG, "bad arguments");
        check_batch(c, M, docs, labels, B, false);
        std::unique_ptr<pft_ft_tape> T(new pft_ft_tape());
        init_tape(c, M, docs, B, *T);
        const int tile = tile_docs(c, M, T->l0);
        for (int b0 = 0; b0 < B; b0 += tile) {
            if (M->variant == 0) fwd_tile(c, *T, labels, b0, std::min(B, b0 + tile));
            else fwd_tile_diag(c, *T, labels, b0, std::min(B, b0 + tile));
        }
        *out = T.release();
    });
}

int pft_ft_tape_score(pft_ctx* c, const pft_ft_tape* T, int b, pft_ct* out) {
    return guard(c, [&] {
        NEED(T && T->ctx == c && b >= 0 && b < T->B, PFT_ERR_ARG, "bad arguments");
        copy_ct(c, T->s[b], out);
    });
}

int pft_fasttext_train_backward(pft_ctx* c, const pft_ft_tape* T, pft_ct* const* grad_H, pft_ct* const* grad_O) {
    return guard(c, [&] {
        NEED(T && T->ctx == c && grad_H && grad_O, PFT_ERR_ARG, "bad arguments");
        const pft_ft_enc_model* M = T->M;
        for (int j = 0; j < M->n; j++) NEED(grad_H[j], PFT_ERR_ARG, "null gradient handle");
        for (int j = 0; j < n_grad_O(M); j++) NEED(grad_O[j], PFT_ERR_ARG, "null gradient handle");
        Accum acc{c};
        alloc_accum(c, M, T->l0, acc);
        const int tile = tile_docs(c, M, T->l0);
        pft_ft_tape& W = const_cast<pft_ft_tape&>(*T);  // read only: the backward does not modify the tape
        for (int b0 = 0; b0 < T->B; b0 += tile) {
            if (M->variant == 0) bwd_tile(c, W, b0, std::min(T->B, b0 + tile), acc, b0 == 0);
            else bwd_tile_diag(c, W, b0, std::min(T->B, b0 + tile), acc, b0 == 0);
        }
        finalize(c, M, T->l0, acc, grad_H, grad_O);
    });
}

int pft_ft_tape_destroy(pft_ft_tape* T) {
    delete T;
    return PFT_OK;
}

int pft_fasttext_train_update(pft_ctx* c, pft_ft_enc_model* M, const pft_ct* const* grad_H,
                              const pft_ct* const* grad_O, double eta) {
    return guard(c, [&] {
        check_model(M, c);
        NEED(grad_H && grad_O && std::isfinite(eta), PFT_ERR_ARG, "bad arguments");
        if (eta == 0) return;
        update(c, M, grad_H, grad_O, eta);
    });
}

int pft_fasttext_train_step(pft_ctx* c, pft_ft_enc_model* M, const pft_ct* const* docs, const pft_ct* const* labels,
                            int B, double eta, pft_ct* const* grad_H, pft_ct* const* grad_O) {
    return guard(c, [&] {
        NEED(std::isfinite(eta), PFT_ERR_ARG, "bad learning rate");
        check_batch(c, M, docs, labels, B, eta != 0);
        const int n = M->n, no = n_grad_O(M);
        std::vector<pft_ct> own;  // gradients the caller does not keep
        std::vector<pft_ct*> gH(n), gO(no);
        if (!grad_H || !grad_O) own.resize((size_t)n + no);
        struct Free {
            pft_ctx* c;
            std::vector<pft_ct>* v;
            ~Free() { free_cts(c, *v, 0, v->size()); }
        } fr{c, &own};
        for (int j = 0; j < n; j++) {
            gH[j] = grad_H ? grad_H[j] : &own[j];
            NEED(gH[j], PFT_ERR_ARG, "null gradient handle");
            gH[j]->ctx = c;
        }
        for (int j = 0; j < no; j++) {
            gO[j] = grad_O ? grad_O[j] : &own[(size_t)n + j];
            NEED(gO[j], PFT_ERR_ARG, "null gradient handle");
            gO[j]->ctx = c;
        }
        pft_ft_tape T;
        init_tape(c, M, docs, B, T);
        Accum acc{c};
        alloc_accum(c, M, T.l0, acc);
        const int tile = tile_docs(c, M, T.l0);
        const size_t per_h = M->variant == 0 ? (size_t)n : 1;
        for (int b0 = 0; b0 < B; b0 += tile) {
            const int b1 = std::min(B, b0 + tile);
            if (M->variant == 0) {
                fwd_tile(c, T, labels, b0, b1);
                bwd_tile(c, T, b0, b1, acc, b0 == 0);
            } else {
                fwd_tile_diag(c, T, labels, b0, b1);
                bwd_tile_diag(c, T, b0, b1, acc, b0 == 0);
                free_cts(c, T.r, (size_t)b0 * n, (size_t)b1 * n);
            }
            free_cts(c, T.h, b0 * per_h, b1 * per_h);
            free_cts(c, T.s, b0, b1);
            free_cts(c, T.g, b0, b1);
        }
        finalize(c, M, T.l0, acc, gH.data(), gO.data());
        if (eta != 0) update(c, M, gH.data(), gO.data(), eta);
    });
}

}  // extern "C"
