// Handles of the evaluator and the host-side helpers shared by its translation units
// (the operations in ckks.cu, the request server in serve.cu).
#pragma once
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "pft_internal.h"

using namespace pft;

#define NEED(cond, code, msg) \
    do {                      \
        if (!(cond)) fail(code, msg); \
    } while (0)

// ---- handles ---------------------------------------------------------------------------
struct pft_ctx {
    pft_params prm;
    int device = 0;                 // CUDA device current at creation; all work runs there
    u64* noalloc_scratch = nullptr;  // device address of the fixed array of pft_rescale_noalloc
    std::string autotune_report;     // JSON of the last pft_autotune search
    int logn = 0, n = 0, L = 0, k = 0, alpha = 0, beta_max = 0;
    std::vector<u64> primes;  // q_0..q_{L-1}, p_0..p_{k-1}
    pft_allocator alloc{};
    bool has_alloc = false;
    cudaStream_t stream = nullptr;
    std::string err;
    DevTables tabs{};
    std::vector<void*> owned;  // table buffers
    // basis-conversion tables: modup[(l-1) * beta_max + j], moddown[l-1] (device offsets)
    std::vector<const u64*> modup_tab, moddown_tab;
    // the same with every source constant times N^-1 (for inputs of an inverse transform that
    // skipped its N^-1)
    std::vector<const u64*> modup_tab_u, moddown_tab_u;
    // the byte-plane tables of the tensor-core conversion (jobs of four source primes; else null)
    std::vector<const uint32_t*> modup_tc, moddown_tc;
    const u64* moddown_consts = nullptr;           // [L][3] {0, P^-1, shoup}
    std::vector<const u64*> rescale_consts;        // [l-1] -> [l-1][3] {0, p^-1, shoup}
    std::vector<const u64*> pmodq_consts;          // digit j -> [alpha][3] {0, P mod q_m, shoup}
    std::vector<u64> P_mod_q;
    std::vector<u32> cdt;
    // keys
    bool have_sk = false;
    u64* s_ntt = nullptr;  // [L+k][N]
    std::vector<i64> s_coeff;
    u64* pk = nullptr;  // [2][L][N]  (b, a)
    std::map<u32, u64*> keys;  // [beta][2][L+k][N], or [beta][L+k][N] (b only) when compressed
    std::map<u32, u64*> keys_mont;  // uncompressed keys in split Montgomery form (KeyRef::mont)
    bool compressed_keys = false;
};

// Every ciphertext and plaintext object -- the handles given to callers and the library's own
// temporaries -- is recorded while it exists, so that a call given a destroyed handle (or a
// pointer that never was one) fails with PFT_ERR_ARG instead of reading freed memory.  A
// pointer value that a later handle happens to reuse is that later handle.
void handle_add(const void* h);
void handle_remove(const void* h);
bool handle_live(const void* h);
struct pft_ct {
    pft_ctx* ctx = nullptr;
    u64* data = nullptr;
    size_t cap = 0;  // words
    int level = 0;
    double scale = 1.0;
    pft_ct() { handle_add(this); }
    pft_ct(const pft_ct& o) : ctx(o.ctx), data(o.data), cap(o.cap), level(o.level), scale(o.scale) { handle_add(this); }
    pft_ct& operator=(const pft_ct&) = default;
    ~pft_ct() { handle_remove(this); }
};
struct pft_pt {
    pft_ctx* ctx = nullptr;
    u64* data = nullptr;
    size_t cap = 0;
    int level = 0;
    double scale = 1.0;
    pft_pt() { handle_add(this); }
    pft_pt(const pft_pt& o) : ctx(o.ctx), data(o.data), cap(o.cap), level(o.level), scale(o.scale) { handle_add(this); }
    pft_pt& operator=(const pft_pt&) = default;
    ~pft_pt() { handle_remove(this); }
};
struct pft_graph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};
struct pft_ft_model {
    pft_ctx* ctx = nullptr;
    int m = 0, n = 0, c = 0, chunks = 0, level = 0;
    int variant = 0;            // 0: Fig. 3 packing; 1: diagonal packing (rotation-light)
    std::vector<pft_pt*> H, O;  // owned copies (variant 1: H = diagonals D_k, O = {P})
};

// ---- memory --------------------------------------------------------------------------
inline void* dalloc(pft_ctx* c, size_t bytes) {
    if (bytes == 0) return nullptr;
    void* p = nullptr;
    if (c->has_alloc) {
        p = c->alloc.alloc(bytes, (void*)c->stream, c->alloc.user);
    } else {
        cudaError_t e = cudaMallocAsync(&p, bytes, c->stream);
        if (e != cudaSuccess) p = nullptr;
    }
    if (!p) fail(PFT_ERR_OOM, "device allocation of " + std::to_string(bytes) + " bytes failed");
    return p;
}
inline void dfree(pft_ctx* c, void* p) {
    if (!p) return;
    if (c->has_alloc) c->alloc.free(p, (void*)c->stream, c->alloc.user);
    else cudaFreeAsync(p, c->stream);
}
struct Scratch {
    pft_ctx* c;
    void* p;
    Scratch(pft_ctx* c_, size_t bytes) : c(c_), p(dalloc(c_, bytes)) {}
    ~Scratch() { dfree(c, p); }
    u64* u() const { return (u64*)p; }
    Scratch(const Scratch&) = delete;
    Scratch& operator=(const Scratch&) = delete;
};
template <class T>
inline T* upload(pft_ctx* c, Scratch& s, const std::vector<T>& v) {
    PFT_CUDA(cudaMemcpyAsync(s.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, c->stream));
    return (T*)s.p;
}
inline void ensure_ct(pft_ctx* c, pft_ct* ct, int level) {
    NEED(ct && handle_live(ct), PFT_ERR_ARG, "output is not a live ciphertext handle");
    NEED(!ct->ctx || ct->ctx == c, PFT_ERR_ARG, "output handle from another context");
    ct->ctx = c;
    const size_t need = (size_t)2 * level * c->n;
    if (ct->cap < need) {
        dfree(c, ct->data);
        ct->data = nullptr;
        ct->cap = 0;
        ct->data = (u64*)dalloc(c, need * 8);
        ct->cap = need;
    }
    ct->level = level;
}
inline void ensure_pt(pft_ctx* c, pft_pt* pt, int level) {
    NEED(pt && handle_live(pt), PFT_ERR_ARG, "output is not a live plaintext handle");
    NEED(!pt->ctx || pt->ctx == c, PFT_ERR_ARG, "output handle from another context");
    pt->ctx = c;
    const size_t need = (size_t)level * c->n;
    if (pt->cap < need) {
        dfree(c, pt->data);
        pt->data = nullptr;
        pt->cap = 0;
        pt->data = (u64*)dalloc(c, need * 8);
        pt->cap = need;
    }
    pt->level = level;
}

// ---- polynomial references ------------------------------------------------------------
inline PolyRef ref(u64* p, int nlimbs, int first = 0, int split = -1, int base2 = 0) {
    PolyRef r;
    r.ptr = p;
    r.nlimbs = (uint16_t)nlimbs;
    r.first = (uint16_t)first;
    r.split = (uint16_t)(split < 0 ? nlimbs : split);
    r.base2 = (uint16_t)base2;
    return r;
}
inline PolySet mkset(const std::vector<PolyRef>& v, size_t a, size_t b) {
    PolySet s;
    s.count = (int)(b - a);
    s.max_limbs = 0;
    for (size_t i = a; i < b; i++) {
        s.p[i - a] = v[i];
        s.max_limbs = std::max<int>(s.max_limbs, v[i].nlimbs);
    }
    return s;
}
template <class F>
inline void chunks(size_t n, F f) {
    for (size_t i = 0; i < n; i += kMaxSet) f(i, std::min(n, i + (size_t)kMaxSet));
}
inline void ntt_fwd(pft_ctx* c, const std::vector<PolyRef>& in, const std::vector<PolyRef>& out) {
    chunks(out.size(), [&](size_t a, size_t b) { ntt_forward(c->tabs, mkset(in, a, b), mkset(out, a, b), c->stream); });
}
inline void ntt_inv(pft_ctx* c, const std::vector<PolyRef>& in, const std::vector<PolyRef>& out) {
    chunks(out.size(), [&](size_t a, size_t b) { ntt_inverse(c->tabs, mkset(in, a, b), mkset(out, a, b), c->stream); });
}
// N times the inverse transform where the transform variant has that kernel (true), else the
// inverse transform itself (false)
inline bool ntt_inv_unscaled(pft_ctx* c, const std::vector<PolyRef>& in, const std::vector<PolyRef>& out) {
    bool unscaled = true;
    chunks(out.size(), [&](size_t a, size_t b) {
        if (unscaled) unscaled = ntt_inverse_unscaled(c->tabs, mkset(in, a, b), mkset(out, a, b), c->stream);
    });
    if (!unscaled) ntt_inv(c, in, out);
    return unscaled;
}
inline void ew(pft_ctx* c, EwOp op, const std::vector<PolyRef>& a, const std::vector<PolyRef>& b,
               const std::vector<PolyRef>& out) {
    chunks(out.size(), [&](size_t x, size_t y) {
        ew_binary(c->tabs, op, mkset(a, x, y), mkset(b.empty() ? a : b, x, y), mkset(out, x, y), c->stream);
    });
}
inline void subscale(pft_ctx* c, const std::vector<PolyRef>& x, const std::vector<PolyRef>* y,
                     const std::vector<PolyRef>* acc, const std::vector<PolyRef>& out, const u64* consts) {
    chunks(out.size(), [&](size_t a, size_t b) {
        PolySet sx = mkset(x, a, b), so = mkset(out, a, b);
        PolySet sy, sa;
        if (y) sy = mkset(*y, a, b);
        if (acc) sa = mkset(*acc, a, b);
        sub_scale(c->tabs, sx, y ? &sy : nullptr, acc ? &sa : nullptr, so, consts, c->stream);
    });
}
// the two polynomials of a ciphertext buffer [2][l][N]
inline PolyRef cpoly(u64* data, int l, int n, int pol) { return ref(data + (size_t)pol * l * n, l); }

// ---- the C ABI guard ------------------------------------------------------------------
template <class F>
inline int guard(pft_ctx* c, F f) {
    try {
        f();
        return PFT_OK;
    } catch (const Error& e) {
        if (c) c->err = e.msg;
        return e.code;
    } catch (const std::bad_alloc&) {
        if (c) c->err = "host out of memory";
        return PFT_ERR_OOM;
    } catch (const std::exception& e) {
        if (c) c->err = e.what();
        return PFT_ERR_ARG;
    }
}
inline void check_ct(const pft_ct* a) {
    NEED(a && handle_live(a), PFT_ERR_ARG, "not a live ciphertext handle (destroyed, or never created)");
    NEED(a->ctx && a->data && a->level > 0, PFT_ERR_ARG, "empty ciphertext");
}
inline void check_pt(const pft_pt* a) {
    NEED(a && handle_live(a), PFT_ERR_ARG, "not a live plaintext handle (destroyed, or never created)");
    NEED(a->ctx && a->data && a->level > 0, PFT_ERR_ARG, "empty plaintext");
}
// The same, for a handle that must belong to context c.
inline void check_ct(const pft_ctx* c, const pft_ct* a) {
    check_ct(a);
    NEED(a->ctx == c, PFT_ERR_ARG, "ciphertext handle from another context");
}
inline void check_pt(const pft_ctx* c, const pft_pt* a) {
    check_pt(a);
    NEED(a->ctx == c, PFT_ERR_ARG, "plaintext handle from another context");
}

// ---- operations shared by the translation units (ckks.cu) ----------------------------------
// Galois element 5^step mod 2N of a left rotation by `step` slots.
u32 galois_of(int n, int32_t step);
struct KsIO {
    const u64* d;     // [l][N] evaluation form
    const u64* acc0;  // may be null
    const u64* acc1;  // may be null
    u64* out0;
    u64* out1;
    int l;  // level of this input
};
// For each input d (any level): (out0, out1) = (acc0, acc1) + ModDown(sum_j ModUp_j(d) * key_j).
void keyswitch_batch(pft_ctx* c, u32 key_id, const std::vector<KsIO>& io);
// The key as the inner product reads it (full or compressed).
KeyRef keyref(pft_ctx* c, u32 key_id);
void op_add_batch(pft_ctx* c, const pft_ct* const* a, const pft_ct* const* b, int B, pft_ct* const* out, EwOp op);
void op_mul_plain_batch(pft_ctx* c, const pft_ct* const* a, const pft_pt* const* p, int B, pft_ct* const* out);
void op_mul_relin_batch(pft_ctx* c, const pft_ct* const* a, const pft_ct* const* b, int B, pft_ct* const* out);
void op_rescale_batch(pft_ctx* c, const pft_ct* const* a, int B, pft_ct* const* out);
// Rotations of one ciphertext by several steps sharing one ModUp (hoisting).
void op_rotate_hoisted(pft_ctx* c, const pft_ct* a, const int32_t* steps, int n, pft_ct* const* outs);
// T[i] += rotate(T[i], g) for every ciphertext of T (any levels), tiled to bound scratch memory.
void rot_accumulate(pft_ctx* c, const std::vector<pft_ct*>& T, u32 g);
// out[i] = the first `level` limbs of a[i] (the same message at a lower level).
void op_drop_level_batch(pft_ctx* c, const pft_ct* const* a, int B, int level, pft_ct* const* out);
// mul = false: out[i] = a[i] + value (the constant round(value * scale) added to c0);
// mul = true:  out[i] = a[i] * round(value * const_scale), scale multiplied by const_scale.
void op_const_batch(pft_ctx* c, const pft_ct* const* a, int B, double value, double const_scale, bool mul,
                    pft_ct* const* out);
// Relinearisation of three-polynomial buffers [3][l][N] (d0, d1, d2) into out[i] (level l, scale).
struct RelinIO {
    const u64* d;
    int l;
    double scale;
    pft_ct* out;
};
void relin_batch(pft_ctx* c, const std::vector<RelinIO>& io);
// Budget for the scratch of one batched key-switching call (inputs are tiled beyond it).
constexpr size_t kKsScratchBudget = (size_t)24 << 30;
// Scratch words of one key switch at level l.
inline size_t ks_scratch_words(const pft_ctx* c, int l) {
    const int E = l + c->k, beta = (l + c->alpha - 1) / c->alpha;
    return (size_t)(l + beta * E + 2 * E + 2 * l) * c->n;
}

// ---- fastText inference as a sequence of stages (Sec. 3.1) ---------------------------------
// One document in flight: its inputs, its working ciphertexts and its score.  A stage runs
// over any set of documents of one model, whatever their levels (3 <= l <= model level; a
// model encoded at level L serves level l through the first l limbs of its plaintexts).
struct FtDoc {
    const pft_ct* const* v = nullptr;  // model chunks (Fig. 3) or 1 (diagonal) input ciphertexts
    int l = 0;                          // level of the inputs
    std::vector<pft_ct> W;              // the n columns (Fig. 3) or Q (diagonal)
    std::vector<pft_ct*> work;          // ciphertexts the next rotate-and-sum step acts on
    pft_ct* score = nullptr;
    FtDoc() = default;
    FtDoc(const FtDoc&) = delete;
    FtDoc& operator=(const FtDoc&) = delete;
    ~FtDoc() {
        for (auto& x : W) dfree(x.ctx, x.data);
    }
};
enum FtStageKind { FT_BEGIN = 0, FT_ROT = 1, FT_MID = 2, FT_FINISH = 3 };
struct FtStage {
    int kind;
    u32 g;  // Galois element of FT_ROT
};
// Stages of one inference with model M, in order.
std::vector<FtStage> ft_program(pft_ctx* c, const pft_ft_model* M);
// Checks one document's inputs against the model and the keys its program needs.
void ft_check_doc(pft_ctx* c, const pft_ft_model* M, const pft_ct* const* v, int n_chunks);
// Runs one stage for every document of `docs` (all at the same stage of the same model).
void ft_stage(pft_ctx* c, const pft_ft_model* M, const FtStage& st, const std::vector<FtDoc*>& docs);
