// Request server for encrypted fastText inference (Sec. 3.1) with continuous batching.
//
// A request is one document: its input ciphertexts in coefficient form in host memory, a
// ring (one context with its keys and model resident on the device) and a level.  Every
// call of pft_server_step is one iteration:
//   1. retire requests whose score has reached host memory (completion time from a CUDA
//      event, so it does not depend on how often the caller polls);
//   2. admit waiting requests in arrival order while their device footprint fits the budget
//      (inputs copied through page-locked staging and taken to evaluation form in one
//      batched call per ring);
//   3. advance every admitted request by one stage of its inference sequence: requests of a
//      ring at the same stage form one batched call, so a request admitted now runs its
//      column products while older ones run their rotate-and-sum steps;
//   4. queue the export of finished scores and return once the iteration before this one
//      has completed on the device, so the host prepares the next iteration while the GPU
//      runs this one.
// Each ring's work goes to its context's stream, so rings of different sizes run
// concurrently.  Results do not depend on the mix: every operation computes each
// ciphertext independently of the others in its batch.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>

#include "evaluator.h"

namespace {

struct PinnedPool {
    std::vector<std::pair<size_t, void*>> free_;
    void* get(size_t bytes) {
        size_t best = free_.size();
        for (size_t i = 0; i < free_.size(); i++)
            if (free_[i].first >= bytes && (best == free_.size() || free_[i].first < free_[best].first)) best = i;
        if (best < free_.size()) {
            void* p = free_[best].second;
            free_.erase(free_.begin() + best);
            used_[p] = sizes_[p];
            return p;
        }
        void* p = nullptr;
        PFT_CUDA(cudaHostAlloc(&p, bytes, cudaHostAllocDefault));
        sizes_[p] = bytes;
        used_[p] = bytes;
        return p;
    }
    void put(void* p) {
        if (!p) return;
        free_.push_back({sizes_[p], p});
        used_.erase(p);
    }
    ~PinnedPool() {
        for (auto& f : free_) cudaFreeHost(f.second);
        for (auto& u : used_) cudaFreeHost(u.first);
    }
    std::map<void*, size_t> sizes_, used_;
};

struct Ring {
    pft_ctx* ctx = nullptr;
    const pft_ft_model* M = nullptr;
    std::vector<FtStage> prog;
    int chunks = 1;
    cudaEvent_t t0 = nullptr;  // origin of this ring's device timeline
    double t0_s = 0;           // host time of t0 on the server clock
    cudaEvent_t iter[2] = {nullptr, nullptr};
    bool iter_used[2] = {false, false};
};

struct Request {
    uint64_t tag = 0;
    int ring = 0, level = 0;
    double scale = 1, t_submit = 0;
    const uint64_t* in = nullptr;
    uint64_t* out = nullptr;
    size_t bytes = 0, in_words = 0, out_words = 0;
    std::vector<pft_ct> v;
    std::vector<const pft_ct*> vp;
    pft_ct score;
    FtDoc doc;
    int stage = 0;
    void* stage_in = nullptr;   // page-locked copy of the inputs
    void* stage_out = nullptr;  // page-locked landing buffer of the score
    cudaEvent_t done = nullptr;
    double out_scale = 0;
};

}  // namespace

struct pft_server {
    std::vector<Ring> rings;
    size_t budget = 0, used = 0, peak = 0;
    long iterations = 0;
    int max_active = 0;
    std::deque<std::unique_ptr<Request>> waiting;
    std::vector<std::unique_ptr<Request>> active, exporting;
    std::deque<pft_server_done> done;
    long n_done = 0;
    PinnedPool pinned;
    std::chrono::steady_clock::time_point t0;
    std::string err;
    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

static thread_local std::string g_create_err;  // error text of the last failed pft_server_create

template <class F>
static int sguard(pft_server* s, F f) {
    try {
        f();
        return PFT_OK;
    } catch (const Error& e) {
        if (s) s->err = e.msg;
        return e.code;
    } catch (const std::bad_alloc&) {
        if (s) s->err = "host out of memory";
        return PFT_ERR_OOM;
    } catch (const std::exception& e) {
        if (s) s->err = e.what();
        return PFT_ERR_ARG;
    }
}

// Device bytes a request holds while admitted: its input ciphertexts, the working
// ciphertexts of its sequence (the n columns; or Q, the n - 1 rotated copies of each input
// and the score of the diagonal variant), its score and the export copy, all at its level.
static size_t footprint(const Ring& r, int level) {
    const size_t ct = (size_t)2 * level * r.ctx->n * 8;
    const int cols = r.M->n;
    return (r.M->variant == 0 ? (size_t)(r.chunks + cols + 2) : (size_t)(r.chunks * cols + 3)) * ct;
}

static void release_device(pft_ctx* c, Request* q) {
    for (auto& x : q->v) {
        dfree(c, x.data);
        x.data = nullptr;
    }
    dfree(c, q->score.data);
    q->score.data = nullptr;
    for (auto& x : q->doc.W) dfree(c, x.data);
    q->doc.W.clear();
}

static void retire(pft_server* s) {
    for (size_t i = 0; i < s->exporting.size();) {
        Request* q = s->exporting[i].get();
        const cudaError_t e = cudaEventQuery(q->done);
        if (e == cudaErrorNotReady) {
            i++;
            continue;
        }
        PFT_CUDA(e);
        const Ring& r = s->rings[q->ring];
        float ms = 0;
        PFT_CUDA(cudaEventElapsedTime(&ms, r.t0, q->done));
        std::memcpy(q->out, q->stage_out, q->out_words * 8);
        pft_server_done d;
        d.tag = q->tag;
        d.ring = q->ring;
        d.level = q->level - 2;
        d.scale = q->out_scale;
        d.t_submit = q->t_submit;
        d.t_done = r.t0_s + ms * 1e-3;
        s->done.push_back(d);
        s->n_done++;
        s->pinned.put(q->stage_in);
        s->pinned.put(q->stage_out);
        cudaEventDestroy(q->done);
        q->done = nullptr;
        s->exporting.erase(s->exporting.begin() + i);
    }
}

static void admit(pft_server* s) {
    std::vector<std::vector<Request*>> fresh(s->rings.size());
    while (!s->waiting.empty()) {
        Request* q = s->waiting.front().get();
        if (s->budget && s->used + q->bytes > s->budget) break;  // arrival order: no overtaking
        s->active.push_back(std::move(s->waiting.front()));  // held here even if a step below fails
        s->waiting.pop_front();
        s->used += q->bytes;
        s->peak = std::max(s->peak, s->used);
        const Ring& r = s->rings[q->ring];
        pft_ctx* c = r.ctx;
        const size_t ctw = (size_t)2 * q->level * c->n;
        q->stage_in = s->pinned.get(q->in_words * 8);
        q->stage_out = s->pinned.get(q->out_words * 8);
        std::memcpy(q->stage_in, q->in, q->in_words * 8);
        q->v.resize(r.chunks);
        for (int i = 0; i < r.chunks; i++) {
            pft_ct& x = q->v[i];
            x.ctx = c;
            ensure_ct(c, &x, q->level);
            x.scale = q->scale;
            PFT_CUDA(cudaMemcpyAsync(x.data, (const u64*)q->stage_in + i * ctw, ctw * 8, cudaMemcpyHostToDevice,
                                     c->stream));
            q->vp.push_back(&x);
        }
        q->score.ctx = c;
        q->doc.v = q->vp.data();
        q->doc.l = q->level;
        q->doc.score = &q->score;
        q->stage = 0;
        fresh[q->ring].push_back(q);
    }
    for (size_t ri = 0; ri < s->rings.size(); ri++) {
        if (fresh[ri].empty()) continue;
        pft_ctx* c = s->rings[ri].ctx;
        std::vector<PolyRef> r;
        for (Request* q : fresh[ri])
            for (auto& x : q->v)
                for (int pol = 0; pol < 2; pol++) r.push_back(cpoly(x.data, q->level, c->n, pol));
        ntt_fwd(c, r, r);
    }
}

static void finish(pft_server* s, Request* q) {
    const Ring& r = s->rings[q->ring];
    pft_ctx* c = r.ctx;
    const int l = q->score.level;
    NEED(l == q->level - 2 && (size_t)2 * l * c->n == q->out_words, PFT_ERR_ARG, "internal: score level");
    {
        Scratch t(c, q->out_words * 8);
        std::vector<PolyRef> in{cpoly(q->score.data, l, c->n, 0), cpoly(q->score.data, l, c->n, 1)};
        std::vector<PolyRef> o{cpoly(t.u(), l, c->n, 0), cpoly(t.u(), l, c->n, 1)};
        ntt_inv(c, in, o);
        PFT_CUDA(cudaMemcpyAsync(q->stage_out, t.p, q->out_words * 8, cudaMemcpyDeviceToHost, c->stream));
    }
    q->out_scale = q->score.scale;
    PFT_CUDA(cudaEventCreate(&q->done));
    PFT_CUDA(cudaEventRecord(q->done, c->stream));
    release_device(c, q);  // stream-ordered: the copies above read the buffers first
    s->used -= q->bytes;
}

static void run_stages(pft_server* s) {
    for (size_t ri = 0; ri < s->rings.size(); ri++) {
        Ring& r = s->rings[ri];
        std::map<int, std::vector<Request*>, std::greater<int>> by_stage;
        for (auto& q : s->active)
            if (q->ring == (int)ri) by_stage[q->stage].push_back(q.get());
        for (auto& kv : by_stage) {
            std::vector<FtDoc*> docs;
            for (Request* q : kv.second) docs.push_back(&q->doc);
            ft_stage(r.ctx, r.M, r.prog[kv.first], docs);
            for (Request* q : kv.second) q->stage++;
        }
    }
    for (size_t i = 0; i < s->active.size();) {
        Request* q = s->active[i].get();
        if (q->stage == (int)s->rings[q->ring].prog.size()) {
            finish(s, q);
            s->exporting.push_back(std::move(s->active[i]));
            s->active.erase(s->active.begin() + i);
        } else {
            i++;
        }
    }
}

static void step(pft_server* s) {
    retire(s);
    admit(s);
    s->max_active = std::max<int>(s->max_active, (int)s->active.size());
    if (s->active.empty()) return;
    run_stages(s);
    const int cur = (int)(s->iterations & 1), prev = cur ^ 1;
    for (Ring& r : s->rings) {
        PFT_CUDA(cudaEventRecord(r.iter[cur], r.ctx->stream));
        r.iter_used[cur] = true;
    }
    s->iterations++;
    for (Ring& r : s->rings)
        if (r.iter_used[prev]) PFT_CUDA(cudaEventSynchronize(r.iter[prev]));
}

extern "C" {

int pft_server_create(pft_ctx* const* ctxs, const pft_ft_model* const* models, int n_rings, size_t budget_bytes,
                      pft_server** out) {
    if (!out) return PFT_ERR_ARG;
    *out = nullptr;
    std::unique_ptr<pft_server> s(new pft_server());
    const int rc = sguard(s.get(), [&] {
        NEED(ctxs && models && n_rings >= 1, PFT_ERR_ARG, "bad arguments");
        s->t0 = std::chrono::steady_clock::now();
        s->budget = budget_bytes;
        for (int i = 0; i < n_rings; i++) {
            NEED(ctxs[i] && models[i] && models[i]->ctx == ctxs[i], PFT_ERR_ARG,
                 "ring " + std::to_string(i) + ": model from another context");
            for (int j = 0; j < i; j++)
                NEED(ctxs[j] != ctxs[i], PFT_ERR_ARG, "each ring needs a context of its own");
            Ring r;
            r.ctx = ctxs[i];
            r.M = models[i];
            r.prog = ft_program(r.ctx, r.M);
            r.chunks = r.M->chunks;
            for (const FtStage& st : r.prog)
                if (st.kind == FT_ROT)
                    NEED(r.ctx->keys.count(st.g), PFT_ERR_NO_KEY, "ring " + std::to_string(i) + ": missing rotation key");
            PFT_CUDA(cudaEventCreate(&r.t0));
            PFT_CUDA(cudaEventCreate(&r.iter[0]));
            PFT_CUDA(cudaEventCreate(&r.iter[1]));
            s->rings.push_back(r);
            Ring& rr = s->rings.back();
            PFT_CUDA(cudaEventRecord(rr.t0, rr.ctx->stream));
            PFT_CUDA(cudaEventSynchronize(rr.t0));
            rr.t0_s = s->now();
        }
    });
    if (rc != PFT_OK) {
        g_create_err = s->err;
        for (Ring& r : s->rings) {
            if (r.t0) cudaEventDestroy(r.t0);
            if (r.iter[0]) cudaEventDestroy(r.iter[0]);
            if (r.iter[1]) cudaEventDestroy(r.iter[1]);
        }
        return rc;
    }
    *out = s.release();
    return PFT_OK;
}

int pft_server_destroy(pft_server* s) {
    if (!s) return PFT_OK;
    for (Ring& r : s->rings) cudaStreamSynchronize(r.ctx->stream);
    for (auto& q : s->active) release_device(s->rings[q->ring].ctx, q.get());
    for (auto& q : s->exporting)
        if (q->done) cudaEventDestroy(q->done);
    for (Ring& r : s->rings) {
        cudaStreamSynchronize(r.ctx->stream);
        cudaEventDestroy(r.t0);
        cudaEventDestroy(r.iter[0]);
        cudaEventDestroy(r.iter[1]);
    }
    delete s;
    return PFT_OK;
}

const char* pft_server_last_error(const pft_server* s) { return s ? s->err.c_str() : g_create_err.c_str(); }

int pft_server_submit(pft_server* s, int ring, const uint64_t* in, int level, double scale, uint64_t* out,
                      uint64_t tag) {
    if (!s) return PFT_ERR_ARG;
    return sguard(s, [&] {
        NEED(ring >= 0 && ring < (int)s->rings.size(), PFT_ERR_ARG, "no such ring");
        NEED(in && out, PFT_ERR_ARG, "null buffer");
        const Ring& r = s->rings[ring];
        NEED(level >= 3 && level <= r.M->level, PFT_ERR_LEVEL_MISMATCH,
             "level must lie in 3.." + std::to_string(r.M->level));
        NEED(scale > 0, PFT_ERR_ARG, "scale must be positive");
        std::unique_ptr<Request> q(new Request());
        q->tag = tag;
        q->ring = ring;
        q->level = level;
        q->scale = scale;
        q->in = in;
        q->out = out;
        q->bytes = footprint(r, level);
        q->in_words = (size_t)r.chunks * 2 * level * r.ctx->n;
        q->out_words = (size_t)2 * (level - 2) * r.ctx->n;
        NEED(!s->budget || q->bytes <= s->budget, PFT_ERR_OOM,
             "request needs " + std::to_string(q->bytes) + " bytes of device memory, the budget is " +
                 std::to_string(s->budget));
        q->t_submit = s->now();
        s->waiting.push_back(std::move(q));
    });
}

int pft_server_step(pft_server* s, int* n_pending) {
    if (!s) return PFT_ERR_ARG;
    return sguard(s, [&] {
        step(s);
        if (n_pending) *n_pending = (int)(s->waiting.size() + s->active.size() + s->exporting.size());
    });
}

int pft_server_drain(pft_server* s) {
    if (!s) return PFT_ERR_ARG;
    return sguard(s, [&] {
        while (!s->waiting.empty() || !s->active.empty()) step(s);
        for (Ring& r : s->rings) PFT_CUDA(cudaStreamSynchronize(r.ctx->stream));
        retire(s);
        NEED(s->exporting.empty(), PFT_ERR_CUDA, "internal: export did not complete");
    });
}

int pft_server_poll(pft_server* s, pft_server_done* done, int max, int* n) {
    if (!s || !n || max < 0 || (max > 0 && !done)) return PFT_ERR_ARG;
    return sguard(s, [&] {
        retire(s);
        int k = 0;
        while (k < max && !s->done.empty()) {
            done[k++] = s->done.front();
            s->done.pop_front();
        }
        *n = k;
    });
}

int pft_server_clock(pft_server* s, double* t) {
    if (!s || !t) return PFT_ERR_ARG;
    *t = s->now();
    return PFT_OK;
}

int pft_server_get_stats(pft_server* s, pft_server_stats* st) {
    if (!s || !st) return PFT_ERR_ARG;
    st->waiting = (int)s->waiting.size();
    st->active = (int)s->active.size();
    st->exporting = (int)s->exporting.size();
    st->max_active = s->max_active;
    st->completed = s->n_done;
    st->iterations = s->iterations;
    st->bytes_in_use = s->used;
    st->peak_bytes = s->peak;
    st->budget = s->budget;
    return PFT_OK;
}

int pft_server_footprint(pft_server* s, int ring, int level, size_t* bytes) {
    if (!s || !bytes || ring < 0 || ring >= (int)s->rings.size() || level < 1) return PFT_ERR_ARG;
    *bytes = footprint(s->rings[ring], level);
    return PFT_OK;
}

}  // extern "C"
