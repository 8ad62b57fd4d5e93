// Persistent job queue (host side): elementwise HADD / subtraction / HMULPLAIN (Sec. 2.3) over
// ciphertexts of any rings and levels, executed by one persistent launch (k_job_queue).
//
// The call checks the jobs in list order against their contexts (a handle written by an
// earlier job is read in the state that job leaves it in), sizes the outputs, checks that each
// buffer a job shares with an earlier job is covered by its chain of `after` links (so tiles
// that run concurrently never touch the same words unordered), numbers the tiles in list order
// and uploads the descriptors; the device counts finished tiles per job.
#include <map>
#include <vector>

#include "evaluator.h"

namespace {

// jobs reached from j through `after` links (j itself excluded)
bool reaches(const pft_job* jobs, int j, int target) {
    for (int k = jobs[j].after; k >= 0; k = jobs[k].after)
        if (k == target) return true;
    return false;
}

}  // namespace

extern "C" int pft_run_jobs(pft_ctx* c, const pft_job* jobs, int n_jobs, double wait_timeout_s) {
    return guard(c, [&] {
        NEED(c && n_jobs >= 0 && (n_jobs == 0 || jobs), PFT_ERR_ARG, "bad arguments");
        NEED(wait_timeout_s > 0 && wait_timeout_s <= 10, PFT_ERR_ARG, "wait_timeout_s must lie in (0, 10]");
        if (n_jobs == 0) return;
        // Jobs are checked in list order.  A handle written by an earlier job of the list is
        // read in the state that job leaves it in (context, level, scale); buffer addresses are
        // taken when a job is checked, so an output may not be reallocated once an earlier job
        // refers to its buffer.
        struct State {
            pft_ctx* ctx;
            int level;
            double scale;
        };
        std::map<const pft_ct*, State> produced;
        auto state = [&](const pft_ct* h) -> State {
            auto it = produced.find(h);
            if (it != produced.end()) return it->second;
            check_ct(h);
            return State{h->ctx, h->level, h->scale};
        };
        std::map<const u64*, std::vector<std::pair<int, bool>>> touched;  // buffer -> (job, writes)
        std::vector<QJob> q(n_jobs);
        std::vector<double> scales(n_jobs);
        long long tiles = 0;
        double bytes = 0;
        for (int j = 0; j < n_jobs; j++) {
            const pft_job& J = jobs[j];
            const std::string at = "job " + std::to_string(j) + ": ";
            NEED(J.op == PFT_JOB_ADD || J.op == PFT_JOB_SUB || J.op == PFT_JOB_MUL_PLAIN, PFT_ERR_ARG, at + "unknown op");
            NEED(J.a && J.out, PFT_ERR_ARG, at + "null operand or output");
            NEED(J.after >= -1 && J.after < j, PFT_ERR_ARG, at + "after must name an earlier job or be -1");
            const State A = state(J.a);
            pft_ctx* jc = A.ctx;
            NEED(jc->stream == c->stream, PFT_ERR_ARG, at + "its context must use the launching context's stream");
            State O{jc, A.level, A.scale};
            const u64* in2 = nullptr;
            if (J.op == PFT_JOB_MUL_PLAIN) {
                check_pt(J.p);
                NEED(J.p->ctx == jc, PFT_ERR_ARG, at + "plaintext from another context");
                NEED(J.p->level >= A.level, PFT_ERR_LEVEL_MISMATCH, at + "plaintext below the ciphertext's level");
                O.scale = A.scale * J.p->scale;
                in2 = J.p->data;
            } else {
                NEED(J.b, PFT_ERR_ARG, at + "null operand");
                const State Bs = state(J.b);
                NEED(Bs.ctx == jc, PFT_ERR_ARG, at + "operands from different contexts");
                NEED(Bs.level == A.level, PFT_ERR_LEVEL_MISMATCH, at + "operands at different levels");
                NEED(Bs.scale == A.scale, PFT_ERR_SCALE_MISMATCH, at + "operands at different scales");
                in2 = J.b->data;
            }
            const auto po = produced.find(J.out);
            NEED((po != produced.end() ? po->second.ctx : J.out->ctx) == jc || !J.out->ctx, PFT_ERR_ARG,
                 at + "output from another context");
            if (J.out->cap < (size_t)2 * O.level * jc->n)
                NEED(!J.out->data || !touched.count(J.out->data), PFT_ERR_ARG,
                     at + "an output that must grow holds a buffer an earlier job refers to");
            J.out->ctx = jc;
            ensure_ct(jc, J.out, O.level);
            produced[J.out] = O;
            scales[j] = O.scale;
            // hazards: every earlier job touching one of these buffers, when either side writes,
            // must be reachable through `after`
            const std::pair<const u64*, bool> mine[3] = {{J.a->data, false}, {in2, false}, {J.out->data, true}};
            for (const auto& m : mine) {
                auto it = touched.find(m.first);
                if (it == touched.end()) continue;
                for (const auto& t : it->second)
                    NEED(!(t.second || m.second) || reaches(jobs, j, t.first), PFT_ERR_ARG,
                         "job " + std::to_string(j) + " shares a buffer with job " + std::to_string(t.first) +
                             " without depending on it (after)");
            }
            for (const auto& m : mine) touched[m.first].push_back({j, m.second});
            QJob& D = q[j];
            D.a = J.a->data;
            D.b = in2;
            D.out = J.out->data;
            D.primes = jc->tabs.primes;
            D.wait_flag = J.wait_flag;
            D.wait_value = J.wait_value;
            D.op = J.op;
            D.logn = jc->logn;
            D.level = O.level;
            D.after = J.after;
            D.ntiles = 2 * D.level * (jc->n / queue_chunk(jc->logn));
            D.tile0 = tiles;
            tiles += D.ntiles;
            bytes += (double)D.level * jc->n * 8 * (J.op == PFT_JOB_MUL_PLAIN ? 5 : 6);
        }
        Scratch dq(c, q.size() * sizeof(QJob));
        Scratch cnt(c, 8 + 4 * (size_t)n_jobs);
        PFT_CUDA(cudaMemsetAsync(cnt.p, 0, 8 + 4 * (size_t)n_jobs, c->stream));
        job_queue(upload(c, dq, q), n_jobs, tiles, cnt.u(), (long long)(wait_timeout_s * 1e9), bytes, c->stream);
        for (int j = 0; j < n_jobs; j++) jobs[j].out->scale = scales[j];
    });
}
