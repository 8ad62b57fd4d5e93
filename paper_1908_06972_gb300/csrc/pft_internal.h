// Internal declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/privft.h"

typedef uint64_t u64;
typedef uint32_t u32;
typedef int64_t i64;

namespace pft {

constexpr int kMaxPrimes = 68;   // L + k
constexpr int kMaxLimbs = 60;    // L
constexpr int kMaxSpecial = 8;   // k
constexpr int kMaxAlpha = 8;     // primes per digit
constexpr int kMaxSet = 256;     // polynomials per launch descriptor
constexpr int kMaxBconv = 96;    // basis-conversion jobs per launch (by-value parameters)

// Per-prime constants on the device.
//   Barrett (single 64-bit word): s = bitlen(q) - 1, mu = floor(2^(64+s) / q);
//   valid for inputs x < 2^(64+s) = 2^(63+bitlen).
struct DPrime {
    u64 q;
    u64 mu;
    u64 r64;   // 2^64 mod q
    u64 mneg;  // -q^-1 mod 2^64 (Montgomery reduction)
    u32 s;
    u32 pad;
};

// A polynomial in a launch: `nlimbs` consecutive limbs of N words at `ptr`.
// Limb r is reduced modulo prime index  (r < split ? first + r : base2 + r - split).
struct PolyRef {
    u64* ptr;
    uint16_t nlimbs;
    uint16_t first;
    uint16_t split;
    uint16_t base2;
};
struct PolySet {
    int count;
    int max_limbs;
    PolyRef p[kMaxSet];
};

__host__ __device__ inline int prime_of(const PolyRef& r, int limb) {
    return limb < r.split ? r.first + limb : r.base2 + (limb - r.split);
}

// Device tables of one context (all device pointers).
struct DevTables {
    int logn;
    int n;
    DPrime* primes;        // [P]
    ulonglong2* fwd;       // [P][N] (psi^brv(i), shoup)
    ulonglong2* inv;       // [P][N] (psi^-brv(i), shoup)
    ulonglong2* ninv;      // [P] (N^-1, shoup)
    ulonglong2* inv1ninv;  // [P] (psi^-brv(1) N^-1, shoup)
    // N = 2^16 only (else null): the twiddles of stages 12..15 of fwd / inv in lane-major order,
    // [P][256 rows u][15 slots][16 lanes w]: slot 2^k - 1 + j, lane w holds entry
    // 2^(12+k) + u 2^(4+k) + w 2^k + j of the natural table
    ulonglong2* fwd_rows;
    ulonglong2* inv_rows;
    int bconv_tc;          // basis conversion of four source primes on the tensor cores (1, opt-in:
                           // environment PFT_BCONV=tc at context creation) or the integer pipes (0)
    // Memory order of the N = 2^16 two-pass transforms (environment PFT_NTT_ORDER at context
    // creation: bit 0 = the second pass visits (polynomial, limb) in reverse, so its first CTAs
    // read what the first pass wrote last, still in L2; bit 1 = the row twiddles are loaded with
    // an L2 evict-last policy, so the streaming data evict them less; bit 2 = the fused ModDown
    // pass asks L2 for its epilogue operands at the start of each CTA: faster while the epilogue
    // read one 8-byte word per row, slower since it reads 16 bytes four rows ahead).  Default 3.
    int ntt_order;
    int ntt_variant;       // N = 2^16 transform: 0 two-pass (3 CTAs/SM), 1 two-pass (4 CTAs/SM),
                           // 2 one-launch cluster, 3 generic staged passes
    // Transform plan per launch size (bucket of the launch's total limbs: <= 64, <= 512,
    // larger), chosen by the autotuner; kind < 0: the fixed variant above.
    struct Plan {
        int8_t kind;   // -1 none, 0 two-pass 3 CTAs/SM, 1 two-pass 4 CTAs/SM, 2 cluster, 3 generic
        int8_t npass;  // generic: passes, first (largest stride) first
        int8_t S[3];   // generic: stages per pass
        int16_t C[3];  // generic: sub-transforms per CTA of each pass
    } plan[3];
};
constexpr int kNttVariants = 4;
constexpr int kNttBuckets = 3;
inline int ntt_bucket(double limbs) { return limbs <= 64 ? 0 : limbs <= 512 ? 1 : 2; }
// Plans before any search: the fixed variant, except that launches of more than 512 limbs at
// N = 2^16 take the two-pass kernels at 4 CTAs per SM (the search's choice for that bucket on a
// GB300: 324.5 against 313.8 mult+relin/s in the benchmark step).
inline void default_plans(DevTables& t) {
    for (int b = 0; b < kNttBuckets; b++) t.plan[b].kind = -1;
    if (t.logn == 16) t.plan[2].kind = 1;
}

struct Error {
    int code;
    std::string msg;
};
[[noreturn]] void fail(int code, const std::string& msg);
void check_cuda(cudaError_t e, const char* what);
#define PFT_CUDA(x) ::pft::check_cuda((x), #x)
// True on the first call for (key, current device), false afterwards: kernel attributes
// (shared-memory size, carveout) are per device, so each device sets them once.
bool first_on_device(const void* key);
#define PFT_LAUNCH_CHECK(what) ::pft::check_cuda(cudaGetLastError(), what)

// Launch accounting: every kernel launch is counted; launches whose name starts
// with the prefix given to pft_prof_start are bracketed by CUDA events on their stream.
// `work` is the launch's algorithmic work (butterflies for transforms, bytes for the
// memory-bound kernels), summed over the timed launches.
void prof_begin(const char* name, cudaStream_t st, double work);
void prof_end(const char* name, cudaStream_t st);
struct ProfScope {
    const char* n;
    cudaStream_t s;
    ProfScope(const char* n_, cudaStream_t s_, double w) : n(n_), s(s_) { prof_begin(n, s, w); }
    ~ProfScope() { prof_end(n, s); }
};
#define PFT_PROF(name, st, work) ::pft::ProfScope pft_prof_scope_(name, st, work)
inline double set_limbs(const PolySet& s) {
    double t = 0;
    for (int i = 0; i < s.count; i++) t += s.p[i].nlimbs;
    return t;
}

// ---- kernels (launchers) ------------------------------------------------------------
// Negacyclic transform of every limb of every polynomial of `out` (input from `in`,
// which may be the same set).
void ntt_forward(const DevTables& t, const PolySet& in, const PolySet& out, cudaStream_t st);
// The ModDown epilogue applied by the last forward pass: out = (x + c - NTT(io)) s (+ acc; a null
// acc pointer: none), per-limb constants {c, s, s'} at consts[3 limb].
struct NttEpi {
    PolySet x, acc, out;
    const u64* consts;
};
// Forward transform of io (in place) fused with the epilogue; false (nothing launched) where
// the ring or the transform variant has no fused kernel.
bool ntt_forward_epilogue(const DevTables& t, const PolySet& io, const NttEpi& e, cudaStream_t st);
// N times the inverse transform (no N^-1 at the last stage, values in [0, 4q)) for consumers
// that scale their input anyway; false (nothing launched) where the ring or the transform
// variant has no such kernel.
bool ntt_inverse_unscaled(const DevTables& t, const PolySet& in, const PolySet& out, cudaStream_t st);
// Butterflies per second of the transform's (exact-path) butterfly arithmetic on register data
// only: the arithmetic ceiling the transforms are measured against (synchronous).
double bfly_ceiling(const DevTables& t, cudaStream_t st);
// Measured issue rates (operations per second, whole GPU) of the 32-bit multiply forms the
// butterflies use: low-word multiply-add, high-word multiply, widening multiply (synchronous).
void mul_rates(cudaStream_t st, double* lo, double* hi, double* wide);
void ntt_inverse(const DevTables& t, const PolySet& in, const PolySet& out, cudaStream_t st);
// The transform plans the autotuner searches for this ring degree (generic plans have S[], C[]),
// with their names; plan_supported: the plan's kernels exist for this ring.
int ntt_candidates(int logn, DevTables::Plan* out, const char** names, int cap);

enum class EwOp { Add, Sub, Mul, Neg, Copy };
// out[i] = a[i] (op) b[i] per limb (b ignored for Neg/Copy).
void ew_binary(const DevTables& t, EwOp op, const PolySet& a, const PolySet& b, const PolySet& out, cudaStream_t st);
// HMUL tensor: a, b refs point at ciphertexts [2][l][N]; d refs at [3][l][N] (nlimbs = l).
void ew_tensor(const DevTables& t, const PolySet& a, const PolySet& b, const PolySet& d, cudaStream_t st);
// O[p] = sum_{k<K} A[p K + k] * B[(shared ? 0 : p K) + k]; device pointer tables; l limbs each.
void ew_dot(const DevTables& t, const u64* const* A, const u64* const* B, u64* const* O, int n_out, int K,
            bool b_shared, int l, cudaStream_t st);
// out = acc + ((x + c) - y) * s per limb, consts_dev[3 limb + {0,1,2}] = {c, s, s_shoup};
// y may be null (taken as 0), acc may be null.
// out[p] (+)= sum_k a (x) b over K pairs (tables in device memory; see poly.cu)
void ew_tensor_dot(const DevTables& t, const u64* const* A, const u64* const* B, u64* const* O, int n_out, int K,
                   int l, bool accumulate, cudaStream_t st);
void sub_scale(const DevTables& t, const PolySet& x, const PolySet* y, const PolySet* acc, const PolySet& out,
               const u64* consts_dev, cudaStream_t st);
// Galois automorphism X -> X^g in the evaluation layout.
void automorph(const DevTables& t, const PolySet& in, const PolySet& out, u64 g, cudaStream_t st);

// Fast basis conversion job: from ns source limbs (primes src_p0 ..) to rows
// [0, nrows) \ [skip_lo, skip_hi) of dst; target prime of row m: m < split ? m : base2 + m - split.
struct BconvJob {
    const u64* src;
    u64* dst;
    const u64* table;  // [ns]{qhat_inv, shoup} then [targets][ns] qhat mod target
    // four source primes only, or null: the byte planes of the conversion constants for the
    // tensor-core form, [targets][8 byte planes b][kBconvTcStride u32] of bf16 pairs: entry
    // k = 8 i + a is byte b of (qhat_i mod t_m) 2^(8a) mod t_m (b, a < 8, i < 4)
    const uint32_t* tc;
    int ns, src_p0, nrows, skip_lo, skip_hi, split, base2, pad;
};
constexpr int kBconvTcStride = 20;  // u32 words per (target, byte plane) row: 16 of data + 4 of padding
void bconv(const DevTables& t, const BconvJob* jobs_host, int n_jobs, cudaStream_t st);  // jobs: host array
// Byte-plane table of the tensor-core conversion for one job: c[m][i] = qhat_i mod t_m (plain
// form) for nt targets of primes tp[m] and 4 sources; returns [nt][8][kBconvTcStride] u32.
std::vector<uint32_t> bconv_tc_table(const std::vector<u64>& c, const std::vector<u64>& tp, int nt);

// Key inner product: u[b][pol][m] = sum_j ext[b][j][m] * key[j][pol][row(m)] over B inputs at
// any levels in one launch (the key is read once for all);
// input b has level l, ext [beta(l)][l+k][N], u [2][l+k][N].
struct KsDesc {
    const u64* ext;
    u64* u;
    const u64* d;  // the input in evaluation form: rows of digit j are read here (ext's copies
                   // of them are not written); null: ext holds them
    int l;
    int pad;
};
constexpr int kMaxKs = 128;  // inputs per launch (by-value parameters)
// A switching key as the inner product reads it: [beta][2 (b, a)][L+k][N] in evaluation form,
// or, compressed, only the b rows [beta][L+k][N] with a regenerated from the ChaCha20 stream
// (seed words, domain DOM_KSK_A_EVAL, object = key id, sub = 256 j + row), entry i of row r
// = the uniform residue of word pair i, already in evaluation form.
constexpr u32 kDomKskAEval = 11;
struct KeyRef {
    const u64* ptr;
    // uncompressed keys: the same words in Montgomery form split into 30-bit halves,
    // (k 2^64 mod p) = k1 2^30 + k0 stored as k0 | k1 << 32 (the key inner product's operand)
    const u64* mont;
    u32 id;
    int compressed;
    u32 seedw[8];
};
void ks_inner_multi(const DevTables& t, const KsDesc* descs_host, int B, const KeyRef& key, int L, int k, int alpha,
                    cudaStream_t st);
// Whether a kernel's bounded wait has expired since the last reset (reads a device flag).
int wait_timeout_flag(bool reset, cudaStream_t st);
// Persistent job queue: elementwise jobs over ciphertexts of any rings and levels in one launch.
// A job is cut into tiles (one chunk of one limb of one polynomial); resident CTAs claim tiles in
// order from a counter.  A job starts only after job `after` (an earlier index, or -1) has
// finished all its tiles and, when wait_flag is set, once *wait_flag >= wait_value; both waits
// are bounded by timeout_ns of %globaltimer, after which the CTA raises the sticky timeout flag
// (read by wait_timeout_flag), skips the tile and still counts it as done.
enum QOp : int { kQAdd = 0, kQSub = 1, kQMulPlain = 2 };
struct QJob {
    const u64* a;          // [2][level][N]
    const u64* b;          // [2][level][N] (add, sub) or [>= level][N] (plaintext)
    u64* out;              // [2][level][N]
    const DPrime* primes;  // the ring's prime table
    const u32* wait_flag;  // device word or null
    u32 wait_value;
    int op, logn, level, after, ntiles;
    long long tile0;       // first tile of the job in the queue's order
};
__host__ __device__ inline int queue_chunk(int logn) { return logn >= 11 ? 2048 : 1 << logn; }  // per tile
void job_queue(const QJob* jobs_dev, int n_jobs, long long total_tiles, u64* counters_dev, long long timeout_ns,
               double bytes, cudaStream_t st);
// Launches a wait that cannot complete, bounded by `polls` polls (it raises the flag).
void wait_selftest(long long polls, cudaStream_t st);
// r = (last + h) mod p, h = floor(p/2), p = prime nlimbs(out); limb k of out = (r - h) mod q_k.
void rescale_bcast(const DevTables& t, const PolySet& last, const PolySet& out, cudaStream_t st);

// Sampling (ChaCha20 streams, nonce (dom, obj, sub)).
void sample_uniform(const DevTables& t, const u64 seed[4], u32 dom, u32 obj, u32 sub_base, const PolySet& out,
                    cudaStream_t st);  // sub = sub_base + prime index of the limb
void sample_small(const DevTables& t, const u64 seed[4], u32 dom, u32 obj, u32 sub, int kind, const u32* cdt,
                  int nt, i64* out_dev, cudaStream_t st);  // kind 0 = ternary, 1 = Gaussian
void reduce_signed(const DevTables& t, const i64* x_dev, const PolySet& out, cudaStream_t st);
// out = in mod q per limb, for words of any 64-bit value (e.g. exact integer sums of residues)
void reduce_words(const DevTables& t, const PolySet& in, const PolySet& out, cudaStream_t st);
// out = (in 2^64 mod q) split into 30-bit halves, k0 | k1 << 32 (canonical residues in)
void mont_split(const DevTables& t, const PolySet& in, const PolySet& out, cudaStream_t st);

// ---- host math (encode.cpp) -----------------------------------------------------------
std::vector<u64> gen_primes(int logn, int bits, int count, const std::vector<u64>& exclude);
std::vector<u32> gauss_cdt(double sigma, int* tail);
u64 mulmod_host(u64 a, u64 b, u64 q);
u64 powmod_host(u64 a, u64 e, u64 q);
u64 invmod_host(u64 a, u64 q);
u64 root_2n_host(u64 q, int logn);
// Encode slots (re, im interleaved, n_slots) -> rounded integer coefficients.
bool encode_slots(int logn, const double* re_im, int n_slots, double scale, std::vector<i64>& coeffs);
// Decode: CRT-centered coefficients as doubles -> slots.
void decode_coeffs(int logn, const std::vector<double>& coeffs, double scale, double* re_im, int n_slots);
// CRT of [l][N] residues to centered doubles.
void crt_to_double(const std::vector<u64>& primes, const u64* rows, int n, std::vector<double>& out);

}  // namespace pft
