/*
 * privft.h -- C ABI of the GB300 RNS-CKKS library behind encrypted fastText
 * (PrivFT, arXiv 1908.06972).
 *
 * Scheme (Sec. 2.3 of the paper): R_q = Z_q[X]/(X^N+1), q = q_0 q_1 ... q_{l-1}
 * a chain of word-sized NTT-friendly primes (here at most 60 bits each, so well
 * below 2^62), CKKS encoding of N/2 complex slots, KEYGEN/ENC/DEC, HADD, HMUL
 * (+ relinearisation), HADDPLAIN, HMULPLAIN, RESCALE (Eq. 1, Algorithm 3) and
 * ROTATE (Sec. 2.3 and the rotation discussion of Sec. 5.3).  The inference
 * entry point follows Sec. 3.1 (Fig. 3, Algorithm 2); the training entry points
 * follow Sec. 4.2 (Algorithm 5).  Beyond the paper: batched forms of every operation
 * over ciphertexts at mixed levels, hoisted rotations, CUDA-graph capture, seeded
 * compressed keys, rotation-light (diagonal) inference and training, a request
 * server with continuous batching, and a persistent job queue over rings of
 * different N.
 *
 * Conventions shared by every call
 *   - Every function returns an int status: PFT_OK (0) or a PFT_ERR_* code.
 *     pft_last_error(ctx) gives a text for the last failure on that context.
 *   - "level" l = number of RNS limbs a ciphertext/plaintext carries (1..L),
 *     as in the paper's q_l = prod_{i<=l} p_i.
 *   - Handles (pft_ctx, pft_ct, pft_pt, pft_ft_model) are created and destroyed
 *     by the library.  Their device memory comes from the allocator given at
 *     context creation (NULL -> cudaMallocAsync/cudaFreeAsync on the context's
 *     stream).
 *   - All device work is issued on the context stream (pft_set_stream; default
 *     the legacy default stream) and is asynchronous; calls that return host
 *     data (pft_decode, pft_ct_export, pft_pt_export) synchronise that stream.
 *   - An output handle may alias an input handle.
 *   - Device layout of a ciphertext: [2][l][N] uint64, limb-major, each limb in
 *     the evaluation ("NTT") domain: entry i of limb r holds a(psi_r^(2 brv(i)+1))
 *     mod q_r, brv the log2(N)-bit reversal, psi_r = x^((q_r-1)/2N) for the
 *     smallest quadratic non-residue x of q_r.  Export/import use COEFFICIENT
 *     form, canonical residues in [0, q_r).
 *   - Primes, when not given, follow the rule: for a bit size b, the candidates
 *     2^b - j*2N + 1, j = 1, 2, ..., that are prime, in that (descending) order;
 *     q_0 takes the first of its size, q_1..q_{L-1} the next ones of theirs, the
 *     special primes the next unused ones of theirs.
 *   - Randomness: a ChaCha20 (RFC 8439) counter-mode stream keyed by the
 *     256-bit seed, nonce (domain, object, sub); see the sampler notes at
 *     pft_keygen.
 */
#ifndef PRIVFT_H
#define PRIVFT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
enum {
    PFT_OK = 0,
    PFT_ERR_ARG = 1,            /* bad argument (NULL, size, range) */
    PFT_ERR_LEVEL_MISMATCH = 2, /* operands at different levels (Sec. 2.3: same level required) */
    PFT_ERR_SCALE_MISMATCH = 3, /* add of operands whose scales differ */
    PFT_ERR_NO_KEY = 4,         /* relinearisation / rotation key not generated */
    PFT_ERR_OOM = 5,            /* the allocator returned NULL */
    PFT_ERR_CUDA = 6,           /* a CUDA runtime call or launch failed */
    PFT_ERR_TIMEOUT = 7,        /* a bounded device wait expired */
    PFT_ERR_SECURITY = 8,       /* log2(QP) above the 128-bit bound without PFT_ALLOW_INSECURE */
    PFT_ERR_NOT_IMPLEMENTED = 9
};

/* ---- opaque handles ------------------------------------------------------ */
typedef struct pft_ctx pft_ctx;
typedef struct pft_ct pft_ct;             /* ciphertext (c0, c1) */
typedef struct pft_pt pft_pt;             /* plaintext mu */
typedef struct pft_ft_model pft_ft_model; /* packed fastText weights (H, O) */

/* Device allocator.  alloc(bytes, stream, user) returns device memory usable on
 * `stream` (NULL on failure); free(ptr, stream, user) releases it once the work
 * already queued on `stream` no longer needs it. */
typedef struct {
    void* (*alloc)(size_t bytes, void* stream, void* user);
    void (*free)(void* ptr, void* stream, void* user);
    void* user;
} pft_allocator;

#define PFT_ALLOW_INSECURE 1 /* pft_params.flags: accept log2(QP) above the 128-bit table */
/* pft_params.flags: seeded compressed switching keys.  Each key keeps only its b_j rows; a_j
 * is drawn uniformly in the evaluation domain from the ChaCha20 stream (seed, domain 11,
 * object = key id (0 relinearisation, g rotation), sub = 256 j + prime index), and the key
 * inner product regenerates it: key memory halves, the inner product trades key reads for
 * ChaCha20 blocks.  Keys differ from the uncompressed ones (a_j is another draw). */
#define PFT_COMPRESSED_KEYS 2

/* Encryption parameters (SETUP, Sec. 2.3 and Sec. 5.4).
 *   log_n        log2 N, 4..16
 *   n_limbs      L, number of ciphertext primes at the top level (1..60)
 *   n_special    k, special primes for key switching (1..8)
 *   alpha        primes per key-switching digit (1..8); beta = ceil(l/alpha) digits
 *   first_bits   bit size of q_0 (20..60)
 *   mid_bits     bit size of q_1..q_{L-1} (20..60)
 *   special_bits bit size of the special primes (20..60)
 *   primes       optional explicit chain [n_limbs + n_special] (q's then p's), or NULL
 *   scale        default encoding scale Delta = 2^rho
 *   seed         256-bit sampler key
 *   sigma        Gaussian standard deviation (the paper uses 3.2); tail cut at floor(6 sigma)
 *   flags        PFT_ALLOW_INSECURE | PFT_COMPRESSED_KEYS
 * Security table (max log2(QP), uniform ternary secret, 128-bit): N=2^10: 27,
 * 2^11: 54, 2^12: 109, 2^13: 218, 2^14: 438, 2^15: 881, 2^16: 1772. */
typedef struct {
    int log_n;
    int n_limbs;
    int n_special;
    int alpha;
    int first_bits;
    int mid_bits;
    int special_bits;
    const uint64_t* primes;
    double scale;
    uint64_t seed[4];
    double sigma;
    int flags;
} pft_params;

/* ---- context ------------------------------------------------------------- */
/* Create a context: primes, transform tables, basis-conversion tables on the
 * device.  `alloc` may be NULL.  Errors: ARG, SECURITY, OOM, CUDA. */
int pft_ctx_create(const pft_params* params, const pft_allocator* alloc, pft_ctx** out);
int pft_ctx_destroy(pft_ctx* ctx);
/* Set the cudaStream_t (passed as void*) on which all later work is queued. */
int pft_set_stream(pft_ctx* ctx, void* stream);
const char* pft_last_error(pft_ctx* ctx);
/* Chain info: N, L, k, alpha; primes_out (may be NULL) receives [L + k] primes. */
int pft_ctx_info(pft_ctx* ctx, int* n, int* n_limbs, int* n_special, int* alpha, uint64_t* primes_out);

/* ---- host-only utilities (no GPU needed) --------------------------------- */
/* First `count` primes of `bits` bits congruent to 1 mod 2^(log_n+1), by the rule
 * above, skipping the `n_exclude` values in `exclude`. */
int pft_gen_primes(int log_n, int bits, int count, const uint64_t* exclude, int n_exclude, uint64_t* out);
/* The 32-bit cumulative table of |X| used by the Gaussian sampler:
 * out[j] = floor(2^32 P(|X| <= j)), j < tail, for P(X=x) ~ exp(-x^2/(2 sigma^2))
 * on [-tail, tail], tail = floor(6 sigma).  Returns the number of entries via n_out. */
int pft_gauss_cdt(double sigma, uint32_t* out, int cap, int* n_out);

/* ---- launch accounting (diagnostics) --------------------------------------
 * pft_prof_start(prefix): from now on count every kernel launch of the library
 * and bracket each launch whose kernel name starts with `prefix` (e.g. "ntt",
 * "ks_inner", "bconv"; "" times none) with CUDA events on its stream.
 * pft_prof_stop: waits for the last timed launch, returns the summed device time
 * (ms) of the timed launches, their number, the number of all launches since
 * pft_prof_start, and the timed launches' summed algorithmic work (butterflies
 * for "ntt*" kernels, bytes read + written for the memory-bound ones, 0 where
 * not counted), then switches timing off.  Process-wide, not thread-safe.
 * Any argument may be NULL. */
int pft_prof_start(const char* prefix);
int pft_prof_stop(double* ms, long long* timed_launches, long long* all_launches, double* work);

/* ---- keys (KEYGEN, Sec. 2.3; key switching keys of the relinearisation and
 * ROTATE footnote) ---------------------------------------------------------
 * Sampler streams (64-bit word w = block w/8, 32-bit words 2(w%8) | 2(w%8)+1 << 32):
 *   secret s        ternary, domain 1 (word c mod 3 - 1)
 *   pk a / e        domain 2 (sub = limb) / domain 3
 *   switching key   a_j: domain 4, object = key id, sub = 256 j + basis row;
 *                   e_j: domain 5, object = key id, sub = j
 *   key id          0 for relinearisation, the Galois element g for rotations
 *   uniform mod q   words 2c, 2c+1 as a 128-bit value, reduced mod q
 *   Gaussian        magnitude = number of table entries the top 32 bits of
 *                   word c reach, sign = its lowest bit
 * Keys: b_j = -a_j s + e_j + [limb in digit j] P s', with s' = s^2 (relin) or
 * s(X^g) (rotation by step r, g = 5^r mod 2N), P = product of special primes.
 * Generates s, pk, the relinearisation key (want_relin != 0) and one rotation key
 * per entry of rot_steps (duplicates and identity steps are skipped). */
int pft_keygen(pft_ctx* ctx, const int32_t* rot_steps, int n_steps, int want_relin);
/* Add rotation keys after pft_keygen. */
int pft_add_rotation_keys(pft_ctx* ctx, const int32_t* rot_steps, int n_steps);
/* Export switching key `key_id` (0 = relin, else a Galois element) in coefficient
 * form, [beta_max][2][L + k][N] uint64, into host memory `out` of `n` words. */
int pft_key_export(pft_ctx* ctx, uint32_t key_id, uint64_t* out, size_t n);
/* Export the secret s as int64[N] coefficients (-1, 0, 1). */
int pft_secret_export(pft_ctx* ctx, int64_t* out, size_t n);

/* ---- plaintexts / ciphertexts --------------------------------------------- */
int pft_ct_create(pft_ctx* ctx, pft_ct** out); /* empty handle (level 0) */
int pft_ct_destroy(pft_ct* ct);
int pft_pt_destroy(pft_pt* pt);
int pft_ct_level(const pft_ct* ct, int* level);
int pft_ct_scale(const pft_ct* ct, double* scale);
int pft_pt_level(const pft_pt* pt, int* level);
/* Device pointer of the [2][l][N] buffer (evaluation domain), for zero-copy use. */
int pft_ct_data(const pft_ct* ct, uint64_t** dev_ptr);

/* ENCODE (Sec. 2.3): re_im = [2 * n_slots] doubles (re, im interleaved), n_slots <=
 * N/2 (the rest zero); mu_k = round half away from zero of
 * (2/N) Re sum_j scale z_j omega^(-(5^j mod 2N) k), omega = exp(i pi/N), computed
 * on the host in FP64 with an FFT; |mu_k| >= 2^62 -> PFT_ERR_ARG. */
int pft_encode(pft_ctx* ctx, const double* re_im, int n_slots, double scale, int level, pft_pt** out);
/* DECODE: z_j = mu(omega^(5^j mod 2N)) / scale with mu's CRT-centered coefficients. */
int pft_decode(pft_ctx* ctx, const pft_pt* pt, double* re_im_out, int n_slots);
/* Plaintext from / to coefficient-form residues [level][N] (canonical < q_r). */
int pft_pt_import(pft_ctx* ctx, const uint64_t* coeffs, int level, double scale, pft_pt** out);
int pft_pt_export(pft_ctx* ctx, const pft_pt* pt, uint64_t* coeffs, size_t n);

#define PFT_ENC_PK 0 /* c0 = v b + mu + e0, c1 = v a + e1 (v ternary, domain 8; e0, e1 domains 9, 10) */
#define PFT_ENC_SK 1 /* c0 = -a s + mu + e, c1 = a (a domain 6, sub = limb; e domain 7) */
/* ENC (Sec. 2.3, reading of the garbled formula as above); object id = nonce. */
int pft_encrypt(pft_ctx* ctx, const pft_pt* pt, int mode, uint32_t nonce, pft_ct** out);
/* DEC (Sec. 2.3): mu = c0 + c1 s. */
int pft_decrypt(pft_ctx* ctx, const pft_ct* ct, pft_pt** out);
/* Ciphertext from / to coefficient form [2][level][N] (canonical < q_r). */
int pft_ct_import(pft_ctx* ctx, const uint64_t* coeffs, int level, double scale, pft_ct** out);
int pft_ct_export(pft_ctx* ctx, const pft_ct* ct, uint64_t* coeffs, size_t n);

/* Batched transfers: B ciphertexts in one call, one transform launch, and (export) one
 * stream synchronisation at the end.  coeffs[i] points at [2][levels[i]][N] host words
 * (pinned host memory makes the copies asynchronous).  Import creates B new handles. */
int pft_ct_import_batch(pft_ctx* ctx, const uint64_t* const* coeffs, const int* levels, const double* scales, int B,
                        pft_ct** out);
/* The same into B existing handles of ctx (created by pft_ct_create or earlier calls): a
 * handle's buffer is reused when it is large enough, so repeated imports allocate nothing.
 * Stream-ordered like every operation: work queued earlier on the context's stream that
 * reads these handles completes before the copies overwrite them. */
int pft_ct_import_batch_into(pft_ctx* ctx, const uint64_t* const* coeffs, const int* levels, const double* scales,
                             int B, pft_ct* const* cts);
int pft_ct_export_batch(pft_ctx* ctx, const pft_ct* const* cts, int B, uint64_t* const* coeffs);
/* The same without the final synchronisation: the copies are queued on the context's stream
 * and coeffs[i] (page-locked host memory) holds the result once that stream has reached
 * this point (an event or a stream synchronisation by the caller); cts must not be modified
 * before then. */
int pft_ct_export_batch_async(pft_ctx* ctx, const pft_ct* const* cts, int B, uint64_t* const* coeffs);

/* ---- exchange of ciphertexts between processes (data-parallel training) ----
 * Sec. 4.2 splits a minibatch over GPUs, so the ranks' encrypted gradients must be summed.  A
 * sum of R ciphertexts of one level and scale is exact as an integer sum of their words when
 * R (q - 1) < 2^64 for every prime q of the level (R <= 16 at 60-bit primes): each rank copies its
 * words out (pft_ct_copy_out), a collective sums them as integers, and pft_ct_reduce_sum turns
 * the sums back into a ciphertext.  Larger R: gather the words and add them with pft_add. */
/* Device-to-device copy of ct's words ([2][l][N], evaluation layout) to dev_dst (2 l N words);
 * asynchronous on the context's stream. */
int pft_ct_copy_out(pft_ctx* ctx, const pft_ct* ct, uint64_t* dev_dst);
/* out = the ciphertext at `level` and `scale` whose words are dev_words ([2][level][N] device
 * words, each the exact integer sum of n_terms canonical residues of its limb's prime) reduced
 * modulo those primes.  PFT_ERR_ARG if n_terms (q - 1) can reach 2^64 for a prime of the level. */
int pft_ct_reduce_sum(pft_ctx* ctx, const uint64_t* dev_words, int level, double scale, int n_terms, pft_ct* out);

/* ---- homomorphic operations (Sec. 2.3) ------------------------------------
 * `out` must be a handle from pft_ct_create / an op; it is resized as needed. */
int pft_add(pft_ctx* ctx, const pft_ct* a, const pft_ct* b, pft_ct* out);       /* HADD */
int pft_sub(pft_ctx* ctx, const pft_ct* a, const pft_ct* b, pft_ct* out);
int pft_add_plain(pft_ctx* ctx, const pft_ct* a, const pft_pt* p, pft_ct* out); /* HADDPLAIN */
int pft_mul_plain(pft_ctx* ctx, const pft_ct* a, const pft_pt* p, pft_ct* out); /* HMULPLAIN, scale_a*scale_p */
/* HMUL followed by relinearisation: tensor (c00c10, c00c11+c01c10, c01c11), then
 * hybrid key switching of the third part (ModUp: fast basis conversion of each
 * alpha-prime digit to the other primes; inner product with the key; ModDown:
 * (x_Q - BConv_P->Q(x_P)) P^-1).  Same level required. */
int pft_mul_relin(pft_ctx* ctx, const pft_ct* a, const pft_ct* b, pft_ct* out);
/* RESCALE (Eq. 1 / Algorithm 3 with the rounding of Sec. 2.3): drop q_{l-1},
 * c'_k = (c_k + h - r) q_{l-1}^-1 mod q_k, r = (c_{l-1} + h) mod q_{l-1},
 * h = floor(q_{l-1}/2); scale /= q_{l-1}. */
int pft_rescale(pft_ctx* ctx, const pft_ct* a, pft_ct* out);
/* ROTATE: slot j of out = slot j+step of a (g = 5^step mod 2N), automorphism then
 * key switching with the rotation key of g.  Steps with no key -> PFT_ERR_NO_KEY. */
int pft_rotate(pft_ctx* ctx, const pft_ct* a, int32_t step, pft_ct* out);

/* ---- device status ---------------------------------------------------------
 * Kernels that wait on asynchronous copies (the key inner product streams the digit rows
 * through an mbarrier-counted shared-memory ring) bound every wait; if one expires the
 * kernel records it in a device flag and returns early, and its results are invalid.
 * pft_device_status synchronises the context's stream and returns PFT_ERR_TIMEOUT (clearing
 * the flag) if that happened since the last check; pft_ct_export_batch checks it too.
 * pft_wait_selftest queues a wait that can never complete, bounded by `polls` (1..2^20)
 * polls, which raises the flag: a diagnostic of the mechanism (no copy is in flight). */
int pft_device_status(pft_ctx* ctx);
int pft_wait_selftest(pft_ctx* ctx, long long polls);
/* Arithmetic ceiling of the transforms: butterflies per second of the transforms' own
 * Cooley-Tukey butterfly (Shoup product with the estimated quotient; the faster of its
 * corrected and uncorrected forms) on register-resident data with no memory traffic, 4 CTAs
 * per SM, timed with CUDA events on the context's stream (synchronous; about 20 ms).
 * *out: butterflies per second. */
int pft_bfly_ceiling(pft_ctx* ctx, double* out);
/* Issue rates of the 32-bit integer multiply forms a butterfly is made of, in operations per
 * second over the whole GPU, timed with CUDA events on the context's stream (synchronous; about
 * 10 ms): lo = low-word multiply-add (mad.lo), hi = high-word multiply (mul.hi / mad.hi),
 * wide = widening multiply (mad.wide).  A butterfly (one Shoup product with the estimated
 * quotient) takes 5 multiplies that produce a high word and 4 low-word multiply-adds, so the
 * transforms' arithmetic bound is 1 / (5 / min(hi, wide) + 4 / lo) butterflies per second.
 * Any pointer may be NULL. */
int pft_mul_rates(pft_ctx* ctx, double* lo, double* hi, double* wide);

/* ---- persistent job queue (batching over uneven levels and ring sizes) -----
 * HADD, subtraction and HMULPLAIN (Sec. 2.3) for ciphertexts of any contexts (rings of
 * different N and prime chains, one device) at any levels, executed by ONE persistent launch
 * on ctx's stream: resident CTAs claim tiles (one chunk of 2048 coefficients of one limb of one
 * polynomial) in list order from a device counter.
 *   op        PFT_JOB_ADD / PFT_JOB_SUB: out = a +- b (same context, level and scale);
 *             PFT_JOB_MUL_PLAIN: out = a (x) p slot-wise (p of a's context, level >= a's,
 *             leading limbs; scale multiplies)
 *   out       a handle of a's context (sized by the call; it may alias a or b)
 *   after     index of an earlier job that must have finished before this one starts, or -1.
 *             Every buffer a job shares with an earlier job (read after write, write after
 *             read or write) must belong to that earlier job or to one reached through the
 *             chain of `after` links; otherwise the call fails with PFT_ERR_ARG.
 *   wait_flag device pointer to a 32-bit word, or NULL: the job also waits until
 *             *wait_flag >= wait_value (written by another stream's kernel or copy).
 * Both waits are bounded by wait_timeout_s (0 < t <= 10 s) of the device's global timer; when
 * one expires the CTA skips that tile (its results are invalid), counts it as done so nothing
 * waits forever, and raises the device flag that pft_device_status reports as PFT_ERR_TIMEOUT.
 * Every job context must have ctx's current stream (pft_set_stream).  Asynchronous; an empty
 * list does nothing. */
enum { PFT_JOB_ADD = 0, PFT_JOB_SUB = 1, PFT_JOB_MUL_PLAIN = 2 };
typedef struct {
    int op;
    const pft_ct* a;
    const pft_ct* b;
    const pft_pt* p;
    pft_ct* out;
    int after;
    const uint32_t* wait_flag;
    uint32_t wait_value;
} pft_job;
int pft_run_jobs(pft_ctx* ctx, const pft_job* jobs, int n_jobs, double wait_timeout_s);

/* ---- level and scale management (used by the training step of Sec. 4.2) ---
 * The paper keeps every operand of a step at one level and scale; training mixes
 * operands of different depths, which these exact operations reconcile. */
/* The same message with the primes above `level` dropped (level <= a's level). */
int pft_drop_level(pft_ctx* ctx, const pft_ct* a, int level, pft_ct* out);
/* Adds `value` to every slot: the constant polynomial k = round(value * scale) (nearest
 * integer, halfway cases away from zero; |value * scale| < 2^63) is added to c0. */
int pft_add_const(pft_ctx* ctx, const pft_ct* a, double value, pft_ct* out);
/* Multiplies every slot by `value`: both polynomials times k = round(value * const_scale);
 * out scale = a's scale * const_scale (a following RESCALE divides it again). */
int pft_mul_const(pft_ctx* ctx, const pft_ct* a, double value, double const_scale, pft_ct* out);
/* Relabels ct's scale: the same integers now decrypt to old_scale / scale times the
 * message (exact; multiplying the scale by 8 divides the message by 8). */
int pft_ct_set_scale(pft_ct* ct, double scale);

/* Sums of HMULPLAIN products (the inner step of Sec. 3.1's matrix products):
 * outs[o] = sum_{k<K} cts[o K + k] * pts[pts_shared ? k : o K + k], all at one level, the
 * products of one output at one scale; one launch for all outputs. */
int pft_dot_plain_batch(pft_ctx* ctx, const pft_ct* const* cts, const pft_pt* const* pts, int K, int n_out,
                        int pts_shared, pft_ct* const* outs);

/* Rotations of one ciphertext by n steps that share one ModUp of c1 (hoisting): the
 * extended digits are computed once and permuted by each step's automorphism before the
 * inner product with that step's key and ModDown.  Fast basis conversion does not commute
 * exactly with the sign changes of the automorphism, so results equal pft_rotate's in
 * meaning, up to key-switching noise, not bit for bit.  outs[i] must differ from a. */
int pft_rotate_hoisted(pft_ctx* ctx, const pft_ct* a, const int32_t* steps, int n, pft_ct* const* outs);

/* Batched forms: one launch per stage over all B ciphertexts (levels may differ
 * between ciphertexts; pairs must match).  Keys are read once per level group. */
int pft_add_batch(pft_ctx* ctx, const pft_ct* const* a, const pft_ct* const* b, int B, pft_ct* const* out);
int pft_mul_plain_batch(pft_ctx* ctx, const pft_ct* const* a, const pft_pt* const* p, int B, pft_ct* const* out);
int pft_mul_relin_batch(pft_ctx* ctx, const pft_ct* const* a, const pft_ct* const* b, int B, pft_ct* const* out);
int pft_rescale_batch(pft_ctx* ctx, const pft_ct* const* a, int B, pft_ct* const* out);
int pft_rotate_batch(pft_ctx* ctx, const pft_ct* const* a, int B, int32_t step, pft_ct* const* out);

/* ---- autotuning -----------------------------------------------------------
 * A search over the ring's transform plans, per launch size.  A plan is one of the
 * specialised N = 2^16 kernels (two-pass 8 + 8 with register rounds at 3 or 4 resident CTAs per
 * SM; one launch on an 8-CTA cluster exchanging through distributed shared memory) or a sequence
 * of generic shared-memory passes with a chosen number of stages and sub-transforms per CTA
 * (N = 2^16: 8+8 at two tile widths, 6+10, 10+6, 7+9, 9+7, 5+5+6; N = 2^15: 8+7, 7+8, 9+6, 6+9,
 * 5+5+5; N <= 2^14 has a single one-pass plan).  For each launch-size bucket (total limbs of a
 * launch: <= 64, <= 512, larger) every plan is timed on a forward + inverse transform of a
 * representative launch (32, 256, 1024 limbs; median of 3 CUDA-event timings on the context's
 * stream) and the fastest is kept for launches of that size.  us_out (may be NULL) receives up
 * to `cap` plan times (microseconds) of the largest bucket, *chosen its choice (an index into
 * the plan list of pft_autotune_report).  Synchronous.  The environment variable PFT_NTT16
 * (twopass, twopass4, cluster, generic) overrides every choice at N = 2^16.  Before any search
 * a context uses the two-pass kernels at 3 CTAs per SM, and at 4 CTAs per SM for launches of more
 * than 512 limbs at N = 2^16 (the search's choice for that bucket on a GB300). */
#define PFT_NTT16_VARIANTS 4
int pft_autotune(pft_ctx* ctx, double* us_out, int cap, int* chosen);
/* The last search as JSON text: {"N": n, "buckets": [{"limbs": k, "chosen": name,
 * "us_fwd_inv": {plan name: microseconds, ...}}, ...]} ("buckets" empty before a search or for a
 * ring with one plan).  buf (may be NULL) receives up to cap - 1 bytes and a terminating zero;
 * *len (may be NULL) the full length. */
int pft_autotune_report(pft_ctx* ctx, char* buf, size_t cap, size_t* len);
/* Use plan `plan` (index into the ring's plan list, in the order above) for every launch size;
 * -1: back to the plans a new context starts with. */
int pft_set_transform_plan(pft_ctx* ctx, int plan);
/* Pin the N = 2^16 transform variant (0..PFT_NTT16_VARIANTS-1: two-pass 3 CTAs/SM, two-pass 4
 * CTAs/SM, cluster, generic 8 + 8) for every launch size, without timing. */
int pft_set_transform_variant(pft_ctx* ctx, int variant);
/* Environment switches (measured defaults otherwise), all kernel choices with identical results:
 *   PFT_NTT_ORDER  read at pft_ctx_create; bit 0: the second pass of an N = 2^16 two-pass
 *                  transform visits (polynomial, limb) in reverse, so it starts on the data the
 *                  first pass wrote last (still in L2); bit 1: the row twiddles are read with an
 *                  L2 evict-last policy; bit 2: the pass that applies ModDown's epilogue asks L2
 *                  for the epilogue's operands at the start of each block (measured slower with
 *                  the current epilogue, off by default).  Default 3.
 *   PFT_BCONV=tc   read at pft_ctx_create: basis conversion of four-prime digits on the tensor
 *                  cores (exact byte-plane products; measured slower than the default). */

/* ---- CUDA graphs of batched operations ------------------------------------
 * pft_graph_begin starts capturing the work the following calls queue on the context
 * stream; pft_graph_end instantiates it; pft_graph_launch replays it on the context stream
 * (a whole batched step becomes one graph launch).  Requirements: a non-default context
 * stream and the default (stream-ordered, capturable) allocator -- a context created with a
 * custom allocator returns PFT_ERR_ARG.  Replaying is valid for calls whose output handles
 * already hold buffers of the right size and keep them (HADD, HMULPLAIN, mul_relin, rotate
 * and their batched forms, after one eager warm-up call); calls that copy host data
 * (import/export, encode/decode, encryption, the fastText entry points) or replace output
 * buffers (rescale) are not capturable.  Keep the captured handles alive while the graph is
 * used. */
typedef struct pft_graph pft_graph;
int pft_graph_begin(pft_ctx* ctx);
int pft_graph_end(pft_ctx* ctx, pft_graph** out);
int pft_graph_launch(pft_ctx* ctx, const pft_graph* graph);
int pft_graph_destroy(pft_graph* graph);

/* ---- rescale without allocation --------------------------------------------
 * The paper has no counterpart to this call; it exists for callers that cannot obtain
 * device memory at the moment they call the library -- for example an application whose
 * device memory is entirely owned by another framework's pool, or a processing loop in
 * which allocator calls are not allowed.  It computes exactly what pft_rescale computes,
 * on raw device buffers, and allocates nothing: the caller passes the input and the output,
 * and the working space comes from a fixed array of 4 Mi 64-bit words (32 MiB) compiled
 * into the library, which every device that loads the library holds until the process
 * exits.
 *   in     device pointer, ciphertext [2][level][N] in the evaluation layout (pft_ct_data)
 *   level  2..L; 2 N level must not exceed 4 Mi words (N = 2^16: level <= 32), else
 *          PFT_ERR_ARG with a message naming the limit
 *   out    device pointer, [2][level-1][N]; must not overlap `in`; receives the rescaled
 *          ciphertext (its scale is the input scale divided by q_{level-1})
 * Work is queued on the context stream.  The context's device (the one current at
 * pft_ctx_create, which also looked up the array's device address there) must be current,
 * else PFT_ERR_ARG.  All calls on a device share the array and it keeps the last call's
 * contents: calls whose GPU work overlaps (different streams or contexts on the same device)
 * race on it. */
int pft_rescale_noalloc(pft_ctx* ctx, const uint64_t* in, int level, uint64_t* out);

/* ---- raw transforms on caller memory (kernel-level access) ----------------
 * data: device buffer of n_polys polynomials [n_polys][n_limbs][N], limb r under
 * prime r of the chain (r < L + k; rows >= L are the special primes).  inverse = 0:
 * coefficient -> evaluation layout above; 1: back. In place. */
int pft_ntt(pft_ctx* ctx, uint64_t* data, int n_polys, int n_limbs, int inverse);

/* ---- encrypted fastText inference (Sec. 3.1, Fig. 3, Algorithm 2) ---------
 * Model: H (m x n, row-major doubles) packed vertically -- plaintext (j, i) holds
 * column j, vocabulary rows i*t .. i*t+t-1, t = N/2 -- at `level`, scale Delta;
 * O (n x c) packed horizontally -- plaintext j holds row j in slots 0..c-1 -- at
 * level-1, scale Delta. */
int pft_ft_model_create(pft_ctx* ctx, const double* H, const double* O, int m, int n, int c, int level,
                        pft_ft_model** out);
/* The same from already encoded plaintexts: H_pts[j * n_chunks + i], O_pts[j]. */
int pft_ft_model_import(pft_ctx* ctx, const pft_pt* const* H_pts, const pft_pt* const* O_pts, int m, int n,
                        int c, pft_ft_model** out);
int pft_ft_model_destroy(pft_ft_model* model);
/* Rotation-light variant (not in the paper): diagonal packing, per vocabulary chunk i (rows
 * i t .. i t + t - 1 of H, ceil(m/t) chunks) D_{i,k}[s] = H[i t + (s+k) mod t, s mod n] (k < n, at
 * `level`; plaintext i n + k) and P[n c' + j] = O[j, c'] (one plaintext, level-1).  Inference
 * computes Q = sum_i sum_k rot(v_i, k) D_{i,k} with n-1 hoisted rotations per chunk,
 * Q += rot(Q, n 2^s) while n 2^s < t, rescale, S = Q P, S += rot(S, 2^s) while 2^s < n,
 * rescale: chunks (n - 1) + log2(t/n) + log2(n) rotations (78 for one chunk, n = 64,
 * t = 32768) instead of n log2(t) (960), the n - 1 of a chunk sharing one ModUp.  Needs n a
 * power of two dividing t, n c <= t, rotation keys for 1..n-1 and n 2^s.  Scores land in slots
 * n c' (c' < c), not 0..c-1.  The input is rotated before its plaintext product, so
 * key-switching noise is relative to the input's scale: encrypt v at a scale of 2^50 or more
 * (instead of 2^40) to keep the scores within 2^-20. */
int pft_ft_model_create_diag(pft_ctx* ctx, const double* H, const double* O, int m, int n, int c, int level,
                             pft_ft_model** out);
int pft_ft_model_import_diag(pft_ctx* ctx, const pft_pt* const* D_pts, const pft_pt* P_pt, int m, int n, int c,
                             pft_ft_model** out);
/* Scores of one document: v = ceil(m/t) ciphertexts at one level l (either packing), 3 <= l <= the model
 * level (the client's count vector, already divided by w; a model encoded at level L serves
 * every l <= L through the first l limbs of its plaintexts, which equal the encoding at
 * level l).  Sequence: h_j = TotalSum(sum_i v_i * H_{j,i}) with TotalSum rotating by 2^i,
 * i = 0..log2(t)-1 (Algorithm 2), rescale; s = sum_j h_j * O_j; rescale.  Needs rotation
 * keys for 2^i.  `scores` receives s in slots 0..c-1 at level l-2. */
int pft_fasttext_infer(pft_ctx* ctx, const pft_ft_model* model, const pft_ct* const* v, int n_chunks,
                       pft_ct* scores);
/* B documents: v[b * n_chunks + i], each at its own level; all columns of all documents
 * share each rotation key read. */
int pft_fasttext_infer_batch(pft_ctx* ctx, const pft_ft_model* model, const pft_ct* const* v, int n_chunks,
                             int B, pft_ct* const* scores);
/* ---- request server: continuous batching of fastText inferences ----------
 * The serving side of Sec. 3.1 (the server evaluates clients' encrypted documents with
 * its own model); the paper measures single inferences and has no request loop.
 * A server drives n_rings rings, each a context (with its rotation keys, its model and
 * its own stream) and a model; rings of different N run concurrently on their streams.
 * Each request is one document for one ring at level 3..model level.  pft_server_step
 * runs one iteration: retire finished requests, admit waiting ones in arrival order
 * while the sum of admitted footprints (pft_server_footprint: the request's inputs,
 * working ciphertexts and score on the device) stays within budget_bytes (0: no
 * limit), then advance every admitted request by one stage of its sequence (column
 * products; one rotate-and-sum step; the output layer), requests at the same stage
 * of a ring forming one batched call.  It returns once the previous iteration has
 * finished on the device.  The key-switching work space of each call is allocated
 * per call besides the budget.  A result equals that of pft_fasttext_infer on the
 * same input, whatever else was in flight.  Destroy the server before its contexts
 * and models.  Calls on one server must not overlap;
 * after an error other than PFT_ERR_ARG / _LEVEL_MISMATCH / _OOM from
 * pft_server_submit, destroy the server. */
typedef struct pft_server pft_server;
typedef struct {
    uint64_t tag;
    int ring;
    int level;      /* level of the score ciphertext (request level - 2) */
    double scale;   /* scale of the score ciphertext */
    double t_submit; /* server clock (seconds) at pft_server_submit */
    double t_done;   /* server clock when the score had reached host memory (CUDA event) */
} pft_server_done;
typedef struct {
    int waiting, active, exporting, max_active;
    long completed, iterations;
    size_t bytes_in_use, peak_bytes, budget;
} pft_server_stats;
int pft_server_create(pft_ctx* const* ctxs, const pft_ft_model* const* models, int n_rings, size_t budget_bytes,
                      pft_server** out);
int pft_server_destroy(pft_server* srv);
/* Text of the last error on srv; srv = NULL: of the last failed pft_server_create. */
const char* pft_server_last_error(const pft_server* srv);
/* Queues one request.  in: host [chunks][2][level][N] u64 in coefficient form, canonical
 * residues (chunks = ceil(m/t) for both packings), at `scale`; out: host
 * buffer of 2 (level-2) N words that receives the score in the same form.  Both stay
 * owned by the caller and must stay valid until the request is returned by
 * pft_server_poll (the inputs are read at admission).  PFT_ERR_OOM if the request's
 * footprint alone exceeds the budget. */
int pft_server_submit(pft_server* srv, int ring, const uint64_t* in, int level, double scale, uint64_t* out,
                      uint64_t tag);
/* One iteration; *n_pending (may be NULL) = requests not yet returned by poll's retire. */
int pft_server_step(pft_server* srv, int* n_pending);
/* Steps until every queued request has completed. */
int pft_server_drain(pft_server* srv);
/* Completed requests, oldest first, up to max; *n = how many were written. */
int pft_server_poll(pft_server* srv, pft_server_done* done, int max, int* n);
/* Seconds since pft_server_create (host steady clock; the time base of submit/done). */
int pft_server_clock(pft_server* srv, double* t);
int pft_server_get_stats(pft_server* srv, pft_server_stats* stats);
int pft_server_footprint(pft_server* srv, int ring, int level, size_t* bytes);

/* ---- encrypted minibatch training (Sec. 4.2, Algorithm 5) ----------------
 * Encrypted model: H_j = column j of H over the vocabulary slots (m <= t), at level l0;
 * O_j = row j of O in slots 0..c-1, at level l0-1; one scale for all H_j, one for all O_j.
 * Per step the client sends documents v_b (count vectors divided by w) at level l0 and
 * labels w_b = y_b - 1/4 on the c class slots (one-hot y_b; the constant term of the
 * softmax polynomial is folded into the label) at the level and scale
 * pft_fasttext_train_spec gives.  The softmax is the paper's P(s) = s^2/8 + s/2 + 1/4;
 * the loss is L = sum_b sum_c [s^3/24 + s^2/4 + s/4 - y s], whose gradient in s is
 * P(s) - y.  Gradients: dO_j = sum_b h_bj g_b (level l0-4, slots 0..c-1), dH_j =
 * sum_b v_b e_bj with e_bj = sum_c g_bc O_jc (level l0-5), g_b = P(s_b) - y_b.
 * SGD: O_j <- O_j - eta dO_j (level l0-5), H_j <- H_j - eta dH_j (level l0-6), the
 * model's scales unchanged.  Needs the relinearisation key and rotation keys 2^i,
 * i < log2(t).  Six levels per step: a model at level l0 affords floor((l0-1)/6) steps. */
typedef struct pft_ft_enc_model pft_ft_enc_model;
typedef struct pft_ft_tape pft_ft_tape; /* forward state kept for the backward pass */
/* Copies H[0..n-1] and O[0..n-1] into a new encrypted model. */
int pft_ft_enc_model_create(pft_ctx* ctx, const pft_ct* const* H, const pft_ct* const* O, int m, int n, int c,
                            pft_ft_enc_model** out);
/* Rotation-light layout (not in the paper): D[k] = the diagonals D_k[i] = H[(i+k) mod t, i mod n]
 * (k < n, level l0), P = O packed as P[n c' + j] = O[j, c'] (one ciphertext, level l0-1) and a
 * plaintext mask with 1 in the score slots n c' (level >= l0-2; its leading limbs serve lower
 * levels).  Labels w_b = y_b - 1/4 spread over the class blocks: w_b[c'] in slots n c' .. n c' + n - 1.
 * Per document n-1 hoisted rotations of v_b and rotate-and-sums by n 2^s, 2^s and -2^s replace
 * the n log2(t) rotations of each TotalSum: h_b comes out replicated with period n, the scores
 * spread over their blocks, and the backward reuses the rotated documents (dD_k = sum_b
 * rot(v_b, k) E_b).  lift_bits K (0..30): the documents are multiplied by the integer 2^K before
 * their rotations, which divides the key-switching noise those rotations add (the only key
 * switches at the input scale, summed over the vocabulary) by 2^K; a mask encoded at 2^-K times
 * the usual scale returns the scores to it.  Gradients: grad_H receives the n diagonals of dH
 * (level l0-6), grad_O[0] receives dO in the layout of P (level l0-5).  Seven levels per step:
 * the update leaves D_k at l0-7 and P at l0-8.  Needs m <= t, n a power of two dividing t,
 * n c <= t, and rotation keys for 1..n-1, n 2^s (< t) and -2^s (< n).  The handles are copied. */
int pft_ft_enc_model_create_diag(pft_ctx* ctx, const pft_ct* const* D, const pft_ct* P, const pft_pt* mask, int m,
                                 int n, int c, int lift_bits, pft_ft_enc_model** out);
/* Copy of H_j (which = 0) or O_j (which = 1) into out (diagonal layout: D_j, and P for j = 0). */
int pft_ft_enc_model_get(pft_ctx* ctx, const pft_ft_enc_model* model, int which, int j, pft_ct* out);
int pft_ft_enc_model_levels(const pft_ft_enc_model* model, int* level_H, int* level_O);
int pft_ft_enc_model_destroy(pft_ft_enc_model* model);
/* Level of the documents and level and scale of the labels for documents encrypted at
 * input_scale (the scale the forward pass reaches at the softmax). */
int pft_fasttext_train_spec(pft_ctx* ctx, const pft_ft_enc_model* model, double input_scale, int* doc_level,
                            int* label_level, double* label_scale);
/* Forward pass of B documents (levels >= 6): keeps h, s and g in *tape.  docs must stay
 * alive until the tape is destroyed.  PFT_ERR_SCALE_MISMATCH if a label is not at the
 * scale of pft_fasttext_train_spec. */
int pft_fasttext_train_forward(pft_ctx* ctx, const pft_ft_enc_model* model, const pft_ct* const* docs,
                               const pft_ct* const* labels, int B, pft_ft_tape** tape);
/* Copy of the encrypted scores s_b of document b (slots 0..c-1, level l0-2). */
int pft_ft_tape_score(pft_ctx* ctx, const pft_ft_tape* tape, int b, pft_ct* out);
/* Backward pass (the adjoint of the forward): grad_H[j], grad_O[j] for j < n. */
int pft_fasttext_train_backward(pft_ctx* ctx, const pft_ft_tape* tape, pft_ct* const* grad_H,
                                pft_ct* const* grad_O);
int pft_ft_tape_destroy(pft_ft_tape* tape);
/* SGD update of the model with the gradients (eta = 0: no change). */
int pft_fasttext_train_update(pft_ctx* ctx, pft_ft_enc_model* model, const pft_ct* const* grad_H,
                              const pft_ct* const* grad_O, double eta);
/* One whole step (forward, backward, update) over B documents, processed in tiles of
 * documents so that only one tile's forward state is held at a time; results equal the
 * three calls above.  grad_H / grad_O may be NULL (the gradients are then not returned).
 * Levels >= 7 when eta != 0. */
int pft_fasttext_train_step(pft_ctx* ctx, pft_ft_enc_model* model, const pft_ct* const* docs,
                            const pft_ct* const* labels, int B, double eta, pft_ct* const* grad_H,
                            pft_ct* const* grad_O);

#ifdef __cplusplus
}
#endif
#endif /* PRIVFT_H */
