// Negacyclic number-theoretic transform over Z_q[X]/(X^N+1), batched over
// (polynomial, limb).  The paper's GPU library used a Discrete Galois Transform
// (Sec. 4.1); this is the psi-twisted radix-2 NTT with merged twiddles:
//
//   forward (Cooley-Tukey), stage s = 0..logN-1, m = 2^s, t = N/(2m):
//     for i < m, j in [2it, 2it+t):  (a_j, a_{j+t}) <- (a_j + W a_{j+t}, a_j - W a_{j+t}),
//     W = psi^brv(m+i);  output entry i = a(psi^(2 brv(i)+1)).
//   inverse (Gentleman-Sande), stages in reverse order with W^-1 and
//     (u, v) <- (u + v, (u - v) W^-1), then a factor N^-1 (folded into the last stage).
//
// GB300 mapping: a launch ("pass") covers S consecutive stages.  Within a pass the
// N points split into independent sub-transforms of 2^S points at stride T =
// N >> (s0 + S); a CTA loads C of them into shared memory with coalesced loads,
// each thread keeps 16 points in registers and applies up to 4 stages per round
// (Harvey butterflies with an estimated Shoup quotient: forward values in [0, 8q), uncorrected
// for primes below 2^57 in the N = 2^16 kernels; inverse values in [0, 4q)), and
// rounds exchange through shared memory.  N <= 2^14: one pass, one CTA per limb.
// N = 2^15, 2^16: two passes (8 + 7 or 8 + 8 stages).
#include <cooperative_groups.h>

#include <algorithm>

#include <cstdlib>
#include <cstring>

#include "modarith.cuh"

namespace cg = cooperative_groups;

namespace pft {

// ---- butterflies ---------------------------------------------------------------------------
// Shoup product x W mod q in [0, 2q), formed as x w + hq (-q) (mod 2^64) so that the
// subtraction folds into the multiply-adds; nq = -q mod 2^64.
__device__ __forceinline__ u64 shoup_nq(u64 x, ulonglong2 W, u64 nq) { return x * W.x + mulhi(x, W.y) * nq; }
// Quotient estimate of the Shoup product without the low x low partial product:
// floor(x w' / 2^64) - {0, 1, 2}.  Writing x = xh 2^32 + xl and w' = wh 2^32 + wl, the exact
// value is xh wh + floor((xh wl + xl wh + floor(xl wl / 2^32)) / 2^32); the three dropped
// low halves sum to less than 3 * 2^32, so at most 2 carries are lost.  With it the Shoup
// product x w - h q lies in [0, 4q) instead of [0, 2q).
__device__ __forceinline__ u64 mulhi_est(u64 x, u64 w) {
    const uint32_t xl = (uint32_t)x, xh = (uint32_t)(x >> 32);
    const uint32_t wl = (uint32_t)w, wh = (uint32_t)(w >> 32);
    return (u64)xh * wh + ((u64)__umulhi(xh, wl) + __umulhi(xl, wh));
}
// y w - q_est q (mod 2^64) with q_est = mulhi_est(y, w'), written as 32-bit multiply-adds with
// explicit carries: the quotient takes two high-word products and one widening product (the
// partial sums hi(yh w'l) + hi(yl w'h) enter the widening product as its 64-bit addend), the
// low 64 bits of y w + q_est (-q) take two widening products and four low-word multiply-adds.
// The same value as y * w + mulhi_est(y, w') * nq in 64-bit C arithmetic, in fewer
// instructions than the compiler forms from that expression.  nq = -q mod 2^64.
__device__ __forceinline__ u64 shoup_est(u64 y, u64 w, u64 wp, u64 nq) {
    u64 T;
    asm("{\n\t"
        ".reg .u32 yl, yh, pl, ph, t, r, c, wl, wh, ql, qh, nl, nh, tl, th;\n\t"
        ".reg .u64 Q, A;\n\t"
        "mov.b64 {yl, yh}, %1;\n\t"
        "mov.b64 {pl, ph}, %3;\n\t"
        "mul.hi.u32 t, yh, pl;\n\t"
        "mad.hi.cc.u32 r, yl, ph, t;\n\t"
        "addc.u32 c, 0, 0;\n\t"
        "mov.b64 A, {r, c};\n\t"
        "mad.wide.u32 Q, yh, ph, A;\n\t"
        "mov.b64 {wl, wh}, %2;\n\t"
        "mov.b64 {ql, qh}, Q;\n\t"
        "mov.b64 {nl, nh}, %4;\n\t"
        "mul.wide.u32 A, yl, wl;\n\t"
        "mad.wide.u32 A, ql, nl, A;\n\t"
        "mov.b64 {tl, th}, A;\n\t"
        "mad.lo.u32 th, yl, wh, th;\n\t"
        "mad.lo.u32 th, yh, wl, th;\n\t"
        "mad.lo.u32 th, ql, nh, th;\n\t"
        "mad.lo.u32 th, qh, nl, th;\n\t"
        "mov.b64 %0, {tl, th};\n\t"
        "}"
        : "=l"(T)
        : "l"(y), "l"(w), "l"(wp), "l"(nq));
    return T;
}
// Cooley-Tukey (Harvey) with the estimated quotient, so WY lies in [0, 4q):
// X, Y in [0, 8q) -> X + WY, X - WY in [0, 8q) (X corrected below 4q; primes below 2^61).
// LAZY (primes below 2^57): no correction of X, values grow by less than 4q per stage: the
// 16 stages of an N = 2^16 forward transform from [0, 2q) stay below 66q < 2^63.1.
template <bool LAZY = false>
__device__ __forceinline__ void ct_bfly(u64& X, u64& Y, ulonglong2 W, u64 q, u64 q2) {
    const u64 q4 = 2 * q2;
    if (!LAZY && X >= q4) X -= q4;
    const u64 T = shoup_est(Y, W.x, W.y, 0 - q);
    Y = X - T + q4;
    X = X + T;
}
// Gentleman-Sande: X, Y in [0, 4q) -> X + Y, (X - Y) W in [0, 4q) (primes below 2^61: sums
// and differences below 8q; the product with the estimated quotient lies in [0, 4q))
__device__ __forceinline__ void gs_bfly(u64& X, u64& Y, ulonglong2 W, u64 q, u64 q2) {
    const u64 q4 = 2 * q2;
    u64 S = X + Y;
    if (S >= q4) S -= q4;
    const u64 D = X - Y + q4;
    X = S;
    Y = shoup_est(D, W.x, W.y, 0 - q);
}
__device__ __forceinline__ u64 canon4(u64 v, u64 q, u64 q2) {
    if (v >= q2) v -= q2;
    if (v >= q) v -= q;
    return v;
}
__device__ __forceinline__ u64 canon8(u64 v, u64 q, u64 q2) {
    if (v >= 2 * q2) v -= 2 * q2;
    return canon4(v, q, q2);
}

// L2 policy of the row twiddles: evict-last keeps the per-row tables (1 MiB per prime) in L2
// while the streamed limbs pass through it; evict-normal is the default behaviour.
__device__ __forceinline__ u64 tw_policy(bool keep) {
    u64 pol;
    if (keep) asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    else asm("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
// read-only 16-byte load under an L2 policy (the tables do not change during a launch)
__device__ __forceinline__ ulonglong2 ldg_pol(const ulonglong2* p, u64 pol) {
    ulonglong2 v;
    asm("ld.global.nc.L2::cache_hint.v2.u64 {%0, %1}, [%2], %3;" : "=l"(v.x), "=l"(v.y) : "l"(p), "l"(pol));
    return v;
}
// Pass flags of the two-pass kernels: bit 0 canonical output (the last pass of a transform),
// bit 1 reverse order: the CTAs visit (polynomial, limb) from the last to the first, so that a
// pass that follows another over the same data starts on what that pass wrote last.
constexpr int kPassFinal = 1, kPassReverse = 2;
// (fused ModDown pass) bit 2: prefetch the epilogue operands into L2 at the start of the CTA
constexpr int kPassPrefetch = 4;
__device__ __forceinline__ int pass_poly(int flags) {
    return (flags & kPassReverse) ? (int)(gridDim.z - 1 - blockIdx.z) : (int)blockIdx.z;
}
__device__ __forceinline__ int pass_limb(int flags) {
    return (flags & kPassReverse) ? (int)(gridDim.y - 1 - blockIdx.y) : (int)blockIdx.y;
}

// ---- N = 2^16 in one launch: an 8-CTA cluster per limb ------------------------------------
// The limb is viewed as a 256 x 256 array, element j = row * 256 + col.  Forward stages
// 0..7 pair elements along a column (row bit 7 - s), stages 8..15 along a row (col bit
// 15 - s); group index i = j / (2t) is row >> (8 - s) for s < 8 and
// row 2^(s-8) + (col >> (16 - s)) for s >= 8.  CTA c of the cluster transforms columns
// 32c..32c+31 (phase 1), then gathers rows 32c..32c+31 from all eight CTAs' shared memory
// (distributed shared memory) and transforms them (phase 2); the inverse runs the same
// two phases in the opposite order.  Lane = sub-transform, so every shared and remote
// access is a stride-33 (odd) walk: conflict-free.  One HBM read and one write per limb.
//
// One round = four stages on 16 registers: register e holds element (e << W0) | wpart of
// the current 256-point sub-transform; DIMHI = 0 for column stages (s = 7 - p), 8 for row
// stages (s = 15 - p, r = the row being transformed).
// LM (the row round W0 = 0 of stages 12..15, thread = row r, lane w): the twiddles come from
// the lane-major copy of that round's twiddles, lm = its entries for (prime, row r, lane w):
// slot (2^k - 1 + j) of stage 12 + k at lm[16 (2^k - 1 + j)], loaded under the L2 policy pol.
// RT (the row round W0 = 4 of stages 8..11, thread = row r): the row's 15 twiddles of those
// stages were copied to shared memory, stage 8 + k entry j at rt[2^k - 1 + j].
template <bool INV, int W0, int DIMHI, bool LAZY = false, bool UNSCALED = false, bool LM = false, bool RT = false>
__device__ __forceinline__ void ntt16_round(u64 (&x)[16], int wpart, int r, const ulonglong2* __restrict__ tw,
                                            u64 q, u64 q2, ulonglong2 NI, ulonglong2 NI1,
                                            const ulonglong2* __restrict__ lm = nullptr,
                                            const ulonglong2* rt = nullptr, u64 pol = 0) {
    static_assert(!LM || (W0 == 0 && DIMHI == 8), "lane-major twiddles serve the row round of stages 12..15");
    static_assert(!RT || (W0 == 4 && DIMHI == 8), "staged row twiddles serve the row round of stages 8..11");
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const int lb = INV ? k : 3 - k;
        const int p = W0 + lb;
        const int s = DIMHI + 7 - p;
#pragma unroll
        for (int e = 0; e < 16; e++) {
            if (e & (1 << lb)) continue;
            const int elem = (e << W0) | wpart;
            const int idx = (1 << s) + (r << (7 - p)) + (elem >> (p + 1));
            const ulonglong2 W = LM   ? ldg_pol(&lm[16 * ((1 << (s - 12)) - 1 + (e >> (p + 1)))], pol)
                                 : RT ? rt[(1 << (s - 8)) - 1 + (elem >> (p + 1))]
                                      : __ldg(&tw[idx]);
            if (!INV) {
                ct_bfly<LAZY>(x[e], x[e | (1 << lb)], W, q, q2);
            } else if (s == 0 && !UNSCALED) {  // last inverse stage: N^-1 folded into both outputs
                u64 S = x[e] + x[e | (1 << lb)];
                if (S >= 2 * q2) S -= 2 * q2;
                const u64 D = x[e] - x[e | (1 << lb)] + 2 * q2;
                x[e] = mul_shoup_lazy(S, NI.x, NI.y, q);
                x[e | (1 << lb)] = mul_shoup_lazy(D, NI1.x, NI1.y, q);
            } else {
                gs_bfly(x[e], x[e | (1 << lb)], W, q, q2);
            }
        }
    }
}


constexpr int kN16Stride = 33;  // shared layout [256][33]: element (a, lane) at a * 33 + lane

template <bool INV, int MINB>
__global__ void __cluster_dims__(8, 1, 1) __launch_bounds__(512, MINB)
    k_ntt16_cluster(DevTables t, PolySet in, PolySet out) {
    extern __shared__ u64 sm[];
    cg::cluster_group cluster = cg::this_cluster();
    const int c = (int)cluster.block_rank();
    const int poly = blockIdx.z, limb = blockIdx.y;
    const PolyRef& Ro = out.p[poly];
    if (limb >= Ro.nlimbs) return;  // uniform over the cluster (same limb)
    const int pi = prime_of(Ro, limb);
    const u64* src = in.p[poly].ptr + ((size_t)limb << 16);
    u64* dst = Ro.ptr + ((size_t)limb << 16);
    const u64 q = __ldg(&t.primes[pi].q);
    const u64 q2 = 2 * q;
    const ulonglong2* tw = (INV ? t.inv : t.fwd) + ((size_t)pi << 16);
    const ulonglong2 NI = INV ? __ldg(&t.ninv[pi]) : make_ulonglong2(0, 0);
    const ulonglong2 NI1 = INV ? __ldg(&t.inv1ninv[pi]) : make_ulonglong2(0, 0);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    constexpr int ST = kN16Stride;
    u64 x[16];

    if (!INV) {
        // phase 1: columns 32c + lane
        const int col = 32 * c + lane;
#pragma unroll
        for (int e = 0; e < 16; e++) x[e] = src[(size_t)((e << 4) | w) * 256 + col];
        ntt16_round<false, 4, 0>(x, w, 0, tw, q, q2, NI, NI1);
#pragma unroll
        for (int e = 0; e < 16; e++) sm[((e << 4) | w) * ST + lane] = x[e];
        __syncthreads();
#pragma unroll
        for (int e = 0; e < 16; e++) x[e] = sm[((w << 4) | e) * ST + lane];
        ntt16_round<false, 0, 0>(x, w << 4, 0, tw, q, q2, NI, NI1);
#pragma unroll
        for (int e = 0; e < 16; e++) sm[((w << 4) | e) * ST + lane] = x[e];
        cluster.sync();
        // phase 2: rows 32c + lane, gathered from the CTA holding each column
        const int r = 32 * c + lane;
#pragma unroll
        for (int e = 0; e < 16; e++) {
            const int cx = (e << 4) | w;
            const u64* rem = cluster.map_shared_rank(sm, cx >> 5);
            x[e] = rem[r * ST + (cx & 31)];
        }
        cluster.sync();
        ntt16_round<false, 4, 8>(x, w, r, tw, q, q2, NI, NI1);
#pragma unroll
        for (int e = 0; e < 16; e++) sm[((e << 4) | w) * ST + lane] = x[e];
        __syncthreads();
#pragma unroll
        for (int e = 0; e < 16; e++) x[e] = sm[((w << 4) | e) * ST + lane];
        ntt16_round<false, 0, 8>(x, w << 4, r, tw, q, q2, NI, NI1);
#pragma unroll
        for (int e = 0; e < 16; e++) sm[((w << 4) | e) * ST + lane] = canon8(x[e], q, q2);
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 16; k++) {
            const int f = threadIdx.x + 512 * k;
            const int rho = f >> 8, cx = f & 255;
            dst[(size_t)(32 * c + rho) * 256 + cx] = sm[cx * ST + rho];
        }
    } else {
        // phase 1: rows 32c + lane (coalesced load through shared memory, layout [col][row])
        const int r = 32 * c + lane;
#pragma unroll
        for (int k = 0; k < 16; k++) {
            const int f = threadIdx.x + 512 * k;
            const int rho = f >> 8, cx = f & 255;
            sm[cx * ST + rho] = src[(size_t)(32 * c + rho) * 256 + cx];
        }
        __syncthreads();
#pragma unroll
        for (int e = 0; e < 16; e++) x[e] = sm[((w << 4) | e) * ST + lane];
        ntt16_round<true, 0, 8>(x, w << 4, r, tw, q, q2, NI, NI1);
#pragma unroll
        for (int e = 0; e < 16; e++) sm[((w << 4) | e) * ST + lane] = x[e];
        __syncthreads();
#pragma unroll
        for (int e = 0; e < 16; e++) x[e] = sm[((e << 4) | w) * ST + lane];
        ntt16_round<true, 4, 8>(x, w, r, tw, q, q2, NI, NI1);
#pragma unroll
        for (int e = 0; e < 16; e++) sm[((e << 4) | w) * ST + lane] = x[e];
        cluster.sync();
        // phase 2: columns 32c + lane, gathered from the CTA holding each row
        const int col = 32 * c + lane;
#pragma unroll
        for (int e = 0; e < 16; e++) {
            const int row = (w << 4) | e;
            const u64* rem = cluster.map_shared_rank(sm, row >> 5);
            x[e] = rem[col * ST + (row & 31)];
        }
        cluster.sync();
        ntt16_round<true, 0, 0>(x, w << 4, 0, tw, q, q2, NI, NI1);
#pragma unroll
        for (int e = 0; e < 16; e++) sm[((w << 4) | e) * ST + lane] = x[e];
        __syncthreads();
#pragma unroll
        for (int e = 0; e < 16; e++) x[e] = sm[((e << 4) | w) * ST + lane];
        ntt16_round<true, 4, 0>(x, w, 0, tw, q, q2, NI, NI1);
#pragma unroll
        for (int e = 0; e < 16; e++) dst[(size_t)((e << 4) | w) * 256 + col] = canon4(x[e], q, q2);
    }
}

// ---- N = 2^16 in two passes of 8 stages, global memory touched from registers ----------------
// Pass A (stages 0..7): 256-point column transforms at stride T = 2^LOGT; a CTA takes 16
// adjacent columns, lane bits 0..3 = column, so every global access of a warp reads or
// writes two 128-byte runs.  Pass B (stages 8..15): 16 contiguous 256-point rows per CTA,
// lane bits 0..3 = point.  Each pass does 2 rounds of 4 stages with one shared-memory
// exchange (odd strides 17 / 273: conflict-free); pass B stages its final store (forward)
// or first load (inverse) through shared memory to keep the global side coalesced.
constexpr int kRowStride = 273;  // 256 + 16 padding + 1
constexpr u64 kLazyBound = 1ull << 57;  // forward butterflies skip the correction below this prime

// UNSCALED (inverse): the last stage is a plain Gentleman-Sande butterfly (no N^-1) and the
// output stays in [0, 4q): N times the inverse transform, for a consumer that scales anyway.
template <bool INV, int LOGT, int MINB, bool UNSCALED = false>
__global__ void __launch_bounds__(256, MINB) k_ntt8_strided(DevTables t, PolySet in, PolySet out, int flags) {
    __shared__ u64 sm[256 * 17];
    const int poly = pass_poly(flags), limb = pass_limb(flags);
    const PolyRef& Ro = out.p[poly];
    if (limb >= Ro.nlimbs) return;
    const int logn = t.logn;
    const int pi = prime_of(Ro, limb);
    const int cc = threadIdx.x & 15, w = threadIdx.x >> 4;
    const int col = blockIdx.x * 16 + cc;
    const u64* src = in.p[poly].ptr + ((size_t)limb << logn) + col;
    u64* dst = Ro.ptr + ((size_t)limb << logn) + col;
    const u64 q = __ldg(&t.primes[pi].q);
    const u64 q2 = 2 * q;
    const ulonglong2* tw = (INV ? t.inv : t.fwd) + ((size_t)pi << logn);
    const ulonglong2 NI = INV ? __ldg(&t.ninv[pi]) : make_ulonglong2(0, 0);
    const ulonglong2 NI1 = INV ? __ldg(&t.inv1ninv[pi]) : make_ulonglong2(0, 0);
    u64 x[16];
    if (!INV) {
        const bool lazy = q < kLazyBound;  // uniform over the CTA (one limb)
#pragma unroll
        for (int e = 0; e < 16; e++) x[e] = src[(size_t)((e << 4) | w) << LOGT];
        if (lazy) ntt16_round<false, 4, 0, true>(x, w, 0, tw, q, q2, NI, NI1);
        else ntt16_round<false, 4, 0>(x, w, 0, tw, q, q2, NI, NI1);
#pragma unroll
        for (int e = 0; e < 16; e++) sm[((e << 4) | w) * 17 + cc] = x[e];
        __syncthreads();
#pragma unroll
        for (int e = 0; e < 16; e++) x[e] = sm[((w << 4) | e) * 17 + cc];
        if (lazy) ntt16_round<false, 0, 0, true>(x, w << 4, 0, tw, q, q2, NI, NI1);
        else ntt16_round<false, 0, 0>(x, w << 4, 0, tw, q, q2, NI, NI1);
#pragma unroll
        for (int e = 0; e < 16; e++) dst[(size_t)((w << 4) | e) << LOGT] = x[e];
    } else {
#pragma unroll
        for (int e = 0; e < 16; e++) x[e] = src[(size_t)((w << 4) | e) << LOGT];
        ntt16_round<true, 0, 0>(x, w << 4, 0, tw, q, q2, NI, NI1);
#pragma unroll
        for (int e = 0; e < 16; e++) sm[((w << 4) | e) * 17 + cc] = x[e];
        __syncthreads();
#pragma unroll
        for (int e = 0; e < 16; e++) x[e] = sm[((e << 4) | w) * 17 + cc];
        ntt16_round<true, 4, 0, false, UNSCALED>(x, w, 0, tw, q, q2, NI, NI1);
#pragma unroll
        for (int e = 0; e < 16; e++)
            dst[(size_t)((e << 4) | w) << LOGT] = (flags & kPassFinal) && !UNSCALED ? canon4(x[e], q, q2) : x[e];
    }
}

// Canonical residue of x < 66q (the output range of the uncorrected forward stages) for a prime
// of s + 1 >= 25 bits, with r = floor(2^(s+32) / q) (= mu >> 32) and sh = s - 24.  The quotient
// is below 66, so one 32-bit high product estimates it: with xh = floor(x / 2^sh) < 2^32,
// est = floor(xh r / 2^56) is at most x/q and more than x/q - 2^-22, i.e. floor(x/q) or one
// less; x - est q then lies in [0, 2q) and one conditional subtraction finishes.
__device__ __forceinline__ u64 reduce_below66(u64 x, u64 q, u32 r, u32 sh) {
    const u32 xh = (u32)(x >> sh);
    const u32 est = __umulhi(xh, r) >> 24;
    const u64 v = x - (u64)est * q;
    return v >= q ? v - q : v;
}

// ---- lane-major copy of the twiddles of stages 12..15 ---------------------------------------
// In the round of stages 12..15 of a row pass, thread (row u, lane w) uses the 15 twiddles
// 2^(12+k) + u 2^(4+k) + w 2^k + j (k < 4, j < 2^k): row- and lane-specific, each read once.
// Read from the natural table, one warp load touches 32 cache lines for 16 bytes each.  The
// lane-major copy holds, per prime and row, [15 slots][16 lanes] (slot 2^k - 1 + j), so the 16
// lanes of a row read 256 contiguous bytes per load.
constexpr int kRowTwSlots = 15;
// The 16 rows' twiddles of stages 8..11 (row u: entry 2^(8+k) + u 2^k + j, k < 4, j < 2^k) into
// rt[16][15]: one 16-byte load and store for 240 of the 256 threads, made visible by the caller's
// next barrier.
__device__ __forceinline__ void stage_row_round1(const ulonglong2* __restrict__ tw, int u0, ulonglong2* rt, u64 pol) {
    const int t = threadIdx.x;
    if (t < 16 * 15) {
        const int cc = t / 15, e = t % 15;
        const int k = e >= 7 ? 3 : e >= 3 ? 2 : e >= 1 ? 1 : 0;
        const int j = e + 1 - (1 << k);
        rt[t] = ldg_pol(&tw[(1 << (8 + k)) + ((u0 + cc) << k) + j], pol);
    }
}
__device__ __forceinline__ const ulonglong2* lm_base(const ulonglong2* rows, int pi, int u, int w) {
    return rows + ((size_t)pi * 256 + u) * (kRowTwSlots * 16) + w;
}

// Forward stages 8..15 of the 16 rows of this CTA (limb `limb` of prime pi, rows read from
// src): canonical results are left in sm, row c2 point m at c2 * kRowStride + m + (m >> 4),
// after a barrier.
template <bool LM = false>
__device__ __forceinline__ void contig_fwd_rows(const DevTables& t, const u64* __restrict__ src, int pi, u64* sm) {
    const int logn = t.logn;
    const int w = threadIdx.x & 15, cc = threadIdx.x >> 4;
    const int u = blockIdx.x * 16 + cc;
    const u64 q = __ldg(&t.primes[pi].q);
    const u64 q2 = 2 * q;
    const ulonglong2* tw = t.fwd + ((size_t)pi << logn);
    const ulonglong2 NI = make_ulonglong2(0, 0);
    const ulonglong2* lm = LM ? lm_base(t.fwd_rows, pi, u, w) : nullptr;
    const u64 pol = tw_policy(t.ntt_order & 2);
    __shared__ ulonglong2 rt[16 * 15];  // LM: twiddles of stages 8..11 of the 16 rows
    u64* my = sm + cc * kRowStride;
    u64 x[16];
    const bool lazy = q < kLazyBound;  // uniform over the CTA (one limb)
    if (LM) stage_row_round1(tw, blockIdx.x * 16, rt, pol);
#pragma unroll
    for (int e = 0; e < 16; e++) x[e] = src[((size_t)u << 8) | (e << 4) | w];
    if (LM) __syncthreads();
    if (lazy) ntt16_round<false, 4, 8, true, false, false, LM>(x, w, u, tw, q, q2, NI, NI, nullptr, rt + cc * 15);
    else ntt16_round<false, 4, 8, false, false, false, LM>(x, w, u, tw, q, q2, NI, NI, nullptr, rt + cc * 15);
#pragma unroll
    for (int e = 0; e < 16; e++) my[e * 17 + w] = x[e];  // point e*16 + w
    __syncthreads();
#pragma unroll
    for (int e = 0; e < 16; e++) x[e] = my[w * 17 + e];  // point w*16 + e
    if (lazy) {
        ntt16_round<false, 0, 8, true, false, LM>(x, w << 4, u, tw, q, q2, NI, NI, lm, nullptr, pol);
        const u32 ps = __ldg(&t.primes[pi].s);
        if (ps >= 24) {
            const u32 r = (u32)(__ldg(&t.primes[pi].mu) >> 32);
#pragma unroll
            for (int e = 0; e < 16; e++) my[w * 17 + e] = reduce_below66(x[e], q, r, ps - 24);
        } else {  // primes below 2^25: Shoup multiplication by 1 with 1' = floor(2^64 / q) = mu >> s
            const u64 one_p = __ldg(&t.primes[pi].mu) >> ps;
#pragma unroll
            for (int e = 0; e < 16; e++) {
                const u64 v = x[e] - mulhi(x[e], one_p) * q;
                my[w * 17 + e] = v >= q ? v - q : v;
            }
        }
    } else {
        ntt16_round<false, 0, 8, false, false, LM>(x, w << 4, u, tw, q, q2, NI, NI, lm, nullptr, pol);
#pragma unroll
        for (int e = 0; e < 16; e++) my[w * 17 + e] = canon8(x[e], q, q2);
    }
    __syncthreads();
}

template <bool INV, int MINB, bool LM = false>
__global__ void __launch_bounds__(256, MINB) k_ntt8_contig(DevTables t, PolySet in, PolySet out, int flags) {
    __shared__ u64 sm[16 * kRowStride];
    const int poly = pass_poly(flags), limb = pass_limb(flags);
    const PolyRef& Ro = out.p[poly];
    if (limb >= Ro.nlimbs) return;
    const int logn = t.logn;
    const int pi = prime_of(Ro, limb);
    const u64* src = in.p[poly].ptr + ((size_t)limb << logn);
    u64* dst = Ro.ptr + ((size_t)limb << logn);
    if (!INV) {
        contig_fwd_rows<LM>(t, src, pi, sm);
#pragma unroll
        for (int k = 0; k < 16; k++) {
            const int f = threadIdx.x + 256 * k;
            const int c2 = f >> 8, m = f & 255;
            dst[((size_t)(blockIdx.x * 16 + c2) << 8) | m] = sm[c2 * kRowStride + m + (m >> 4)];
        }
        return;
    }
    const int w = threadIdx.x & 15, cc = threadIdx.x >> 4;
    const int u = blockIdx.x * 16 + cc;
    const u64 q = __ldg(&t.primes[pi].q);
    const u64 q2 = 2 * q;
    const ulonglong2* tw = t.inv + ((size_t)pi << logn);
    const ulonglong2 NI = __ldg(&t.ninv[pi]);
    const ulonglong2 NI1 = __ldg(&t.inv1ninv[pi]);
    const ulonglong2* lm = LM ? lm_base(t.inv_rows, pi, u, w) : nullptr;
    const u64 pol = tw_policy(t.ntt_order & 2);
    u64* my = sm + cc * kRowStride;
    u64 x[16];
#pragma unroll
    for (int k = 0; k < 16; k++) {
        const int f = threadIdx.x + 256 * k;
        const int c2 = f >> 8, m = f & 255;
        sm[c2 * kRowStride + m + (m >> 4)] = src[((size_t)(blockIdx.x * 16 + c2) << 8) | m];
    }
    __syncthreads();
#pragma unroll
    for (int e = 0; e < 16; e++) x[e] = my[w * 17 + e];  // point w*16 + e
    ntt16_round<true, 0, 8, false, false, LM>(x, w << 4, u, tw, q, q2, NI, NI1, lm, nullptr, pol);
#pragma unroll
    for (int e = 0; e < 16; e++) my[w * 17 + e] = x[e];
    __syncthreads();
#pragma unroll
    for (int e = 0; e < 16; e++) x[e] = my[e * 17 + w];  // point e*16 + w
    ntt16_round<true, 4, 8>(x, w, u, tw, q, q2, NI, NI1);
#pragma unroll
    for (int e = 0; e < 16; e++)
        dst[((size_t)u << 8) | (e << 4) | w] = (flags & kPassFinal) ? canon4(x[e], q, q2) : x[e];
}

// Forward stages 8..15 fused with the ModDown epilogue: for the canonical transform value v,
// out = (x + c - v) s mod q (+ acc when the polynomial has one), with per-limb constants
// {c, s, s'} (Shoup) at consts[3 limb].  The rows of `in` hold the output of stages 0..7.
template <int MINB, bool LM = false>
__global__ void __launch_bounds__(256, MINB) k_ntt8_contig_epi(DevTables t, PolySet in, NttEpi e, int flags) {
    __shared__ u64 sm[16 * kRowStride];
    const int poly = pass_poly(flags), limb = pass_limb(flags);
    const PolyRef& Ri = in.p[poly];
    if (limb >= Ri.nlimbs) return;
    const int logn = t.logn;
    const int pi = prime_of(Ri, limb);
    const size_t base = (size_t)limb << logn;
    const u64* __restrict__ xs = e.x.p[poly].ptr + base;
    const u64* __restrict__ as = e.acc.p[poly].ptr;  // null: no accumulator for this polynomial
    u64* __restrict__ os = e.out.p[poly].ptr + base;
    if (flags & kPassPrefetch) {
        // ask L2 for this CTA's tile of the epilogue operands (one 128-byte line per thread and
        // operand: 16 rows x 256 words) so that their DRAM reads overlap the transform
        const int f = threadIdx.x * 16;
        const size_t j = ((size_t)(blockIdx.x * 16 + (f >> 8)) << 8) | (f & 255);
        asm volatile("prefetch.global.L2 [%0];" ::"l"(xs + j));
        if (as) asm volatile("prefetch.global.L2 [%0];" ::"l"(as + base + j));
    }
    contig_fwd_rows<LM>(t, Ri.ptr + base, pi, sm);
    const u64 q = __ldg(&t.primes[pi].q);
    const u64 c = __ldg(&e.consts[3 * limb]), s = __ldg(&e.consts[3 * limb + 1]), sp = __ldg(&e.consts[3 * limb + 2]);
    // each thread: two adjacent points (16-byte loads and stores) of rows r0, r0 + 2, ..., r0 + 14;
    // the operands of four rows are loaded before any is used, so that more bytes are in flight
    // (the transform's registers are free by now).  An even point m and m + 1 share their
    // 16-point group, so their transform values are adjacent in shared memory.
    const int m = 2 * (threadIdx.x & 127), r0 = threadIdx.x >> 7;
#pragma unroll
    for (int h = 0; h < 2; h++) {
        ulonglong2 xv[4], av[4];
#pragma unroll
        for (int i = 0; i < 4; i++) {
            const size_t j = ((size_t)(blockIdx.x * 16 + r0 + 2 * (4 * h + i)) << 8) | m;
            xv[i] = *reinterpret_cast<const ulonglong2*>(xs + j);
            if (as) av[i] = *reinterpret_cast<const ulonglong2*>(as + base + j);
        }
#pragma unroll
        for (int i = 0; i < 4; i++) {
            const int c2 = r0 + 2 * (4 * h + i);
            const size_t j = ((size_t)(blockIdx.x * 16 + c2) << 8) | m;
            const u64* v = sm + c2 * kRowStride + m + (m >> 4);
            ulonglong2 r;
            r.x = mul_shoup(submod(addmod(xv[i].x, c, q), v[0], q), s, sp, q);
            r.y = mul_shoup(submod(addmod(xv[i].y, c, q), v[1], q), s, sp, q);
            if (as) {
                r.x = addmod(r.x, av[i].x, q);
                r.y = addmod(r.y, av[i].y, q);
            }
            *reinterpret_cast<ulonglong2*>(os + j) = r;
        }
    }
}

template <int MINB>
static void prepare_twopass(void) {
    if (MINB == 4 && first_on_device((const void*)&k_ntt8_contig_epi<MINB, true>)) {
        // four CTAs of 35 KB shared memory: a carveout that fits them, the rest L1
        const int co = 64;
        PFT_CUDA(cudaFuncSetAttribute(k_ntt8_strided<false, 8, MINB>, cudaFuncAttributePreferredSharedMemoryCarveout, co));
        PFT_CUDA(cudaFuncSetAttribute(k_ntt8_strided<true, 8, MINB>, cudaFuncAttributePreferredSharedMemoryCarveout, co));
        PFT_CUDA(cudaFuncSetAttribute(k_ntt8_strided<true, 8, MINB, true>,
                                      cudaFuncAttributePreferredSharedMemoryCarveout, co));
        PFT_CUDA(cudaFuncSetAttribute(k_ntt8_contig<false, MINB, true>, cudaFuncAttributePreferredSharedMemoryCarveout, co));
        PFT_CUDA(cudaFuncSetAttribute(k_ntt8_contig<true, MINB, true>, cudaFuncAttributePreferredSharedMemoryCarveout, co));
        PFT_CUDA(cudaFuncSetAttribute(k_ntt8_contig_epi<MINB, true>, cudaFuncAttributePreferredSharedMemoryCarveout, co));
    }
}

template <bool INV, int MINB, bool LM>
static void launch_contig(const DevTables& t, const PolySet& in, const PolySet& out, int flags, cudaStream_t st) {
    dim3 grid(16, (unsigned)out.max_limbs, (unsigned)out.count);
    k_ntt8_contig<INV, MINB, LM><<<grid, 256, 0, st>>>(t, in, out, flags);
}
// flags of the second pass of a transform over the same data
static int second_pass(const DevTables& t, int flags) { return flags | ((t.ntt_order & 1) ? kPassReverse : 0); }

template <int MINB, bool LM>
static void launch_ntt16_twopass_v(const DevTables& t, const PolySet& in, const PolySet& out, bool inverse,
                                   cudaStream_t st) {
    prepare_twopass<MINB>();
    dim3 grid(16, (unsigned)out.max_limbs, (unsigned)out.count);  // 256 sub-transforms / 16 per CTA
    const double work = set_limbs(out) * (double)(t.n / 2) * 8;
    if (!inverse) {
        {
            PFT_PROF("ntt.fwd.strided", st, work);
            k_ntt8_strided<false, 8, MINB><<<grid, 256, 0, st>>>(t, in, out, 0);
        }
        PFT_LAUNCH_CHECK("ntt pass A");
        {
            PFT_PROF("ntt.fwd.contig", st, work);
            launch_contig<false, MINB, LM>(t, out, out, second_pass(t, kPassFinal), st);
        }
        PFT_LAUNCH_CHECK("ntt pass B");
    } else {
        {
            PFT_PROF("ntt.inv.contig", st, work);
            launch_contig<true, MINB, LM>(t, in, out, 0, st);
        }
        PFT_LAUNCH_CHECK("intt pass B");
        {
            PFT_PROF("ntt.inv.strided", st, work);
            k_ntt8_strided<true, 8, MINB><<<grid, 256, 0, st>>>(t, out, out, second_pass(t, kPassFinal));
        }
        PFT_LAUNCH_CHECK("intt pass A");
    }
}

// variant 0: 3 CTAs per SM; 1: 4 CTAs per SM (both with the lane-major row twiddles)
static void launch_ntt16_twopass(const DevTables& t, const PolySet& in, const PolySet& out, bool inverse, int v16,
                                 cudaStream_t st) {
    if (v16 == 1) launch_ntt16_twopass_v<4, true>(t, in, out, inverse, st);
    else launch_ntt16_twopass_v<3, true>(t, in, out, inverse, st);
}

template <int MINB, bool LM>
static void launch_ntt16_inverse_unscaled_v(const DevTables& t, const PolySet& in, const PolySet& out,
                                            cudaStream_t st) {
    prepare_twopass<MINB>();
    dim3 grid(16, (unsigned)out.max_limbs, (unsigned)out.count);
    const double work = set_limbs(out) * (double)(t.n / 2) * 8;
    {
        PFT_PROF("ntt.inv.contig", st, work);
        launch_contig<true, MINB, LM>(t, in, out, 0, st);
    }
    PFT_LAUNCH_CHECK("intt pass B");
    {
        PFT_PROF("ntt.inv.strided", st, work);
        k_ntt8_strided<true, 8, MINB, true><<<grid, 256, 0, st>>>(t, out, out, second_pass(t, kPassFinal));
    }
    PFT_LAUNCH_CHECK("intt pass A (unscaled)");
}

template <int MINB, bool LM>
static void launch_ntt16_epi_v(const DevTables& t, const PolySet& io, const NttEpi& e, cudaStream_t st) {
    prepare_twopass<MINB>();
    dim3 grid(16, (unsigned)io.max_limbs, (unsigned)io.count);
    const double work = set_limbs(io) * (double)(t.n / 2) * 8;
    {
        PFT_PROF("ntt.fwd.strided", st, work);
        k_ntt8_strided<false, 8, MINB><<<grid, 256, 0, st>>>(t, io, io, 0);
    }
    PFT_LAUNCH_CHECK("ntt pass A");
    {
        // named apart from the plain transform launches: it also moves the epilogue's operands
        PFT_PROF("epi.ntt_moddown", st, work);
        k_ntt8_contig_epi<MINB, LM><<<grid, 256, 0, st>>>(t, io, e,
                                                           second_pass(t, (t.ntt_order & 4) ? kPassPrefetch : 0));
    }
    PFT_LAUNCH_CHECK("ntt pass B + ModDown epilogue");
}

template <bool INV, int MINB>
static void launch_ntt16_cluster_v(const DevTables& t, const PolySet& in, const PolySet& out, cudaStream_t st) {
    const size_t smem = (size_t)256 * kN16Stride * sizeof(u64);
    if (first_on_device((const void*)&k_ntt16_cluster<INV, MINB>))
        PFT_CUDA(cudaFuncSetAttribute(k_ntt16_cluster<INV, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
    dim3 grid(8, (unsigned)out.max_limbs, (unsigned)out.count);
    PFT_PROF(INV ? "ntt.inv.cluster" : "ntt.fwd.cluster", st, set_limbs(out) * (double)(t.n / 2) * 16);
    k_ntt16_cluster<INV, MINB><<<grid, 512, smem, st>>>(t, in, out);
    PFT_LAUNCH_CHECK("ntt16 cluster");
}

template <bool INV>
static void launch_ntt16_cluster(const DevTables& t, const PolySet& in, const PolySet& out, cudaStream_t st) {
    launch_ntt16_cluster_v<INV, 2>(t, in, out, st);
}

// N = 2^16 variant: the context's choice (pft_autotune), unless PFT_NTT16 names one
// (twopass, twopass4, cluster, generic).
// the N = 2^16 kernel family of a launch of `limbs` limbs: the environment's choice, else the
// autotuned plan of the launch's size bucket, else the context's fixed variant
static int ntt16_variant(const DevTables& t, double limbs = -1) {
    static int env = -2;
    if (env == -2) {
        const char* e = getenv("PFT_NTT16");
        env = !e ? -1
                 : strcmp(e, "twopass") == 0  ? 0
                 : strcmp(e, "twopass4") == 0 ? 1
                 : strcmp(e, "cluster") == 0  ? 2
                 : strcmp(e, "generic") == 0  ? 3
                                              : -1;
    }
    if (env >= 0) return env;
    if (limbs >= 0) {
        const int k = t.plan[ntt_bucket(limbs)].kind;
        if (k >= 0) return k;
    }
    return t.ntt_variant;
}

template <int S, int C, bool INV>
__global__ void __launch_bounds__(C*(1 << (S - 4)))
    k_ntt_pass(DevTables t, PolySet in, PolySet out, int s0, int logT, int is_final) {
    constexpr int TPS = 1 << (S - 4);  // threads per sub-transform
    constexpr int NT = C * TPS;
    constexpr int SUB = (1 << S) + (1 << (S - 4));  // padded stride (1 word per 16)
    extern __shared__ u64 sm[];

    const int poly = blockIdx.z, limb = blockIdx.y;
    const PolyRef& Ro = out.p[poly];
    if (limb >= Ro.nlimbs) return;
    const PolyRef& Ri = in.p[poly];
    const int pi = prime_of(Ro, limb);
    const int logn = t.logn;
    const u64* src = Ri.ptr + ((size_t)limb << logn);
    u64* dst = Ro.ptr + ((size_t)limb << logn);
    const u64 q = __ldg(&t.primes[pi].q);
    const u64 q2 = 2 * q;
    const ulonglong2* tw = (INV ? t.inv : t.fwd) + ((size_t)pi << logn);
    const int T = 1 << logT;
    const int ubase = blockIdx.x * C;

    // ---- coalesced load into shared memory
    for (int f = threadIdx.x; f < (C << S); f += NT) {
        int cc, mid;
        if (logT > 0) {
            cc = f % C;
            mid = f / C;
        } else {
            cc = f >> S;
            mid = f & ((1 << S) - 1);
        }
        const int u = ubase + cc;
        const size_t j = ((size_t)(u >> logT) << (S + logT)) + ((size_t)mid << logT) + (u & (T - 1));
        sm[cc * SUB + mid + (mid >> 4)] = src[j];
    }
    __syncthreads();

    const int w = threadIdx.x % TPS, cc = threadIdx.x / TPS;
    const int hi = (ubase + cc) >> logT;
    u64* my = sm + cc * SUB;
    u64 x[16];

    if (!INV) {
#pragma unroll
        for (int hb = S - 1; hb >= 0; hb -= 4) {
            const int r = hb + 1 < 4 ? hb + 1 : 4;
            const int w0 = hb - 3 > 0 ? hb - 3 : 0;
            const int base = ((w >> w0) << (w0 + 4)) | (w & ((1 << w0) - 1));
#pragma unroll
            for (int e = 0; e < 16; e++) {
                const int mid = base | (e << w0);
                x[e] = my[mid + (mid >> 4)];
            }
#pragma unroll
            for (int lb = 3; lb >= 0; lb--) {
                const int p = w0 + lb;
                if (p > hb || p < hb - r + 1) continue;
                const int s = s0 + (S - 1 - p);
#pragma unroll
                for (int e = 0; e < 16; e++) {
                    if (e & (1 << lb)) continue;
                    const int mid = base | (e << w0);
                    const int i = (hi << (S - p - 1)) + (mid >> (p + 1));
                    ct_bfly<false>(x[e], x[e | (1 << lb)], __ldg(&tw[(1 << s) + i]), q, q2);
                }
            }
#pragma unroll
            for (int e = 0; e < 16; e++) {
                const int mid = base | (e << w0);
                my[mid + (mid >> 4)] = x[e];
            }
            __syncthreads();
        }
    } else {
        const ulonglong2 NI = __ldg(&t.ninv[pi]);
        const ulonglong2 NI1 = __ldg(&t.inv1ninv[pi]);
#pragma unroll
        for (int lb0 = 0; lb0 < S; lb0 += 4) {
            const int r = S - lb0 < 4 ? S - lb0 : 4;
            const int w0 = lb0 < S - 4 ? lb0 : S - 4;
            const int base = ((w >> w0) << (w0 + 4)) | (w & ((1 << w0) - 1));
#pragma unroll
            for (int e = 0; e < 16; e++) {
                const int mid = base | (e << w0);
                x[e] = my[mid + (mid >> 4)];
            }
#pragma unroll
            for (int lb = 0; lb < 4; lb++) {
                const int p = w0 + lb;
                if (p < lb0 || p > lb0 + r - 1) continue;
                const int s = s0 + (S - 1 - p);
#pragma unroll
                for (int e = 0; e < 16; e++) {
                    if (e & (1 << lb)) continue;
                    if (s == 0) {  // last inverse stage: fold N^-1 into both outputs
                        u64 Sm = x[e] + x[e | (1 << lb)];
                        if (Sm >= 2 * q2) Sm -= 2 * q2;
                        const u64 D = x[e] - x[e | (1 << lb)] + 2 * q2;
                        x[e] = mul_shoup_lazy(Sm, NI.x, NI.y, q);
                        x[e | (1 << lb)] = mul_shoup_lazy(D, NI1.x, NI1.y, q);
                    } else {
                        const int mid = base | (e << w0);
                        const int i = (hi << (S - p - 1)) + (mid >> (p + 1));
                        gs_bfly(x[e], x[e | (1 << lb)], __ldg(&tw[(1 << s) + i]), q, q2);
                    }
                }
            }
#pragma unroll
            for (int e = 0; e < 16; e++) {
                const int mid = base | (e << w0);
                my[mid + (mid >> 4)] = x[e];
            }
            __syncthreads();
        }
    }

    // ---- coalesced store (canonical residues after the last pass)
    for (int f = threadIdx.x; f < (C << S); f += NT) {
        int c2, mid;
        if (logT > 0) {
            c2 = f % C;
            mid = f / C;
        } else {
            c2 = f >> S;
            mid = f & ((1 << S) - 1);
        }
        const int u = ubase + c2;
        const size_t j = ((size_t)(u >> logT) << (S + logT)) + ((size_t)mid << logT) + (u & (T - 1));
        u64 v = sm[c2 * SUB + mid + (mid >> 4)];
        if (is_final) v = canon8(v, q, q2);  // forward values below 8q, inverse below 2q
        dst[j] = v;
    }
}

template <int S, int C, bool INV>
static void launch_pass(const DevTables& t, const PolySet& in, const PolySet& out, int s0, int is_final,
                        cudaStream_t st) {
    constexpr int TPS = 1 << (S - 4);
    constexpr int SUB = (1 << S) + (1 << (S - 4));
    const size_t smem = (size_t)C * SUB * sizeof(u64);
    if (first_on_device((const void*)&k_ntt_pass<S, C, INV>))
        PFT_CUDA(cudaFuncSetAttribute(k_ntt_pass<S, C, INV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int logT = t.logn - s0 - S;
    dim3 grid((unsigned)((t.n >> S) / C), (unsigned)out.max_limbs, (unsigned)out.count);
    PFT_PROF(INV ? (logT > 0 ? "ntt.inv.strided" : "ntt.inv.contig") : (logT > 0 ? "ntt.fwd.strided" : "ntt.fwd.contig"),
             st, set_limbs(out) * (double)(t.n / 2) * S);
    k_ntt_pass<S, C, INV><<<grid, C * TPS, smem, st>>>(t, in, out, s0, logT, is_final);
    PFT_LAUNCH_CHECK("ntt pass");
}

// One pass of a generic plan: the (S, C) shapes the autotuner searches (256 threads per CTA, and
// 128 for 8 stages with 8 sub-transforms per CTA).
template <bool INV>
static void launch_generic_pass(const DevTables& t, const PolySet& in, const PolySet& out, int S, int C, int s0,
                                int is_final, cudaStream_t st) {
    switch (S * 1000 + C) {
        case 5128: launch_pass<5, 128, INV>(t, in, out, s0, is_final, st); break;
        case 6064: launch_pass<6, 64, INV>(t, in, out, s0, is_final, st); break;
        case 7032: launch_pass<7, 32, INV>(t, in, out, s0, is_final, st); break;
        case 7016: launch_pass<7, 16, INV>(t, in, out, s0, is_final, st); break;
        case 8016: launch_pass<8, 16, INV>(t, in, out, s0, is_final, st); break;
        case 8008: launch_pass<8, 8, INV>(t, in, out, s0, is_final, st); break;
        case 9008: launch_pass<9, 8, INV>(t, in, out, s0, is_final, st); break;
        case 10004: launch_pass<10, 4, INV>(t, in, out, s0, is_final, st); break;
        default: fail(PFT_ERR_ARG, "internal: no kernel for this transform pass shape");
    }
}
// A generic plan: forward passes in order (stage offsets accumulate), inverse in reverse order.
static void run_generic(const DevTables& t, const DevTables::Plan& p, const PolySet& in, const PolySet& out,
                        bool inverse, cudaStream_t st) {
    int s0[3] = {0, 0, 0};
    for (int i = 1; i < p.npass; i++) s0[i] = s0[i - 1] + p.S[i - 1];
    if (!inverse) {
        for (int i = 0; i < p.npass; i++)
            launch_generic_pass<false>(t, i == 0 ? in : out, out, p.S[i], p.C[i], s0[i], i == p.npass - 1, st);
    } else {
        for (int i = p.npass - 1; i >= 0; i--)
            launch_generic_pass<true>(t, i == p.npass - 1 ? in : out, out, p.S[i], p.C[i], s0[i], i == 0, st);
    }
}

int ntt_candidates(int logn, DevTables::Plan* out, const char** names, int cap) {
    struct Cand {
        const char* name;
        DevTables::Plan p;
    };
    static const Cand c16[] = {
        {"two-pass 8+8 (register rounds), 3 CTAs/SM", {0, 0, {0, 0, 0}, {0, 0, 0}}},
        {"two-pass 8+8 (register rounds), 4 CTAs/SM", {1, 0, {0, 0, 0}, {0, 0, 0}}},
        {"one launch, 8-CTA cluster (DSMEM exchange)", {2, 0, {0, 0, 0}, {0, 0, 0}}},
        {"staged 8+8, 16 sub-transforms/CTA", {3, 2, {8, 8, 0}, {16, 16, 0}}},
        {"staged 8+8, 8 sub-transforms/CTA", {3, 2, {8, 8, 0}, {8, 8, 0}}},
        {"staged 6+10", {3, 2, {6, 10, 0}, {64, 4, 0}}},
        {"staged 10+6", {3, 2, {10, 6, 0}, {4, 64, 0}}},
        {"staged 7+9", {3, 2, {7, 9, 0}, {32, 8, 0}}},
        {"staged 9+7", {3, 2, {9, 7, 0}, {8, 32, 0}}},
        {"staged 5+5+6 (three passes)", {3, 3, {5, 5, 6}, {128, 128, 64}}},
    };
    static const Cand c15[] = {
        {"staged 8+7", {3, 2, {8, 7, 0}, {16, 16, 0}}},
        {"staged 7+8", {3, 2, {7, 8, 0}, {16, 16, 0}}},
        {"staged 9+6", {3, 2, {9, 6, 0}, {8, 64, 0}}},
        {"staged 6+9", {3, 2, {6, 9, 0}, {64, 8, 0}}},
        {"staged 5+5+5 (three passes)", {3, 3, {5, 5, 5}, {128, 128, 128}}},
    };
    const Cand* c = logn == 16 ? c16 : logn == 15 ? c15 : nullptr;
    const int n = logn == 16 ? (int)(sizeof(c16) / sizeof(c16[0])) : logn == 15 ? (int)(sizeof(c15) / sizeof(c15[0])) : 0;
    for (int i = 0; i < n && i < cap; i++) {
        if (out) out[i] = c[i].p;
        if (names) names[i] = c[i].name;
    }
    return n;
}

template <bool INV>
static void run_single(const DevTables& t, const PolySet& in, const PolySet& out, cudaStream_t st) {
    switch (t.logn) {
        case 4: launch_pass<4, 1, INV>(t, in, out, 0, 1, st); break;
        case 5: launch_pass<5, 1, INV>(t, in, out, 0, 1, st); break;
        case 6: launch_pass<6, 1, INV>(t, in, out, 0, 1, st); break;
        case 7: launch_pass<7, 1, INV>(t, in, out, 0, 1, st); break;
        case 8: launch_pass<8, 1, INV>(t, in, out, 0, 1, st); break;
        case 9: launch_pass<9, 1, INV>(t, in, out, 0, 1, st); break;
        case 10: launch_pass<10, 1, INV>(t, in, out, 0, 1, st); break;
        case 11: launch_pass<11, 1, INV>(t, in, out, 0, 1, st); break;
        case 12: launch_pass<12, 1, INV>(t, in, out, 0, 1, st); break;
        case 13: launch_pass<13, 1, INV>(t, in, out, 0, 1, st); break;
        case 14: launch_pass<14, 1, INV>(t, in, out, 0, 1, st); break;
        default: fail(PFT_ERR_ARG, "unsupported ring degree");
    }
}

static void run(const DevTables& t, const PolySet& in, const PolySet& out, bool inverse, cudaStream_t st) {
    if (out.count == 0) return;
    if (t.logn <= 14) {
        if (inverse) run_single<true>(t, in, out, st);
        else run_single<false>(t, in, out, st);
        return;
    }
    const DevTables::Plan& pl = t.plan[ntt_bucket(set_limbs(out))];
    const int v16 = t.logn == 16 ? ntt16_variant(t, set_limbs(out)) : (pl.kind == 3 ? 3 : -1);
    if (v16 == 3 && pl.kind == 3) {  // a generic plan chosen for this launch size
        run_generic(t, pl, in, out, inverse, st);
        return;
    }
    if (v16 == 0 || v16 == 1) {
        launch_ntt16_twopass(t, in, out, inverse, v16, st);
    } else if (v16 == 2) {
        if (!inverse) launch_ntt16_cluster<false>(t, in, out, st);
        else launch_ntt16_cluster<true>(t, in, out, st);
    } else if (t.logn == 16) {
        if (!inverse) {
            launch_pass<8, 16, false>(t, in, out, 0, 0, st);   // stages 0..7, stride 256
            launch_pass<8, 16, false>(t, out, out, 8, 1, st);  // stages 8..15, contiguous
        } else {
            launch_pass<8, 16, true>(t, in, out, 8, 0, st);
            launch_pass<8, 16, true>(t, out, out, 0, 1, st);
        }
    } else if (t.logn == 15) {
        if (!inverse) {
            launch_pass<8, 16, false>(t, in, out, 0, 0, st);
            launch_pass<7, 16, false>(t, out, out, 8, 1, st);
        } else {
            launch_pass<7, 16, true>(t, in, out, 8, 0, st);
            launch_pass<8, 16, true>(t, out, out, 0, 1, st);
        }
    } else {
        fail(PFT_ERR_ARG, "unsupported ring degree");
    }
}

void ntt_forward(const DevTables& t, const PolySet& in, const PolySet& out, cudaStream_t st) {
    run(t, in, out, false, st);
}
// Register-only ceiling of the transform's butterfly: each thread runs `rounds` rounds of two
// stages of 8 independent Cooley-Tukey butterflies (the ct_bfly of the transforms, twiddle in
// registers, no memory traffic); one word is written only if the data take a value they cannot
// reach, which keeps the work.
template <bool LAZY>
__global__ void __launch_bounds__(256) k_bfly_ceiling(u64* sink, u64 q, ulonglong2 W, int rounds) {
    u64 x[16];
#pragma unroll
    for (int i = 0; i < 16; i++) x[i] = ((u64)threadIdx.x * 16 + i + blockIdx.x) % q;
    const ulonglong2 Wt = make_ulonglong2(W.x, W.y);
    const u64 q2 = 2 * q;
    for (int k = 0; k < rounds; k++) {
#pragma unroll
        for (int i = 0; i < 8; i++) ct_bfly<LAZY>(x[i], x[i + 8], Wt, q, q2);
#pragma unroll
        for (int i = 0; i < 8; i++) ct_bfly<LAZY>(x[2 * i], x[2 * i + 1], Wt, q, q2);
    }
    u64 acc = 0;
#pragma unroll
    for (int i = 0; i < 16; i++) acc ^= x[i];
    if (acc == ~0ull) sink[0] = acc;  // never true for the corrected form (values below 8q < 2^63)
}

double bfly_ceiling(const DevTables& t, cudaStream_t st) {
    int dev = 0, sms = 0;
    PFT_CUDA(cudaGetDevice(&dev));
    PFT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    DPrime p0;
    PFT_CUDA(cudaMemcpy(&p0, t.primes, sizeof(DPrime), cudaMemcpyDeviceToHost));
    ulonglong2 W0;
    PFT_CUDA(cudaMemcpy(&W0, t.fwd + 1, sizeof(W0), cudaMemcpyDeviceToHost));  // a twiddle of q_0
    u64* sink = nullptr;
    PFT_CUDA(cudaMalloc(&sink, 8));
    cudaEvent_t a, b;
    PFT_CUDA(cudaEventCreate(&a));
    PFT_CUDA(cudaEventCreate(&b));
    const int grid = sms * 4, rounds = 2000;
    // the corrected form (primes of 57 bits and more) and the uncorrected one (below 2^57; the
    // register data just wrap around here, which costs the same): the faster is the ceiling
    double best = 0;
    for (int lazy = 0; lazy < 2; lazy++) {
        auto kern = lazy ? k_bfly_ceiling<true> : k_bfly_ceiling<false>;
        kern<<<grid, 256, 0, st>>>(sink, p0.q, W0, 16);  // warm-up
        PFT_CUDA(cudaEventRecord(a, st));
        kern<<<grid, 256, 0, st>>>(sink, p0.q, W0, rounds);
        PFT_CUDA(cudaEventRecord(b, st));
        PFT_CUDA(cudaEventSynchronize(b));
        float ms = 0;
        PFT_CUDA(cudaEventElapsedTime(&ms, a, b));
        best = std::max(best, (double)grid * 256 * rounds * 16 / (ms / 1e3));
    }
    PFT_CUDA(cudaEventDestroy(a));
    PFT_CUDA(cudaEventDestroy(b));
    PFT_CUDA(cudaFree(sink));
    return best;
}

// Issue rates of the two forms of 32-bit integer multiply the butterflies use: the low-word
// multiply-add (mad.lo) and the forms that produce a high word (mad.hi, mad.wide).  Each thread
// runs 8 independent chains of one form; the result word is written only for a value the
// chains cannot reach, which keeps the work.  (Written as single PTX multiply-adds, the
// high-word form measured slower, 24.2 against 28.1 per SM and clock: the faster forms below
// give the higher, stricter bound.)
template <int FORM>
__global__ void __launch_bounds__(256) k_mul_rate(u32* sink, u32 a, u32 b, int rounds) {
    u32 x[8];
    u64 y[8];
#pragma unroll
    for (int i = 0; i < 8; i++) {
        x[i] = threadIdx.x * 8 + i + blockIdx.x;
        y[i] = x[i];
    }
    for (int k = 0; k < rounds; k++) {
#pragma unroll
        for (int i = 0; i < 8; i++) {
            if (FORM == 0) x[i] = x[i] * a + b;
            if (FORM == 1) x[i] = __umulhi(x[i], a) + b;
            if (FORM == 2) y[i] = (u64)(u32)y[i] * a + y[i];
        }
    }
    u32 acc = 0;
#pragma unroll
    for (int i = 0; i < 8; i++) acc ^= x[i] ^ (u32)y[i] ^ (u32)(y[i] >> 32);
    if (acc == 0x9e3779b9u) sink[0] = acc;
}

void mul_rates(cudaStream_t st, double* lo, double* hi, double* wide) {
    int dev = 0, sms = 0;
    PFT_CUDA(cudaGetDevice(&dev));
    PFT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    u32* sink = nullptr;
    PFT_CUDA(cudaMalloc(&sink, 64));
    cudaEvent_t a, b;
    PFT_CUDA(cudaEventCreate(&a));
    PFT_CUDA(cudaEventCreate(&b));
    const int grid = sms * 8, rounds = 8000;
    double* outs[3] = {lo, hi, wide};
    for (int form = 0; form < 3; form++) {
        auto kern = form == 0 ? k_mul_rate<0> : form == 1 ? k_mul_rate<1> : k_mul_rate<2>;
        kern<<<grid, 256, 0, st>>>(sink, 3, 5, 16);  // warm-up
        PFT_CUDA(cudaEventRecord(a, st));
        kern<<<grid, 256, 0, st>>>(sink, 3, 5, rounds);
        PFT_CUDA(cudaEventRecord(b, st));
        PFT_CUDA(cudaEventSynchronize(b));
        float ms = 0;
        PFT_CUDA(cudaEventElapsedTime(&ms, a, b));
        if (outs[form]) *outs[form] = (double)grid * 256 * rounds * 8 / (ms / 1e3);
    }
    PFT_CUDA(cudaEventDestroy(a));
    PFT_CUDA(cudaEventDestroy(b));
    PFT_CUDA(cudaFree(sink));
}

bool ntt_inverse_unscaled(const DevTables& t, const PolySet& in, const PolySet& out, cudaStream_t st) {
    if (out.count == 0) return true;
    if (t.logn != 16) return false;
    const int v16 = ntt16_variant(t, set_limbs(out));
    if (v16 != 0 && v16 != 1) return false;
    if (v16 == 1) launch_ntt16_inverse_unscaled_v<4, true>(t, in, out, st);
    else launch_ntt16_inverse_unscaled_v<3, true>(t, in, out, st);
    return true;
}

bool ntt_forward_epilogue(const DevTables& t, const PolySet& io, const NttEpi& e, cudaStream_t st) {
    if (io.count == 0) return true;
    if (t.logn != 16) return false;
    const int v16 = ntt16_variant(t, set_limbs(io));
    if (v16 != 0 && v16 != 1) return false;
    if (v16 == 1) launch_ntt16_epi_v<4, true>(t, io, e, st);
    else launch_ntt16_epi_v<3, true>(t, io, e, st);
    return true;
}
void ntt_inverse(const DevTables& t, const PolySet& in, const PolySet& out, cudaStream_t st) {
    run(t, in, out, true, st);
}

}  // namespace pft
