// Limb-wise kernels of the RNS-CKKS evaluator (device side).
//
// Every kernel is a grid over (coefficient block, limb, polynomial) on the
// limb-major [poly][limb][N] layout, moving two 64-bit words per thread with
// 16-byte accesses.  Residues are canonical in [0, q) at every kernel boundary.
#include <algorithm>
#include <vector>

#include <cstdlib>
#include <cstring>

#include "modarith.cuh"

namespace pft {

static constexpr int kEwThreads = 256;

struct BconvBatch {
    BconvJob j[kMaxBconv];
};
struct KsBatch {
    KsDesc d[kMaxKs];
    uint8_t need[kMaxPrimes];  // per key row: digits used by any input of the batch (0: row unused)
};

static dim3 ew_grid(int n, const PolySet& s) {
    return dim3((unsigned)((n / 2 + kEwThreads - 1) / kEwThreads), (unsigned)s.max_limbs, (unsigned)s.count);
}

// ---- HADD / sub / pointwise product / negate / copy --------------------------------------
template <int OP>
__global__ void k_ew_binary(DevTables t, PolySet a, PolySet b, PolySet out) {
    const int poly = blockIdx.z, limb = blockIdx.y;
    const PolyRef& Ro = out.p[poly];
    if (limb >= Ro.nlimbs) return;
    const int x2 = blockIdx.x * blockDim.x + threadIdx.x;
    if (2 * x2 >= t.n) return;
    const DPrime P = load_prime(t.primes, prime_of(Ro, limb));
    const size_t off = ((size_t)limb << t.logn) + 2 * (size_t)x2;
    const ulonglong2 va = *reinterpret_cast<const ulonglong2*>(a.p[poly].ptr + off);
    ulonglong2 vb = make_ulonglong2(0, 0);
    if (OP <= 2) vb = *reinterpret_cast<const ulonglong2*>(b.p[poly].ptr + off);
    ulonglong2 r;
    if (OP == 0) {
        r.x = addmod(va.x, vb.x, P.q);
        r.y = addmod(va.y, vb.y, P.q);
    } else if (OP == 1) {
        r.x = submod(va.x, vb.x, P.q);
        r.y = submod(va.y, vb.y, P.q);
    } else if (OP == 2) {
        r.x = mulmod(va.x, vb.x, P);
        r.y = mulmod(va.y, vb.y, P);
    } else if (OP == 3) {
        r.x = va.x ? P.q - va.x : 0;
        r.y = va.y ? P.q - va.y : 0;
    } else {
        r = va;
    }
    *reinterpret_cast<ulonglong2*>(Ro.ptr + off) = r;
}

void ew_binary(const DevTables& t, EwOp op, const PolySet& a, const PolySet& b, const PolySet& out,
               cudaStream_t st) {
    if (out.count == 0) return;
    dim3 g = ew_grid(t.n, out);
    PFT_PROF(op == EwOp::Mul ? "ew.mul" : (op == EwOp::Copy ? "ew.copy" : "ew.add"), st,
             set_limbs(out) * t.n * 8.0 * (op == EwOp::Copy || op == EwOp::Neg ? 2 : 3));
    switch (op) {
        case EwOp::Add: k_ew_binary<0><<<g, kEwThreads, 0, st>>>(t, a, b, out); break;
        case EwOp::Sub: k_ew_binary<1><<<g, kEwThreads, 0, st>>>(t, a, b, out); break;
        case EwOp::Mul: k_ew_binary<2><<<g, kEwThreads, 0, st>>>(t, a, b, out); break;
        case EwOp::Neg: k_ew_binary<3><<<g, kEwThreads, 0, st>>>(t, a, b, out); break;
        case EwOp::Copy: k_ew_binary<4><<<g, kEwThreads, 0, st>>>(t, a, b, out); break;
    }
    PFT_LAUNCH_CHECK("ew_binary");
}

// ---- HMUL tensor: d0 = a0 b0, d1 = a0 b1 + a1 b0, d2 = a1 b1 (evaluation domain) -----------
// set a / b / d hold one ref per ciphertext: ptr to [2][l][N] (a, b) or [3][l][N] (d).
__global__ void k_tensor(DevTables t, PolySet a, PolySet b, PolySet d) {
    const int c = blockIdx.z, limb = blockIdx.y;
    const int l = d.p[c].nlimbs;
    if (limb >= l) return;
    const int x2 = blockIdx.x * blockDim.x + threadIdx.x;
    if (2 * x2 >= t.n) return;
    const DPrime P = load_prime(t.primes, limb);
    const size_t off = ((size_t)limb << t.logn) + 2 * (size_t)x2;
    const size_t ps = (size_t)l << t.logn;
    const u64* A = a.p[c].ptr;
    const u64* B = b.p[c].ptr;
    u64* D = d.p[c].ptr;
    const ulonglong2 a0 = *reinterpret_cast<const ulonglong2*>(A + off);
    const ulonglong2 a1 = *reinterpret_cast<const ulonglong2*>(A + ps + off);
    const ulonglong2 b0 = *reinterpret_cast<const ulonglong2*>(B + off);
    const ulonglong2 b1 = *reinterpret_cast<const ulonglong2*>(B + ps + off);
    ulonglong2 r0, r1, r2;
    r0.x = mulmod(a0.x, b0.x, P);
    r0.y = mulmod(a0.y, b0.y, P);
    r2.x = mulmod(a1.x, b1.x, P);
    r2.y = mulmod(a1.y, b1.y, P);
    U128 s = mul_wide(a0.x, b1.x);
    mac_wide(s, a1.x, b0.x);
    r1.x = barrett_reduce(s.hi, s.lo, P);
    s = mul_wide(a0.y, b1.y);
    mac_wide(s, a1.y, b0.y);
    r1.y = barrett_reduce(s.hi, s.lo, P);
    *reinterpret_cast<ulonglong2*>(D + off) = r0;
    *reinterpret_cast<ulonglong2*>(D + ps + off) = r1;
    *reinterpret_cast<ulonglong2*>(D + 2 * ps + off) = r2;
}

void ew_tensor(const DevTables& t, const PolySet& a, const PolySet& b, const PolySet& d, cudaStream_t st) {
    if (d.count == 0) return;
    PFT_PROF("tensor", st, set_limbs(d) * t.n * 8.0 * 7);
    k_tensor<<<ew_grid(t.n, d), kEwThreads, 0, st>>>(t, a, b, d);
    PFT_LAUNCH_CHECK("tensor");
}

// ---- dot products: out[p] = sum_k a[p*K + k] * b[(shared ? 0 : p*K) + k] --------------------
// Pointer tables live in device memory (they can be long).  All polynomials carry
// `l` limbs of the ciphertext chain.  128-bit accumulation, reduced every 8 terms.
__global__ void k_dot(DevTables t, const u64* const* A, const u64* const* Bp, u64* const* O, int K, int b_shared,
                      int l) {
    const int p = blockIdx.z, limb = blockIdx.y;
    if (limb >= l) return;
    const int x2 = blockIdx.x * blockDim.x + threadIdx.x;
    if (2 * x2 >= t.n) return;
    const DPrime P = load_prime(t.primes, limb);
    const size_t off = ((size_t)limb << t.logn) + 2 * (size_t)x2;
    U128 sx = {0, 0}, sy = {0, 0};
    for (int k = 0; k < K; k++) {
        const ulonglong2 va = *reinterpret_cast<const ulonglong2*>(A[(size_t)p * K + k] + off);
        const ulonglong2 vb = *reinterpret_cast<const ulonglong2*>(Bp[(b_shared ? 0 : (size_t)p * K) + k] + off);
        mac_wide(sx, va.x, vb.x);
        mac_wide(sy, va.y, vb.y);
        if ((k & 7) == 7) {
            sx.lo = barrett_reduce(sx.hi, sx.lo, P);
            sx.hi = 0;
            sy.lo = barrett_reduce(sy.hi, sy.lo, P);
            sy.hi = 0;
        }
    }
    ulonglong2 r;
    r.x = barrett_reduce(sx.hi, sx.lo, P);
    r.y = barrett_reduce(sy.hi, sy.lo, P);
    *reinterpret_cast<ulonglong2*>(O[p] + off) = r;
}

void ew_dot(const DevTables& t, const u64* const* A, const u64* const* B, u64* const* O, int n_out, int K,
            bool b_shared, int l, cudaStream_t st) {
    if (n_out == 0) return;
    dim3 g((unsigned)((t.n / 2 + kEwThreads - 1) / kEwThreads), (unsigned)l, (unsigned)n_out);
    PFT_PROF("dot", st, (double)n_out * l * t.n * 8.0 * (2 * K + 1));
    k_dot<<<g, kEwThreads, 0, st>>>(t, A, B, O, K, b_shared ? 1 : 0, l);
    PFT_LAUNCH_CHECK("dot");
}

// ---- sums of HMUL tensors: out[p] (+)= sum_k a[p*K+k] (x) b[p*K+k] ---------------------------
// (a0, a1) (x) (b0, b1) = (a0 b0, a0 b1 + a1 b0, a1 b1).  Tables: A[(p*K + k)*2 + pol] and
// B likewise point at polynomial bases (limb r at r*N, so operands of a higher level are
// read through their leading limbs); O[p*3 + i] at the three output polynomials.  128-bit
// sums reduced every 4 terms (8 products in the middle term).
__global__ void k_tensor_dot(DevTables t, const u64* const* A, const u64* const* B, u64* const* O, int K, int l,
                             int accumulate) {
    const int p = blockIdx.z, limb = blockIdx.y;
    if (limb >= l) return;
    const int x2 = blockIdx.x * blockDim.x + threadIdx.x;
    if (2 * x2 >= t.n) return;
    const DPrime P = load_prime(t.primes, limb);
    const size_t off = ((size_t)limb << t.logn) + 2 * (size_t)x2;
    U128 s0x = {0, 0}, s0y = {0, 0}, s1x = {0, 0}, s1y = {0, 0}, s2x = {0, 0}, s2y = {0, 0};
    for (int k = 0; k < K; k++) {
        const size_t e = ((size_t)p * K + k) * 2;
        const ulonglong2 a0 = *reinterpret_cast<const ulonglong2*>(A[e] + off);
        const ulonglong2 a1 = *reinterpret_cast<const ulonglong2*>(A[e + 1] + off);
        const ulonglong2 b0 = *reinterpret_cast<const ulonglong2*>(B[e] + off);
        const ulonglong2 b1 = *reinterpret_cast<const ulonglong2*>(B[e + 1] + off);
        mac_wide(s0x, a0.x, b0.x);
        mac_wide(s0y, a0.y, b0.y);
        mac_wide(s1x, a0.x, b1.x);
        mac_wide(s1x, a1.x, b0.x);
        mac_wide(s1y, a0.y, b1.y);
        mac_wide(s1y, a1.y, b0.y);
        mac_wide(s2x, a1.x, b1.x);
        mac_wide(s2y, a1.y, b1.y);
        if ((k & 3) == 3) {
            s0x = {barrett_reduce(s0x.hi, s0x.lo, P), 0};
            s0y = {barrett_reduce(s0y.hi, s0y.lo, P), 0};
            s1x = {barrett_reduce(s1x.hi, s1x.lo, P), 0};
            s1y = {barrett_reduce(s1y.hi, s1y.lo, P), 0};
            s2x = {barrett_reduce(s2x.hi, s2x.lo, P), 0};
            s2y = {barrett_reduce(s2y.hi, s2y.lo, P), 0};
        }
    }
    const U128* S[3][2] = {{&s0x, &s0y}, {&s1x, &s1y}, {&s2x, &s2y}};
    for (int i = 0; i < 3; i++) {
        ulonglong2 r;
        r.x = barrett_reduce(S[i][0]->hi, S[i][0]->lo, P);
        r.y = barrett_reduce(S[i][1]->hi, S[i][1]->lo, P);
        u64* dst = O[(size_t)p * 3 + i] + off;
        if (accumulate) {
            const ulonglong2 o = *reinterpret_cast<const ulonglong2*>(dst);
            r.x = addmod(r.x, o.x, P.q);
            r.y = addmod(r.y, o.y, P.q);
        }
        *reinterpret_cast<ulonglong2*>(dst) = r;
    }
}

void ew_tensor_dot(const DevTables& t, const u64* const* A, const u64* const* B, u64* const* O, int n_out, int K,
                   int l, bool accumulate, cudaStream_t st) {
    if (n_out == 0) return;
    dim3 g((unsigned)((t.n / 2 + kEwThreads - 1) / kEwThreads), (unsigned)l, (unsigned)n_out);
    PFT_PROF("tensor_dot", st, (double)n_out * l * t.n * 8.0 * (4 * K + (accumulate ? 6 : 3)));
    k_tensor_dot<<<g, kEwThreads, 0, st>>>(t, A, B, O, K, l, accumulate ? 1 : 0);
    PFT_LAUNCH_CHECK("tensor_dot");
}

// ---- out = acc + (x - y) * s  (s per limb, Shoup pair) ---------------------------------
// Used by ModDown (s = P^-1, acc = the other tensor part or the rotated c0) and by
// rescale (x = c + h, y = NTT(r), s = p^-1): consts[limb] = {add_to_x, s, s_shoup}.
__global__ void k_sub_scale(DevTables t, PolySet x, PolySet y, PolySet acc, PolySet out, const u64* consts,
                            int has_y, int has_acc) {
    const int poly = blockIdx.z, limb = blockIdx.y;
    const PolyRef& Ro = out.p[poly];
    if (limb >= Ro.nlimbs) return;
    const int x2 = blockIdx.x * blockDim.x + threadIdx.x;
    if (2 * x2 >= t.n) return;
    const int pi = prime_of(Ro, limb);
    const u64 q = __ldg(&t.primes[pi].q);
    const u64 c = __ldg(&consts[3 * limb]);
    const u64 s = __ldg(&consts[3 * limb + 1]);
    const u64 sp = __ldg(&consts[3 * limb + 2]);
    const size_t off = ((size_t)limb << t.logn) + 2 * (size_t)x2;
    const ulonglong2 vx = *reinterpret_cast<const ulonglong2*>(x.p[poly].ptr + off);
    ulonglong2 vy = make_ulonglong2(0, 0);
    if (has_y) vy = *reinterpret_cast<const ulonglong2*>(y.p[poly].ptr + off);
    ulonglong2 r;
    r.x = mul_shoup(submod(addmod(vx.x, c, q), vy.x, q), s, sp, q);
    r.y = mul_shoup(submod(addmod(vx.y, c, q), vy.y, q), s, sp, q);
    if (has_acc) {
        const ulonglong2 va = *reinterpret_cast<const ulonglong2*>(acc.p[poly].ptr + off);
        r.x = addmod(r.x, va.x, q);
        r.y = addmod(r.y, va.y, q);
    }
    *reinterpret_cast<ulonglong2*>(Ro.ptr + off) = r;
}

void sub_scale(const DevTables& t, const PolySet& x, const PolySet* y, const PolySet* acc, const PolySet& out,
               const u64* consts_dev, cudaStream_t st) {
    if (out.count == 0) return;
    PFT_PROF("sub_scale", st, set_limbs(out) * t.n * 8.0 * (2 + (y ? 1 : 0) + (acc ? 1 : 0)));
    k_sub_scale<<<ew_grid(t.n, out), kEwThreads, 0, st>>>(t, x, y ? *y : out, acc ? *acc : out, out, consts_dev,
                                                         y ? 1 : 0, acc ? 1 : 0);
    PFT_LAUNCH_CHECK("sub_scale");
}

// ---- Galois automorphism X -> X^g in the evaluation layout ---------------------------------
// Entry i holds a(psi^(2 brv(i) + 1)); a(X^g) there equals a(psi^((2 brv(i) + 1) g)),
// i.e. entry brv(((2 brv(i) + 1) g mod 2N - 1) / 2) of the input.
__device__ __forceinline__ u32 automorph_src(u32 i, int logn, u64 g) {
    const u32 mask2n = (2u << logn) - 1;
    const u32 bi = __brev(i) >> (32 - logn);
    const u32 e = (u32)(((u64)(2 * bi + 1) * g) & mask2n);
    return __brev((e - 1) >> 1) >> (32 - logn);
}

// Multiplication by an odd g modulo 2N fixes the low bits of an exponent given its low bits,
// so in the bit-reversed layout the top bits of a source index depend only on the top bits of
// its destination: every block of kAutBlock consecutive outputs reads one block of
// kAutBlock consecutive inputs.  A CTA stages kAutBlocks such input blocks in shared memory
// with coalesced loads, permutes there and writes its outputs coalesced.
constexpr int kAutBlock = 256, kAutBlocks = 4;

__global__ void __launch_bounds__(256) k_automorph_blocked(DevTables t, PolySet in, PolySet out, u64 g) {
    __shared__ u64 sm[kAutBlocks * kAutBlock];
    const int poly = blockIdx.z, limb = blockIdx.y;
    const PolyRef& Ro = out.p[poly];
    if (limb >= Ro.nlimbs) return;
    const int logn = t.logn;
    const size_t base = (size_t)limb << logn;
    const u64* src = in.p[poly].ptr + base;
    const u32 o0 = blockIdx.x * (kAutBlocks * kAutBlock);
#pragma unroll
    for (int k = 0; k < kAutBlocks; k++) {
        const u32 ib = automorph_src(o0 + k * kAutBlock, logn, g) & ~(u32)(kAutBlock - 1);
        sm[k * kAutBlock + threadIdx.x] = __ldg(src + ib + threadIdx.x);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kAutBlocks; k++) {
        const u32 i = o0 + k * kAutBlock + threadIdx.x;
        Ro.ptr[base + i] = sm[k * kAutBlock + (automorph_src(i, logn, g) & (kAutBlock - 1))];
    }
}

// small rings (N < kAutBlocks * kAutBlock): one gather per output
__global__ void k_automorph(DevTables t, PolySet in, PolySet out, u64 g) {
    const int poly = blockIdx.z, limb = blockIdx.y;
    const PolyRef& Ro = out.p[poly];
    if (limb >= Ro.nlimbs) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= t.n) return;
    const size_t base = (size_t)limb << t.logn;
    Ro.ptr[base + i] = __ldg(in.p[poly].ptr + base + automorph_src((u32)i, t.logn, g));
}

void automorph(const DevTables& t, const PolySet& in, const PolySet& out, u64 g, cudaStream_t st) {
    if (out.count == 0) return;
    PFT_PROF("automorph", st, set_limbs(out) * t.n * 16.0);
    if (t.n >= kAutBlocks * kAutBlock) {
        dim3 grid((unsigned)(t.n / (kAutBlocks * kAutBlock)), (unsigned)out.max_limbs, (unsigned)out.count);
        k_automorph_blocked<<<grid, 256, 0, st>>>(t, in, out, g);
    } else {
        dim3 grid((unsigned)((t.n + 255) / 256), (unsigned)out.max_limbs, (unsigned)out.count);
        k_automorph<<<grid, 256, 0, st>>>(t, in, out, g);
    }
    PFT_LAUNCH_CHECK("automorph");
}

// ---- fast basis conversion (ModUp of one digit, or ModDown from the special primes) ------
// For each coefficient: y_i = x_i * qhat_i^-1 mod s_i (Shoup), then for every target row m
// (rows [0, nrows) except [skip_lo, skip_hi), enumerated in order as targets 0..nt-1):
//   out_m = sum_i y_i * (qhat_i mod t_m) mod t_m   (128-bit sum, one Montgomery reduction),
// left in [0, 2 t_m): every output feeds a forward transform, whose butterflies take it.
// Target prime of row m: m < split ? m : base2 + m - split.  Table: [ns] {inv, inv_shoup},
// then [nt][ns] qhat_i 2^64 mod t_m (Montgomery form, target-major, each split into 30-bit
// halves: low word = c mod 2^30, high word = c >> 30).  NS (the number of source primes) is a
// compile-time constant; each thread converts two adjacent coefficients for two targets at
// a time (four independent accumulation chains).
template <int NS, int TP>
__global__ void __launch_bounds__(256) k_bconv(DevTables t, BconvBatch jobs) {
    extern __shared__ u64 bsm[];
    const BconvJob J = jobs.j[blockIdx.y];
    const int gap = J.skip_hi - J.skip_lo;
    const int nt = J.nrows - gap;
    // the job's constants and, per target, its output row, prime and Montgomery constant,
    // staged once per CTA so that the accumulation loop reads only shared memory
    uint2* sT = reinterpret_cast<uint2*>(bsm);          // [nt][NS] (30-bit split)
    u64* sQ = bsm + (size_t)nt * NS;                    // [nt] target prime
    u64* sM = sQ + nt;                                  // [nt] -q^-1 mod 2^64
    u32* sRow = reinterpret_cast<u32*>(sM + nt);        // [nt] output row
    const uint2* T = reinterpret_cast<const uint2*>(J.table + 2 * NS);
    for (int i = threadIdx.x; i < nt * NS; i += blockDim.x) sT[i] = __ldg(&T[i]);
    for (int i = threadIdx.x; i < nt; i += blockDim.x) {
        const int m = i < J.skip_lo ? i : i + gap;
        const int tp = m < J.split ? m : J.base2 + m - J.split;
        sQ[i] = __ldg(&t.primes[tp].q);
        sM[i] = __ldg(&t.primes[tp].mneg);
        sRow[i] = (u32)m;
    }
    __syncthreads();
    const int x2 = blockIdx.x * blockDim.x + threadIdx.x;
    if (2 * x2 >= t.n) return;
    const int logn = t.logn;
    u64 ya[NS], yb[NS];
#pragma unroll
    for (int i = 0; i < NS; i++) {
        const u64 q = __ldg(&t.primes[J.src_p0 + i].q);
        const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(J.src + ((size_t)i << logn) + 2 * (size_t)x2);
        const u64 w = __ldg(&J.table[2 * i]), wp = __ldg(&J.table[2 * i + 1]);
        ya[i] = mul_shoup(v.x, w, wp, q);
        yb[i] = mul_shoup(v.y, w, wp, q);
    }
    u32 ya0[NS], ya1[NS], yb0[NS], yb1[NS];
#pragma unroll
    for (int i = 0; i < NS; i++) {
        split30(ya[i], ya0[i], ya1[i]);
        split30(yb[i], yb0[i], yb1[i]);
    }
    u64* dst = J.dst + 2 * (size_t)x2;
    // TP targets per iteration (the last group may repeat a target; its result is not stored)
    for (int m0 = 0; m0 < nt; m0 += TP) {
        Acc3 a[TP], b[TP];
        const uint2* cp[TP];
#pragma unroll
        for (int u = 0; u < TP; u++) cp[u] = sT + (m0 + u < nt ? m0 + u : m0) * NS;
        if constexpr (NS <= 4) {  // Karatsuba: three products per term
            Acc3K ka[TP], kb[TP];
#pragma unroll
            for (int u = 0; u < TP; u++) {
                ka[u] = {0, 0, 0};
                kb[u] = {0, 0, 0};
            }
#pragma unroll
            for (int i = 0; i < NS; i++) {
#pragma unroll
                for (int u = 0; u < TP; u++) {
                    const uint2 c = cp[u][i];
                    const u32 c01 = c.x + c.y;
                    acc3k_mac(ka[u], ya0[i], ya1[i], ya0[i] + ya1[i], c.x, c.y, c01);
                    acc3k_mac(kb[u], yb0[i], yb1[i], yb0[i] + yb1[i], c.x, c.y, c01);
                }
            }
#pragma unroll
            for (int u = 0; u < TP; u++) {
                a[u] = acc3k_fold(ka[u]);
                b[u] = acc3k_fold(kb[u]);
            }
        } else {
#pragma unroll
            for (int u = 0; u < TP; u++) {
                a[u] = {0, 0, 0};
                b[u] = {0, 0, 0};
            }
#pragma unroll
            for (int i = 0; i < NS; i++) {
#pragma unroll
                for (int u = 0; u < TP; u++) {
                    const uint2 c = cp[u][i];
                    acc3_mac(a[u], ya0[i], ya1[i], c.x, c.y);
                    acc3_mac(b[u], yb0[i], yb1[i], c.x, c.y);
                }
            }
        }
        // constants are c 2^64 mod t, so a Montgomery reduction of the sum (< t 2^63) gives
        // sum y_i c_i mod t
#pragma unroll
        for (int u = 0; u < TP; u++) {
            if (m0 + u < nt) {
                const u64 q = sQ[m0 + u], mneg = sM[m0 + u];
                const U128 va = acc3_value(a[u]), vb = acc3_value(b[u]);
                ulonglong2 r;
                r.x = mont_reduce_lazy(va.hi, va.lo, q, mneg);
                r.y = mont_reduce_lazy(vb.hi, vb.lo, q, mneg);
                *reinterpret_cast<ulonglong2*>(dst + ((size_t)sRow[m0 + u] << logn)) = r;
            }
        }
    }
}

// ---- basis conversion of four source primes on the tensor cores ----------------------------
// The sum out_m = sum_i y_i c_im mod t_m (y_i the scaled source residues, c_im < t_m) as an
// exact bf16 matrix product: with y_i = sum_a y_ia 2^(8a) (bytes) and the byte planes
// byte_b(c_im 2^(8a) mod t_m) of bconv_tc_table, the FP32 products
//   P_mb = sum_(i,a) y_ia byte_b(c_im 2^(8a) mod t_m)      (32 terms below 2^16: exact below 2^21)
// give sum_b P_mb 2^(8b) = out_m (mod t_m), a value below 2^77, reduced once (Barrett).  One
// mma.sync.m16n8k16 covers 16 coefficients (rows) x the 8 byte planes of one target (columns)
// x 16 of the 32 (source, byte) pairs (k): two per target.  The accumulators start at 2^23, so
// each P arrives as the FP32 bit pattern 0x4B000000 + P (P < 2^23 keeps it exact) and becomes
// an integer by one subtraction.  A CTA converts 1024 coefficients of one job in tiles of 128:
// warp w 16 of each tile,
// with the A fragments (the bytes of its coefficients' y_i) built in registers once for all
// targets; two targets per iteration, then each lane recombines one (coefficient, target).
// The byte planes (about 22 KiB for 34 targets) are staged once per CTA of 1024 coefficients.
constexpr int kTcRows = 1024;  // coefficients per CTA (each warp: 8 tiles of 16)
__device__ __forceinline__ uint32_t bf16_byte(uint32_t v) {  // bf16 bits of an integer 0..255
    return __float_as_uint(__uint_as_float(0x4B000000u | v) - 8388608.0f) >> 16;
}
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__global__ void __launch_bounds__(256) k_bconv_tc(DevTables t, BconvBatch jobs) {
    extern __shared__ __align__(16) uint32_t tsm[];
    const BconvJob J = jobs.j[blockIdx.y];
    const int gap = J.skip_hi - J.skip_lo;
    const int nt = J.nrows - gap;
    uint32_t* Bs = tsm;                                         // [nt][8][kBconvTcStride]
    uint32_t* Cs = tsm + (size_t)nt * 8 * kBconvTcStride;       // [8 warps][2][16][8]
    u64* sP = reinterpret_cast<u64*>(Cs + 8 * 2 * 16 * 8);      // [nt][3]: q, mu, (output row << 8) | s
    for (int i = threadIdx.x; i < nt * 8 * kBconvTcStride; i += blockDim.x) Bs[i] = __ldg(&J.tc[i]);
    for (int m = threadIdx.x; m < nt; m += blockDim.x) {
        const int mrow = m < J.skip_lo ? m : m + gap;
        const int tp = mrow < J.split ? mrow : J.base2 + mrow - J.split;
        sP[3 * m] = __ldg(&t.primes[tp].q);
        sP[3 * m + 1] = __ldg(&t.primes[tp].mu);
        sP[3 * m + 2] = ((u64)mrow << 8) | __ldg(&t.primes[tp].s);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int g = lane >> 2, c = lane & 3;
    const int logn = t.logn;
    __syncthreads();  // the byte planes are in shared memory
    uint32_t* cw = Cs + (size_t)w * 2 * 16 * 8;
    const int my_t = lane >> 4, my_r = lane & 15;  // the (target, row) this lane recombines
    const u64 K1 = 0x4B000000ull * 0x01010101ull;  // the accumulators' offset in four byte planes
    for (int rt = 0; rt < kTcRows / 128; rt++) {
        const size_t row0 = (size_t)blockIdx.x * kTcRows + (size_t)(rt * 8 + w) * 16;  // this tile's first coefficient
        // A fragments: rows g and g + 8, k = 16 s + {2c, 2c+1} (source 2s) and + 8 (source 2s+1)
        uint32_t A[2][4];
        {
            u64 y[2][4];
#pragma unroll
            for (int i = 0; i < 4; i++) {
                const u64 q = __ldg(&t.primes[J.src_p0 + i].q);
                const u64 wv = __ldg(&J.table[2 * i]), wp = __ldg(&J.table[2 * i + 1]);
                const u64* src = J.src + ((size_t)i << logn) + row0;
                y[0][i] = mul_shoup(src[g], wv, wp, q);
                y[1][i] = mul_shoup(src[g + 8], wv, wp, q);
            }
#pragma unroll
            for (int s2 = 0; s2 < 2; s2++)
#pragma unroll
                for (int h = 0; h < 2; h++) {      // h = 0: source 2 s2 (k 0..7), 1: source 2 s2 + 1 (k 8..15)
#pragma unroll
                    for (int r = 0; r < 2; r++) {  // row g, g + 8
                        const u64 v = y[r][2 * s2 + h];
                        const uint32_t lo = bf16_byte((uint32_t)(v >> (16 * c)) & 0xff);
                        const uint32_t hi = bf16_byte((uint32_t)(v >> (16 * c + 8)) & 0xff);
                        A[s2][2 * h + r] = lo | (hi << 16);
                    }
                }
        }
        for (int m0 = 0; m0 < nt; m0 += 2) {
#pragma unroll
            for (int tt = 0; tt < 2; tt++) {
                const int m = m0 + tt < nt ? m0 + tt : m0;  // an odd last target repeats one (not stored)
                float d[4] = {8388608.0f, 8388608.0f, 8388608.0f, 8388608.0f};
                const uint32_t* brow = Bs + ((size_t)m * 8 + g) * kBconvTcStride;
#pragma unroll
                for (int s2 = 0; s2 < 2; s2++) mma_bf16(d, A[s2], brow[8 * s2 + c], brow[8 * s2 + 4 + c]);
                uint32_t* o = cw + tt * 16 * 8;
                *reinterpret_cast<uint2*>(o + g * 8 + 2 * c) = make_uint2(__float_as_uint(d[0]), __float_as_uint(d[1]));
                *reinterpret_cast<uint2*>(o + (g + 8) * 8 + 2 * c) =
                    make_uint2(__float_as_uint(d[2]), __float_as_uint(d[3]));
            }
            __syncwarp();
            const int m = m0 + my_t;
            if (m < nt) {
                const uint4 p0 = *reinterpret_cast<const uint4*>(cw + (my_t * 16 + my_r) * 8);
                const uint4 p1 = *reinterpret_cast<const uint4*>(cw + (my_t * 16 + my_r) * 8 + 4);
                // sum_b P_b 2^(8b) = lo4 + hi4 2^32, lo4/hi4 = sum of four planes (< 2^45 each)
                const u64 lo4 = (u64)p0.x + ((u64)p0.y << 8) + ((u64)p0.z << 16) + ((u64)p0.w << 24) - K1;
                const u64 hi4 = (u64)p1.x + ((u64)p1.y << 8) + ((u64)p1.z << 16) + ((u64)p1.w << 24) - K1;
                const u64 vlo = lo4 + (hi4 << 32);
                const u64 vhi = (hi4 >> 32) + (vlo < lo4 ? 1 : 0);
                DPrime P;
                P.q = sP[3 * m];
                P.mu = sP[3 * m + 1];
                const u64 rs = sP[3 * m + 2];
                P.s = (u32)(rs & 0xff);
                const size_t mrow = (size_t)(rs >> 8);
                J.dst[(mrow << logn) + row0 + my_r] = barrett_reduce(vhi, vlo, P);
            }
            __syncwarp();
        }
    }
}

void bconv(const DevTables& t, const BconvJob* jobs, int n_jobs, cudaStream_t st) {
    // one launch per source-prime count (the last ModUp digit can be shorter)
    for (int ns = 1; ns <= kMaxAlpha; ns++) {
        std::vector<BconvJob> sel;
        for (int i = 0; i < n_jobs; i++)
            if (jobs[i].ns == ns) sel.push_back(jobs[i]);
        // longest jobs (most targets) first, so that short ones fill the last wave
        std::stable_sort(sel.begin(), sel.end(), [](const BconvJob& x, const BconvJob& y) {
            return x.nrows - (x.skip_hi - x.skip_lo) > y.nrows - (y.skip_hi - y.skip_lo);
        });
        for (size_t a = 0; a < sel.size(); a += kMaxBconv) {
            const int cnt = (int)std::min(sel.size() - a, (size_t)kMaxBconv);
            BconvBatch b;
            int ntmax = 1;
            for (int i = 0; i < cnt; i++) {
                b.j[i] = sel[a + i];
                ntmax = max(ntmax, b.j[i].nrows - (b.j[i].skip_hi - b.j[i].skip_lo));
            }
            bool tc = ns == 4 && t.bconv_tc && t.n % kTcRows == 0;
            for (int i = 0; i < cnt && tc; i++) tc = b.j[i].tc != nullptr;
            if (tc) {
                const size_t smem_tc =
                    ((size_t)ntmax * 8 * kBconvTcStride + 8 * 2 * 16 * 8) * sizeof(uint32_t) + (size_t)ntmax * 24;
                if (first_on_device((const void*)k_bconv_tc))
                    PFT_CUDA(cudaFuncSetAttribute(k_bconv_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  (int)((size_t)(kMaxPrimes * 8 * kBconvTcStride + 8 * 2 * 16 * 8) *
                                                            sizeof(uint32_t) + (size_t)kMaxPrimes * 24)));
                PFT_PROF("bconv", st, 0.0);
                k_bconv_tc<<<dim3((unsigned)(t.n / kTcRows), (unsigned)cnt), 256, smem_tc, st>>>(t, b);
                PFT_LAUNCH_CHECK("bconv (tensor cores)");
                continue;
            }
            const size_t smem = (size_t)ntmax * ns * 8 + (size_t)ntmax * 20;
            dim3 grid((unsigned)((t.n / 2 + 255) / 256), (unsigned)cnt);
            PFT_PROF("bconv", st, 0.0);
            switch (ns) {
                case 1: k_bconv<1, 2><<<grid, 256, smem, st>>>(t, b); break;
                case 2: k_bconv<2, 2><<<grid, 256, smem, st>>>(t, b); break;
                case 3: k_bconv<3, 2><<<grid, 256, smem, st>>>(t, b); break;
                case 4: k_bconv<4, 2><<<grid, 256, smem, st>>>(t, b); break;
                case 5: k_bconv<5, 2><<<grid, 256, smem, st>>>(t, b); break;
                case 6: k_bconv<6, 2><<<grid, 256, smem, st>>>(t, b); break;
                case 7: k_bconv<7, 2><<<grid, 256, smem, st>>>(t, b); break;
                default: k_bconv<8, 2><<<grid, 256, smem, st>>>(t, b); break;
            }
            PFT_LAUNCH_CHECK("bconv");
        }
    }
}

// ---- ChaCha20 sampler (RFC 8439 block function, counter mode) -----------------------------
__device__ __forceinline__ u32 rotl(u32 x, int n) { return __funnelshift_l(x, x, n); }
#define PFT_QR(a, b, c, d)                \
    a += b; d ^= a; d = rotl(d, 16);      \
    c += d; b ^= c; b = rotl(b, 12);      \
    a += b; d ^= a; d = rotl(d, 8);       \
    c += d; b ^= c; b = rotl(b, 7);

__device__ void chacha_block(const u32 key[8], u32 ctr, u32 n0, u32 n1, u32 n2, u64 outw[8]) {
    u32 s[16], x[16];
    s[0] = 0x61707865u; s[1] = 0x3320646eu; s[2] = 0x79622d32u; s[3] = 0x6b206574u;
#pragma unroll
    for (int i = 0; i < 8; i++) s[4 + i] = key[i];
    s[12] = ctr; s[13] = n0; s[14] = n1; s[15] = n2;
#pragma unroll
    for (int i = 0; i < 16; i++) x[i] = s[i];
#pragma unroll
    for (int r = 0; r < 10; r++) {
        PFT_QR(x[0], x[4], x[8], x[12]);
        PFT_QR(x[1], x[5], x[9], x[13]);
        PFT_QR(x[2], x[6], x[10], x[14]);
        PFT_QR(x[3], x[7], x[11], x[15]);
        PFT_QR(x[0], x[5], x[10], x[15]);
        PFT_QR(x[1], x[6], x[11], x[12]);
        PFT_QR(x[2], x[7], x[8], x[13]);
        PFT_QR(x[3], x[4], x[9], x[14]);
    }
#pragma unroll
    for (int i = 0; i < 8; i++) outw[i] = (u64)(x[2 * i] + s[2 * i]) | ((u64)(x[2 * i + 1] + s[2 * i + 1]) << 32);
}

struct SeedKey {
    u32 w[8];
};
static SeedKey seed_key(const u64 seed[4]) {
    SeedKey k;
    for (int i = 0; i < 4; i++) {
        k.w[2 * i] = (u32)(seed[i] & 0xffffffffu);
        k.w[2 * i + 1] = (u32)(seed[i] >> 32);
    }
    return k;
}

// (hi 2^64 + lo) mod q = ((hi mod q) (2^64 mod q) + lo) mod q; the sum is below
// q^2 + 2^64 < 2^(63 + bitlen(q)), inside the Barrett bound.
__device__ __forceinline__ u64 uniform_mod(u64 lo, u64 hi, const DPrime& P) {
    const u64 hr = reduce64(hi, P);
    U128 acc = mul_wide(hr, P.r64);
    acc.lo += lo;
    acc.hi += (acc.lo < lo) ? 1 : 0;
    return barrett_reduce(acc.hi, acc.lo, P);
}

// Row m of extended digit j of an input: the input itself for the digit's own rows (when it
// is given), the basis-conversion output otherwise.
__device__ __forceinline__ const u64* ks_row(const KsDesc& D, int j, int E, int m, int alpha, int logn) {
    const int lo = j * alpha;
    if (D.d && m >= lo && m < lo + alpha && m < D.l) return D.d + ((size_t)m << logn);
    return D.ext + (((size_t)j * E + m) << logn);
}

// ---- key inner product over inputs at different levels -----------------------------------
// Row `row` of the key (q rows 0..L-1, special rows L..L+k-1) is used by every input whose
// level l exceeds it (q rows) or by every input (special rows); for input b its extended row
// is m = row (q rows) or l + row - L.  The key slice of two coefficients (digits up to the
// largest the participating inputs need) stays in registers across all inputs.
template <int BMAX, bool COMP>
__global__ void __launch_bounds__(128) k_ks_inner_multi(DevTables t, KsBatch bt, int B, KeyRef kr, int L, int k,
                                                        int alpha) {
    const u64* key = kr.ptr;
    const int row = blockIdx.y;
    const int x2 = blockIdx.x * blockDim.x + threadIdx.x;
    if (2 * x2 >= t.n) return;
    const int logn = t.logn;
    const int rows_total = L + k;
    const int need = bt.need[row];
    if (need == 0) return;
    const DPrime P = load_prime(t.primes, row);
    const size_t xo = 2 * (size_t)x2;
    ulonglong2 kb[BMAX], ka[BMAX];
    if (!COMP) {
#pragma unroll
        for (int j = 0; j < BMAX; j++) {
            if (j < need) {
                kb[j] = __ldg(reinterpret_cast<const ulonglong2*>(key + ((((size_t)j * 2 + 0) * rows_total + row) << logn) + xo));
                ka[j] = __ldg(reinterpret_cast<const ulonglong2*>(key + ((((size_t)j * 2 + 1) * rows_total + row) << logn) + xo));
            }
        }
    } else {
        // ChaCha20 block xo/4 holds the word pairs of coefficients 4(xo/4) .. +3: lanes 2i and
        // 2i+1 (coefficients +0,+1 and +2,+3 of one block) each draw the block of one digit of
        // a pair and swap the halves the other lane needs.
        const int par = (int)(threadIdx.x & 1);
#pragma unroll
        for (int j = 0; j < BMAX; j += 2) {
            if (j < need) {  // uniform over the CTA (one key row)
                u64 w[8];
                chacha_block(kr.seedw, (u32)(xo >> 2), kDomKskAEval, kr.id, 256u * (j + par) + (u32)row, w);
                // this lane's coefficients are word pairs 2 par, 2 par + 1 of the block
                const u64 own0 = uniform_mod(par ? w[4] : w[0], par ? w[5] : w[1], P);
                const u64 own1 = uniform_mod(par ? w[6] : w[2], par ? w[7] : w[3], P);
                const u64 give0 = uniform_mod(par ? w[0] : w[4], par ? w[1] : w[5], P);
                const u64 give1 = uniform_mod(par ? w[2] : w[6], par ? w[3] : w[7], P);
                const u64 got0 = __shfl_xor_sync(0xffffffffu, give0, 1);
                const u64 got1 = __shfl_xor_sync(0xffffffffu, give1, 1);
                // lane parity 0 drew digit j, parity 1 drew digit j + 1
                const ulonglong2 a_own = make_ulonglong2(own0, own1), a_got = make_ulonglong2(got0, got1);
                ka[j] = par ? a_got : a_own;
                if (j + 1 < BMAX) ka[j + 1] = par ? a_own : a_got;
                kb[j] = __ldg(reinterpret_cast<const ulonglong2*>(key + (((size_t)j * rows_total + row) << logn) + xo));
                if (j + 1 < need)
                    kb[j + 1] =
                        __ldg(reinterpret_cast<const ulonglong2*>(key + (((size_t)(j + 1) * rows_total + row) << logn) + xo));
            }
        }
    }
    for (int b = 0; b < B; b++) {
        const KsDesc D = bt.d[b];
        const int l = D.l;
        if (row < L && row >= l) continue;
        const int m = row < L ? row : l + row - L;
        const int E = l + k;
        const int beta = (l + alpha - 1) / alpha;
        ulonglong2 v[BMAX];
#pragma unroll
        for (int j = 0; j < BMAX; j++)
            if (j < beta) v[j] = __ldg(reinterpret_cast<const ulonglong2*>(ks_row(D, j, E, m, alpha, logn) + xo));
        U128 s0x = {0, 0}, s0y = {0, 0}, s1x = {0, 0}, s1y = {0, 0};
#pragma unroll
        for (int j = 0; j < BMAX; j++) {
            if (j < beta) {  // beta <= 8: 128-bit sums of at most 8 products
                mac_wide(s0x, v[j].x, kb[j].x);
                mac_wide(s0y, v[j].y, kb[j].y);
                mac_wide(s1x, v[j].x, ka[j].x);
                mac_wide(s1y, v[j].y, ka[j].y);
            }
        }
        ulonglong2 r0, r1;
        r0.x = barrett_reduce(s0x.hi, s0x.lo, P);
        r0.y = barrett_reduce(s0y.hi, s0y.lo, P);
        r1.x = barrett_reduce(s1x.hi, s1x.lo, P);
        r1.y = barrett_reduce(s1y.hi, s1y.lo, P);
        *reinterpret_cast<ulonglong2*>(D.u + ((size_t)m << logn) + xo) = r0;
        *reinterpret_cast<ulonglong2*>(D.u + (((size_t)E + m) << logn) + xo) = r1;
    }
}

// ---- the same with bulk copies (cp.async.bulk + mbarrier) ---------------------------------
// CTA = one key row x 256 coefficients, 128 threads with two coefficients each and the key
// slice in registers.  The digit rows of the inputs that use the row stream through a ring
// of kKsStages shared-memory stages (one input's digits, 2 KiB each) filled by one thread
// with 1-D bulk copies whose bytes an mbarrier per stage counts: the CTA computes input u
// while the copies of the next inputs are in flight.  Every wait is bounded; on expiry the
// kernel records the failure in g_wait_timeout, then drains its own copies in flight: one
// thread waits for every stage that still expects bytes, with a bound 16 times the first
// (kDrainPolls), before the CTA returns.  A copy of 2 KiB per digit row lands in microseconds;
// only a memory system that has stopped answering could outlast both bounds, and then the CTA
// returns with the copy still pending and its results flagged invalid (the host reads
// PFT_ERR_TIMEOUT from pft_device_status).  (Per-warp waits with an "empty" mbarrier per stage
// in place of the two CTA barriers per input measured slower: 201 against 196 us for 4
// ciphertexts at level 30; so did one coefficient per thread in CTAs of 256 threads, 64
// registers and twice the resident warps: 221 us.)
constexpr int kKsStages = 3;
constexpr int kKsChunk = 256;                // coefficients per CTA (2 KiB per digit row)
constexpr long long kWaitPolls = 1ll << 22;  // polls of a bounded wait (seconds at most)
constexpr long long kDrainPolls = kWaitPolls << 4;  // polls of the drain after an expired wait

__device__ int g_wait_timeout;

__device__ __forceinline__ u32 smem_addr(const void* p) { return (u32)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(u64* bar, u32 count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(u64* bar, u32 bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, u32 bytes, u64* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_test(u64* bar, u32 parity) {
    u32 ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_wait(u64* bar, u32 parity, long long polls = kWaitPolls) {
    for (long long i = 0; i < polls; i++)
        if (mbar_test(bar, parity)) return true;
    return false;
}

// One digit's term of both key products for one coefficient: v (a residue below 2^60) times the
// key words kb and ka (split Montgomery form k0 | k1 << 32, k0 and k1 below 2^30), added to the
// Karatsuba sums of the b and a outputs.
__device__ __forceinline__ void ks_mac(Acc3K& sb, Acc3K& sa, u64 v, u64 kb, u64 ka) {
    u32 x0, x1;
    split30(v, x0, x1);
    const u32 x01 = x0 + x1;
    const u32 b0 = (u32)kb, b1 = (u32)(kb >> 32), a0 = (u32)ka, a1 = (u32)(ka >> 32);
    acc3k_mac(sb, x0, x1, x01, b0, b1, b0 + b1);
    acc3k_mac(sa, x0, x1, x01, a0, a1, a0 + a1);
}
// the canonical residue of the sum: (S00 + 2^30 S01 + 2^60 S11) 2^-64 mod p
__device__ __forceinline__ u64 ks_value(const Acc3K& s, const DPrime& P) {
    const U128 a = acc3_value(acc3k_fold(s));
    return mont_reduce(a.hi, a.lo, P.q, P.mneg);
}

template <int BMAX>
__global__ void __launch_bounds__(128) k_ks_inner_bulk(DevTables t, KsBatch bt, int B, KeyRef kr, int L, int k,
                                                       int alpha, int stage_digits) {
    extern __shared__ __align__(128) u64 ring[];  // [kKsStages][stage_digits][kKsChunk]
    __shared__ __align__(8) u64 bars[kKsStages];
    // special rows first: every input uses them, so their CTAs are the longest and should not
    // form the last wave
    const int row = (int)blockIdx.y < k ? L + (int)blockIdx.y : (int)blockIdx.y - k;
    const int logn = t.logn;
    const int rows_total = L + k;
    const int need = bt.need[row];
    if (need == 0) return;  // uniform over the CTA
    const size_t chunk0 = (size_t)blockIdx.x * kKsChunk;
    const int xl = 2 * threadIdx.x;
    const size_t xo = chunk0 + xl;
    const DPrime P = load_prime(t.primes, row);
    const u64* key = kr.mont;  // split Montgomery form: k0 | k1 << 32 with k 2^64 mod p = k1 2^30 + k0
    ulonglong2 kb[BMAX], ka[BMAX];
#pragma unroll
    for (int j = 0; j < BMAX; j++) {
        if (j < need) {
            kb[j] = __ldg(reinterpret_cast<const ulonglong2*>(key + ((((size_t)j * 2 + 0) * rows_total + row) << logn) + xo));
            ka[j] = __ldg(reinterpret_cast<const ulonglong2*>(key + ((((size_t)j * 2 + 1) * rows_total + row) << logn) + xo));
        }
    }
    auto used = [&](int b) { return !(row < L && row >= bt.d[b].l); };
    auto next = [&](int b) {
        while (b < B && !used(b)) b++;
        return b;
    };
    // thread 0 fills stage s with the digit rows of input b
    auto issue = [&](int b, int s) {
        const KsDesc& D = bt.d[b];
        const int l = D.l, E = l + k, beta = (l + alpha - 1) / alpha;
        const int m = row < L ? row : l + row - L;
        mbar_expect_tx(&bars[s], (u32)(beta * kKsChunk * 8));
        for (int j = 0; j < beta; j++)
            bulk_g2s(ring + ((size_t)s * stage_digits + j) * kKsChunk, ks_row(D, j, E, m, alpha, logn) + chunk0,
                     (u32)(kKsChunk * 8), &bars[s]);
    };
    if (threadIdx.x == 0) {
        for (int s2 = 0; s2 < kKsStages; s2++) mbar_init(&bars[s2], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // prologue: the first kKsStages used inputs
    int ib = next(0);
    if (threadIdx.x == 0) {
        int bb = ib;
        for (int s2 = 0; s2 < kKsStages && bb < B; s2++, bb = next(bb + 1)) issue(bb, s2);
    }
    for (int s2 = 0; s2 < kKsStages && ib < B; s2++) ib = next(ib + 1);  // ib: next input to issue
    int u = 0;
    for (int b = next(0); b < B; b = next(b + 1), u++) {
        const int s = u % kKsStages;
        const u32 parity = (u32)((u / kKsStages) & 1);
        const bool ok = __syncthreads_and(mbar_wait(&bars[s], parity));
        if (!ok) {
            // record, then wait (bounded) for the copies still in flight on the other stages
            if (threadIdx.x == 0) {
                atomicExch(&g_wait_timeout, 1);
                mbar_wait(&bars[s], parity, kDrainPolls);
                int uu = u + 1;
                for (int bb = next(b + 1); bb < ib; bb = next(bb + 1), uu++)
                    mbar_wait(&bars[uu % kKsStages], (u32)((uu / kKsStages) & 1), kDrainPolls);
            }
            return;
        }
        const KsDesc& D = bt.d[b];
        const int l = D.l, E = l + k, beta = (l + alpha - 1) / alpha;
        const int m = row < L ? row : l + row - L;
        const u64* st = ring + (size_t)s * stage_digits * kKsChunk + xl;
        // sums of at most 8 products of residues below 2^60 in 30-bit-split Karatsuba partial
        // sums (three widening multiply-adds per product), then one Montgomery reduction: the key
        // words carry the factor 2^64 (sum < 8 p^2 < p 2^63)
        Acc3K s0x = {0, 0, 0}, s0y = {0, 0, 0}, s1x = {0, 0, 0}, s1y = {0, 0, 0};
#pragma unroll
        for (int j = 0; j < BMAX; j++) {
            if (j < beta) {
                const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(st + (size_t)j * kKsChunk);
                ks_mac(s0x, s1x, v.x, kb[j].x, ka[j].x);
                ks_mac(s0y, s1y, v.y, kb[j].y, ka[j].y);
            }
        }
        ulonglong2 r0, r1;
        r0.x = ks_value(s0x, P);
        r0.y = ks_value(s0y, P);
        r1.x = ks_value(s1x, P);
        r1.y = ks_value(s1y, P);
        *reinterpret_cast<ulonglong2*>(D.u + ((size_t)m << logn) + xo) = r0;
        *reinterpret_cast<ulonglong2*>(D.u + (((size_t)E + m) << logn) + xo) = r1;
        __syncthreads();  // every thread has read stage s
        if (ib < B) {
            if (threadIdx.x == 0) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                issue(ib, s);
            }
            ib = next(ib + 1);
        }
    }
}

// Self-test of the bounded wait: an mbarrier that expects bytes no copy delivers (no copy is
// issued, so nothing is in flight) must give up after `polls` polls and raise the flag.
__global__ void k_wait_selftest(long long polls) {
    __shared__ __align__(8) u64 bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    mbar_expect_tx(&bar, 16);
    bool ok = false;
    for (long long i = 0; i < polls && !ok; i++) ok = mbar_test(&bar, 0);
    if (!ok) atomicExch(&g_wait_timeout, 1);
}

void wait_selftest(long long polls, cudaStream_t st) {
    k_wait_selftest<<<1, 32, 0, st>>>(polls);
    PFT_LAUNCH_CHECK("wait self-test");
}

int wait_timeout_flag(bool reset, cudaStream_t st) {
    int v = 0;
    PFT_CUDA(cudaMemcpyFromSymbolAsync(&v, g_wait_timeout, sizeof(int), 0, cudaMemcpyDeviceToHost, st));
    PFT_CUDA(cudaStreamSynchronize(st));
    if (reset && v) {
        static const int z = 0;
        PFT_CUDA(cudaMemcpyToSymbolAsync(g_wait_timeout, &z, sizeof(int), 0, cudaMemcpyHostToDevice, st));
        PFT_CUDA(cudaStreamSynchronize(st));
    }
    return v;
}

// ---- persistent job queue -------------------------------------------------------------------
constexpr int kQThreads = 256;

__device__ __forceinline__ u64 globaltimer() {
    u64 t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ u32 load_acquire(const u32* p) {
    u32 v;
    asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
// true once *p >= target; false after timeout_ns of %globaltimer
__device__ __forceinline__ bool wait_at_least(const u32* p, u32 target, long long timeout_ns) {
    const u64 t0 = globaltimer();
    for (;;) {
        if (load_acquire(p) >= target) return true;
        if ((long long)(globaltimer() - t0) > timeout_ns) return false;
        __nanosleep(256);
    }
}

// counters: [0] next tile (claimed with atomicAdd), [1 + j] tiles of job j finished
__global__ void __launch_bounds__(kQThreads) k_job_queue(const QJob* __restrict__ jobs, int n_jobs,
                                                          long long total_tiles, u64* counters, long long timeout_ns) {
    __shared__ long long s_tile;
    __shared__ int s_job, s_ok;
    u32* done = reinterpret_cast<u32*>(counters + 1);
    for (;;) {
        if (threadIdx.x == 0) s_tile = (long long)atomicAdd(reinterpret_cast<unsigned long long*>(counters), 1ull);
        __syncthreads();
        const long long tile = s_tile;
        if (tile >= total_tiles) return;  // uniform over the CTA
        if (threadIdx.x == 0) {
            int lo = 0, hi = n_jobs - 1;  // the job holding this tile: last job with tile0 <= tile
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (jobs[mid].tile0 <= tile) lo = mid;
                else hi = mid - 1;
            }
            const QJob& J = jobs[lo];
            bool ok = true;
            if (J.after >= 0) ok = wait_at_least(&done[J.after], (u32)jobs[J.after].ntiles, timeout_ns);
            if (ok && J.wait_flag) ok = wait_at_least(J.wait_flag, J.wait_value, timeout_ns);
            if (!ok) atomicExch(&g_wait_timeout, 1);
            s_job = lo;
            s_ok = ok ? 1 : 0;
        }
        __syncthreads();
        if (s_ok) {
            const QJob& J = jobs[s_job];
            const int n = 1 << J.logn, chunk = queue_chunk(J.logn), cpl = n / chunk;
            const long long tl = tile - J.tile0;
            const int poly = (int)(tl / ((long long)J.level * cpl));
            const int rem = (int)(tl % ((long long)J.level * cpl));
            const int limb = rem / cpl, c0 = (rem % cpl) * chunk;
            const DPrime P = load_prime(J.primes, limb);
            const size_t off = ((size_t)poly * J.level + limb) * (size_t)n + c0;
            const size_t offb = J.op == kQMulPlain ? (size_t)limb * n + c0 : off;
            for (int x = 2 * threadIdx.x; x < chunk; x += 2 * kQThreads) {
                const ulonglong2 va = *reinterpret_cast<const ulonglong2*>(J.a + off + x);
                const ulonglong2 vb = *reinterpret_cast<const ulonglong2*>(J.b + offb + x);
                ulonglong2 r;
                if (J.op == kQAdd) {
                    r.x = addmod(va.x, vb.x, P.q);
                    r.y = addmod(va.y, vb.y, P.q);
                } else if (J.op == kQSub) {
                    r.x = submod(va.x, vb.x, P.q);
                    r.y = submod(va.y, vb.y, P.q);
                } else {
                    r.x = mulmod(va.x, vb.x, P);
                    r.y = mulmod(va.y, vb.y, P);
                }
                *reinterpret_cast<ulonglong2*>(J.out + off + x) = r;
            }
        }
        __syncthreads();  // the tile's writes precede its completion count
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(&done[s_job], 1u);
        }
    }
}

void job_queue(const QJob* jobs_dev, int n_jobs, long long total_tiles, u64* counters_dev, long long timeout_ns,
               double bytes, cudaStream_t st) {
    if (total_tiles == 0) return;
    static int resident = 0;  // CTAs per SM x SMs: every CTA of the grid is resident at once
    if (!resident) {
        int dev = 0, sms = 0, per_sm = 0;
        PFT_CUDA(cudaGetDevice(&dev));
        PFT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        PFT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_job_queue, kQThreads, 0));
        resident = std::max(1, sms * per_sm);
    }
    const int grid = (int)std::min<long long>(resident, total_tiles);
    PFT_PROF("queue", st, bytes);
    k_job_queue<<<grid, kQThreads, 0, st>>>(jobs_dev, n_jobs, total_tiles, counters_dev, timeout_ns);
    PFT_LAUNCH_CHECK("job queue");
}

// Any number of digits: the key is re-read (or regenerated) for every input.
__global__ void k_ks_inner_multi_generic(DevTables t, KsBatch bt, int B, KeyRef kr, int L, int k, int alpha) {
    const u64* key = kr.ptr;
    const int row = blockIdx.y;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= t.n) return;
    const int logn = t.logn;
    const int rows_total = L + k;
    const DPrime P = load_prime(t.primes, row);
    for (int b = 0; b < B; b++) {
        const KsDesc D = bt.d[b];
        const int l = D.l;
        if (row < L && row >= l) continue;
        const int m = row < L ? row : l + row - L;
        const int E = l + k;
        const int beta = (l + alpha - 1) / alpha;
        U128 s0 = {0, 0}, s1 = {0, 0};
        for (int j = 0; j < beta; j++) {
            const u64 v = __ldg(ks_row(D, j, E, m, alpha, logn) + x);
            u64 kb, ka;
            if (!kr.compressed) {
                kb = __ldg(key + ((((size_t)j * 2 + 0) * rows_total + row) << logn) + x);
                ka = __ldg(key + ((((size_t)j * 2 + 1) * rows_total + row) << logn) + x);
            } else {
                kb = __ldg(key + (((size_t)j * rows_total + row) << logn) + x);
                u64 w[8];
                chacha_block(kr.seedw, (u32)(x >> 2), kDomKskAEval, kr.id, 256u * j + (u32)row, w);
                ka = uniform_mod(w[2 * (x & 3)], w[2 * (x & 3) + 1], P);
            }
            mac_wide(s0, v, kb);
            mac_wide(s1, v, ka);
            if ((j & 7) == 7) {
                s0.lo = barrett_reduce(s0.hi, s0.lo, P);
                s0.hi = 0;
                s1.lo = barrett_reduce(s1.hi, s1.lo, P);
                s1.hi = 0;
            }
        }
        D.u[((size_t)m << logn) + x] = barrett_reduce(s0.hi, s0.lo, P);
        D.u[(((size_t)E + m) << logn) + x] = barrett_reduce(s1.hi, s1.lo, P);
    }
}

void ks_inner_multi(const DevTables& t, const KsDesc* descs, int B, const KeyRef& key, int L, int k, int alpha,
                    cudaStream_t st) {
    const int beta_max = (L + alpha - 1) / alpha;
    for (int a = 0; a < B; a += kMaxKs) {
        const int cnt = B - a < kMaxKs ? B - a : kMaxKs;
        KsBatch bt;
        double bytes = 0;
        int lmax = 0;
        for (int r = 0; r < kMaxPrimes; r++) bt.need[r] = 0;
        for (int i = 0; i < cnt; i++) {
            bt.d[i] = descs[a + i];
            const int l = descs[a + i].l, E = l + k, beta = (l + alpha - 1) / alpha;
            bytes += (double)(beta + 2) * E * t.n * 8.0;
            lmax = max(lmax, l);
            for (int r = 0; r < L + k; r++)
                if ((r >= L || r < l) && bt.need[r] < beta) bt.need[r] = (uint8_t)beta;
        }
        bytes += (key.compressed ? 1.0 : 2.0) * ((lmax + alpha - 1) / alpha) * (lmax + k) * t.n * 8.0;  // key rows read
        dim3 grid2((unsigned)((t.n / 2 + 127) / 128), (unsigned)(L + k));
        dim3 grid1((unsigned)((t.n + 127) / 128), (unsigned)(L + k));
        PFT_PROF("ks_inner", st, bytes);
        if (beta_max <= 8 && !key.compressed && key.mont && t.n % kKsChunk == 0) {
            const int sd = beta_max <= 4 ? 4 : 8;
            dim3 gb((unsigned)(t.n / kKsChunk), (unsigned)(L + k));
            const size_t smem = (size_t)kKsStages * sd * kKsChunk * 8;
            // the 8-digit ring needs 48 KiB of dynamic shared memory
            if (first_on_device((const void*)&k_ks_inner_bulk<8>)) {
                PFT_CUDA(cudaFuncSetAttribute(k_ks_inner_bulk<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)((size_t)kKsStages * 8 * kKsChunk * 8)));
                PFT_CUDA(cudaFuncSetAttribute(k_ks_inner_bulk<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)((size_t)kKsStages * 8 * kKsChunk * 8)));
            }
            if (sd == 4) k_ks_inner_bulk<4><<<gb, 128, smem, st>>>(t, bt, cnt, key, L, k, alpha, sd);
            else k_ks_inner_bulk<8><<<gb, 128, smem, st>>>(t, bt, cnt, key, L, k, alpha, sd);
        } else if (key.compressed && t.n < 256) {  // lane pairs need full warps
            k_ks_inner_multi_generic<<<grid1, 128, 0, st>>>(t, bt, cnt, key, L, k, alpha);
        } else if (beta_max <= 4 && !key.compressed) k_ks_inner_multi<4, false><<<grid2, 128, 0, st>>>(t, bt, cnt, key, L, k, alpha);
        else if (beta_max <= 8 && !key.compressed) k_ks_inner_multi<8, false><<<grid2, 128, 0, st>>>(t, bt, cnt, key, L, k, alpha);
        else if (beta_max <= 4) k_ks_inner_multi<4, true><<<grid2, 128, 0, st>>>(t, bt, cnt, key, L, k, alpha);
        else if (beta_max <= 8) k_ks_inner_multi<8, true><<<grid2, 128, 0, st>>>(t, bt, cnt, key, L, k, alpha);
        else k_ks_inner_multi_generic<<<grid1, 128, 0, st>>>(t, bt, cnt, key, L, k, alpha);
        PFT_LAUNCH_CHECK("ks_inner_multi");
    }
}

// ---- rescale broadcast: r = (c_{l-1} + h) mod p, h = floor(p/2), per coefficient; every
// lower limb k receives (r - h) mod q_k (coefficient form), so that after the transform
// c'_k = (c_k - out_k) p^-1 = (c_k + h - r) / p coefficient by coefficient.
// last: coefficient-form last limb of each polynomial; out: [l-1][N] per polynomial.
__global__ void k_rescale_bcast(DevTables t, PolySet last, PolySet out) {
    const int poly = blockIdx.z, limb = blockIdx.y;
    const PolyRef& Ro = out.p[poly];
    if (limb >= Ro.nlimbs) return;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= t.n) return;
    const int lp = Ro.nlimbs;  // index of the dropped prime
    const u64 p = __ldg(&t.primes[lp].q);
    u64 r = __ldg(last.p[poly].ptr + x) + (p >> 1);
    if (r >= p) r -= p;
    const DPrime P = load_prime(t.primes, limb);
    Ro.ptr[((size_t)limb << t.logn) + x] = submod(reduce64(r, P), reduce64(p >> 1, P), P.q);
}

void rescale_bcast(const DevTables& t, const PolySet& last, const PolySet& out, cudaStream_t st) {
    if (out.count == 0) return;
    dim3 grid((unsigned)((t.n + 255) / 256), (unsigned)out.max_limbs, (unsigned)out.count);
    PFT_PROF("rescale_bcast", st, set_limbs(out) * t.n * 8.0);
    k_rescale_bcast<<<grid, 256, 0, st>>>(t, last, out);
    PFT_LAUNCH_CHECK("rescale_bcast");
}

// uniform mod q: block b (counter b) gives coefficients 4b..4b+3 from word pairs.
__global__ void k_sample_uniform(DevTables t, SeedKey key, u32 dom, u32 obj, u32 sub_base, PolySet out) {
    const int poly = blockIdx.z, limb = blockIdx.y;
    const PolyRef& Ro = out.p[poly];
    if (limb >= Ro.nlimbs) return;
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (4 * b >= t.n) return;
    const int pi = prime_of(Ro, limb);
    const DPrime P = load_prime(t.primes, pi);
    u64 w[8];
    chacha_block(key.w, (u32)b, dom, obj, sub_base + (u32)pi, w);
    u64* dst = Ro.ptr + ((size_t)limb << t.logn) + 4 * (size_t)b;
#pragma unroll
    for (int c = 0; c < 4; c++) dst[c] = uniform_mod(w[2 * c], w[2 * c + 1], P);
}

void sample_uniform(const DevTables& t, const u64 seed[4], u32 dom, u32 obj, u32 sub_base, const PolySet& out,
                    cudaStream_t st) {
    if (out.count == 0) return;
    dim3 grid((unsigned)((t.n / 4 + 127) / 128), (unsigned)out.max_limbs, (unsigned)out.count);
    PFT_PROF("sample", st, 0.0);
    k_sample_uniform<<<grid, 128, 0, st>>>(t, seed_key(seed), dom, obj, sub_base, out);
    PFT_LAUNCH_CHECK("sample_uniform");
}

struct Cdt {
    u32 v[64];
    int n;
};
// ternary (kind 0): word c mod 3 - 1;  Gaussian (kind 1): magnitude = #{j : top32(w) >= T_j}, sign = w & 1.
__global__ void k_sample_small(DevTables t, SeedKey key, u32 dom, u32 obj, u32 sub, int kind, Cdt cdt, i64* out) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (8 * b >= t.n) return;
    u64 w[8];
    chacha_block(key.w, (u32)b, dom, obj, sub, w);
#pragma unroll
    for (int c = 0; c < 8; c++) {
        i64 v;
        if (kind == 0) {
            v = (i64)(w[c] % 3) - 1;
        } else {
            const u32 top = (u32)(w[c] >> 32);
            i64 mag = 0;
            for (int j = 0; j < cdt.n; j++) mag += (top >= cdt.v[j]) ? 1 : 0;
            v = (w[c] & 1) ? -mag : mag;
        }
        out[8 * b + c] = v;
    }
}

void sample_small(const DevTables& t, const u64 seed[4], u32 dom, u32 obj, u32 sub, int kind, const u32* cdt,
                  int nt, i64* out_dev, cudaStream_t st) {
    Cdt c;
    c.n = nt;
    for (int i = 0; i < nt && i < 64; i++) c.v[i] = cdt[i];
    dim3 grid((unsigned)((t.n / 8 + 127) / 128));
    PFT_PROF("sample", st, 0.0);
    k_sample_small<<<grid, 128, 0, st>>>(t, seed_key(seed), dom, obj, sub, kind, c, out_dev);
    PFT_LAUNCH_CHECK("sample_small");
}

// signed integer polynomial -> residues in every limb of every polynomial of `out`
__global__ void k_reduce_signed(DevTables t, const i64* x, PolySet out) {
    const int poly = blockIdx.z, limb = blockIdx.y;
    const PolyRef& Ro = out.p[poly];
    if (limb >= Ro.nlimbs) return;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= t.n) return;
    const DPrime P = load_prime(t.primes, prime_of(Ro, limb));
    const i64 v = x[c];
    const u64 m = reduce64((u64)(v < 0 ? -v : v), P);
    Ro.ptr[((size_t)limb << t.logn) + c] = (v < 0 && m) ? P.q - m : m;
}

void reduce_signed(const DevTables& t, const i64* x_dev, const PolySet& out, cudaStream_t st) {
    if (out.count == 0) return;
    dim3 grid((unsigned)((t.n + 255) / 256), (unsigned)out.max_limbs, (unsigned)out.count);
    PFT_PROF("reduce_signed", st, 0.0);
    k_reduce_signed<<<grid, 256, 0, st>>>(t, x_dev, out);
    PFT_LAUNCH_CHECK("reduce_signed");
}

// words of `in` (any 64-bit values) -> residues modulo each limb's prime in `out`
__global__ void k_reduce_words(DevTables t, PolySet in, PolySet out) {
    const int poly = blockIdx.z, limb = blockIdx.y;
    const PolyRef& Ro = out.p[poly];
    if (limb >= Ro.nlimbs) return;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= t.n) return;
    const DPrime P = load_prime(t.primes, prime_of(Ro, limb));
    const size_t o = ((size_t)limb << t.logn) + c;
    Ro.ptr[o] = reduce64(in.p[poly].ptr[o], P);
}

__global__ void k_mont_split(DevTables t, PolySet in, PolySet out) {
    const int poly = blockIdx.z, limb = blockIdx.y;
    const PolyRef& Ro = out.p[poly];
    if (limb >= Ro.nlimbs) return;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= t.n) return;
    const DPrime P = load_prime(t.primes, prime_of(Ro, limb));
    const size_t o = ((size_t)limb << t.logn) + c;
    const u64 m = mulmod(in.p[poly].ptr[o], P.r64, P);  // k 2^64 mod p
    Ro.ptr[o] = (m & 0x3fffffffull) | ((m >> 30) << 32);
}

void mont_split(const DevTables& t, const PolySet& in, const PolySet& out, cudaStream_t st) {
    if (out.count == 0) return;
    dim3 grid((unsigned)((t.n + 255) / 256), (unsigned)out.max_limbs, (unsigned)out.count);
    PFT_PROF("mont_split", st, 0.0);
    k_mont_split<<<grid, 256, 0, st>>>(t, in, out);
    PFT_LAUNCH_CHECK("mont_split");
}

void reduce_words(const DevTables& t, const PolySet& in, const PolySet& out, cudaStream_t st) {
    if (out.count == 0) return;
    dim3 grid((unsigned)((t.n + 255) / 256), (unsigned)out.max_limbs, (unsigned)out.count);
    PFT_PROF("reduce_words", st, set_limbs(out) * t.n * 16.0);
    k_reduce_words<<<grid, 256, 0, st>>>(t, in, out);
    PFT_LAUNCH_CHECK("reduce_words");
}

}  // namespace pft
