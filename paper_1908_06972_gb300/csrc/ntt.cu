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
// (Harvey lazy butterflies: forward values in [0, 4q), inverse in [0, 2q)), and
// rounds exchange through shared memory.  N <= 2^14: one pass, one CTA per limb.
// N = 2^15, 2^16: two passes (8 + 7 or 8 + 8 stages).
#include "modarith.cuh"

namespace pft {

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
                    const ulonglong2 W = __ldg(&tw[(1 << s) + i]);
                    u64 X = x[e];
                    const u64 Y = x[e | (1 << lb)];
                    if (X >= q2) X -= q2;
                    const u64 Tm = mul_shoup_lazy(Y, W.x, W.y, q);
                    x[e] = X + Tm;
                    x[e | (1 << lb)] = X - Tm + q2;
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
                    const u64 X = x[e];
                    const u64 Y = x[e | (1 << lb)];
                    u64 Sm = X + Y;
                    if (Sm >= q2) Sm -= q2;
                    const u64 D = X - Y + q2;
                    if (s == 0) {  // last inverse stage: fold N^-1 into both outputs
                        x[e] = mul_shoup_lazy(Sm, NI.x, NI.y, q);
                        x[e | (1 << lb)] = mul_shoup_lazy(D, NI1.x, NI1.y, q);
                    } else {
                        const int mid = base | (e << w0);
                        const int i = (hi << (S - p - 1)) + (mid >> (p + 1));
                        const ulonglong2 W = __ldg(&tw[(1 << s) + i]);
                        x[e] = Sm;
                        x[e | (1 << lb)] = mul_shoup_lazy(D, W.x, W.y, q);
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
        if (is_final) {
            if (v >= q2) v -= q2;
            if (v >= q) v -= q;
        }
        dst[j] = v;
    }
}

template <int S, int C, bool INV>
static void launch_pass(const DevTables& t, const PolySet& in, const PolySet& out, int s0, int is_final,
                        cudaStream_t st) {
    constexpr int TPS = 1 << (S - 4);
    constexpr int SUB = (1 << S) + (1 << (S - 4));
    const size_t smem = (size_t)C * SUB * sizeof(u64);
    static bool attr_set = false;  // per template instance
    if (!attr_set) {
        PFT_CUDA(cudaFuncSetAttribute(k_ntt_pass<S, C, INV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr_set = true;
    }
    const int logT = t.logn - s0 - S;
    dim3 grid((unsigned)((t.n >> S) / C), (unsigned)out.max_limbs, (unsigned)out.count);
    PFT_PROF(INV ? (logT > 0 ? "ntt.inv.strided" : "ntt.inv.contig") : (logT > 0 ? "ntt.fwd.strided" : "ntt.fwd.contig"),
             st, set_limbs(out) * (double)(t.n / 2) * S);
    k_ntt_pass<S, C, INV><<<grid, C * TPS, smem, st>>>(t, in, out, s0, logT, is_final);
    PFT_LAUNCH_CHECK("ntt pass");
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
    if (t.logn == 16) {
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
void ntt_inverse(const DevTables& t, const PolySet& in, const PolySet& out, cudaStream_t st) {
    run(t, in, out, true, st);
}

}  // namespace pft
