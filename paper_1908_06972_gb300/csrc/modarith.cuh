// 64-bit modular arithmetic for primes of at most 60 bits (device).
//
//  * Shoup multiplication by a fixed operand w with w' = floor(w 2^64 / q):
//    x w - floor(x w' / 2^64) q lies in [0, 2q) for any 64-bit x.
//  * Single-word Barrett reduction of a 128-bit value x < 2^(63 + bitlen(q)):
//    with s = bitlen(q) - 1 and mu = floor(2^(64+s) / q), the estimate
//    floor((x >> s) mu / 2^64) is at most 3 below floor(x / q), so the
//    remainder is in [0, 3q) before two conditional subtractions.  Sums of up
//    to 8 products of residues (each below 2^60 and below the target prime)
//    stay inside that bound.
#pragma once
#include <stdint.h>

#include "pft_internal.h"

namespace pft {

__device__ __forceinline__ u64 mulhi(u64 a, u64 b) { return __umul64hi(a, b); }

// x * w mod q in [0, 2q)
__device__ __forceinline__ u64 mul_shoup_lazy(u64 x, u64 w, u64 wp, u64 q) {
    u64 hq = mulhi(x, wp);
    return x * w - hq * q;
}
__device__ __forceinline__ u64 mul_shoup(u64 x, u64 w, u64 wp, u64 q) {
    u64 r = mul_shoup_lazy(x, w, wp, q);
    return r >= q ? r - q : r;
}

struct U128 {
    u64 lo, hi;
};
__device__ __forceinline__ U128 mul_wide(u64 a, u64 b) {
    U128 r;
    r.lo = a * b;
    r.hi = mulhi(a, b);
    return r;
}
__device__ __forceinline__ void mac_wide(U128& acc, u64 a, u64 b) {
    u64 lo = a * b, hi = mulhi(a, b);
    acc.lo += lo;
    acc.hi += hi + (acc.lo < lo ? 1 : 0);
}

// x mod q for x = hi 2^64 + lo < 2^(64 + s)
__device__ __forceinline__ u64 barrett_reduce(u64 hi, u64 lo, const DPrime& P) {
    u64 x1 = (hi << (64 - P.s)) | (lo >> P.s);
    u64 qt = mulhi(x1, P.mu);
    u64 r = lo - qt * P.q;
    if (r >= 2 * P.q) r -= 2 * P.q;
    if (r >= P.q) r -= P.q;
    return r;
}
__device__ __forceinline__ u64 mulmod(u64 a, u64 b, const DPrime& P) {
    U128 x = mul_wide(a, b);
    return barrett_reduce(x.hi, x.lo, P);
}
__device__ __forceinline__ u64 reduce64(u64 a, const DPrime& P) { return barrett_reduce(0, a, P); }

__device__ __forceinline__ u64 addmod(u64 a, u64 b, u64 q) {
    u64 s = a + b;
    return s >= q ? s - q : s;
}
__device__ __forceinline__ u64 submod(u64 a, u64 b, u64 q) { return a >= b ? a - b : a + q - b; }

__device__ __forceinline__ DPrime load_prime(const DPrime* tab, int i) {
    DPrime p;
    p.q = __ldg(&tab[i].q);
    p.mu = __ldg(&tab[i].mu);
    p.r64 = __ldg(&tab[i].r64);
    p.s = __ldg(&tab[i].s);
    return p;
}

}  // namespace pft
