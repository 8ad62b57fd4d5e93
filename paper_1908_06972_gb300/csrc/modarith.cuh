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

// Sums of up to 8 products of values below 2^60 in three 64-bit partial sums: with
// a = a1 2^30 + a0 and b = b1 2^30 + b0 (all halves below 2^30),
//   sum a b = S00 + 2^30 S01 + 2^60 S11,  S00 = sum a0 b0 < 2^63,
//   S01 = sum (a0 b1 + a1 b0) < 2^64,  S11 = sum a1 b1 < 2^63,
// so every term is one 32x32+64 multiply-add and no carry is handled per term.
struct Acc3 {
    u64 s00, s01, s11;
};
__device__ __forceinline__ void split30(u64 a, u32& lo, u32& hi) {
    lo = (u32)a & 0x3fffffffu;
    hi = (u32)(a >> 30);
}
// acc + a b as one widening multiply-add (32 x 32 + 64 -> 64)
__device__ __forceinline__ u64 mad_wide(u32 a, u32 b, u64 acc) {
    u64 r;
    asm("mad.wide.u32 %0, %1, %2, %3;" : "=l"(r) : "r"(a), "r"(b), "l"(acc));
    return r;
}
__device__ __forceinline__ void acc3_mac(Acc3& A, u32 a0, u32 a1, u32 b0, u32 b1) {
    A.s00 = mad_wide(a0, b0, A.s00);
    A.s01 = mad_wide(a0, b1, A.s01);
    A.s01 = mad_wide(a1, b0, A.s01);
    A.s11 = mad_wide(a1, b1, A.s11);
}
// Karatsuba form: S00 = sum a0 b0, S11 = sum a1 b1 and SM = sum (a0 + a1)(b0 + b1) (each
// factor below 2^31); the middle sum is SM - S00 - S11.  Three products per term instead of
// four.  SM is kept modulo 2^64: up to 4 terms it does not wrap; up to 8 terms it may, but the
// middle sum itself is below 2^64 (8 terms of a0 b1 + a1 b0 < 2^61), so SM - S00 - S11 taken
// modulo 2^64 is still exactly the middle sum.
struct Acc3K {
    u64 s00, sm, s11;
};
__device__ __forceinline__ void acc3k_mac(Acc3K& A, u32 a0, u32 a1, u32 a01, u32 b0, u32 b1, u32 b01) {
    A.s00 = mad_wide(a0, b0, A.s00);
    A.s11 = mad_wide(a1, b1, A.s11);
    A.sm = mad_wide(a01, b01, A.sm);
}
__device__ __forceinline__ Acc3 acc3k_fold(const Acc3K& A) { return Acc3{A.s00, A.sm - A.s00 - A.s11, A.s11}; }
// the 128-bit value S00 + 2^30 S01 + 2^60 S11
__device__ __forceinline__ U128 acc3_value(const Acc3& A) {
    U128 r;
    r.lo = A.s00;
    r.hi = 0;
    const u64 t1 = A.s01 << 30;
    r.lo += t1;
    r.hi += (A.s01 >> 34) + (r.lo < t1 ? 1 : 0);
    const u64 t2 = A.s11 << 60;
    r.lo += t2;
    r.hi += (A.s11 >> 4) + (r.lo < t2 ? 1 : 0);
    return r;
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

// Montgomery reduction with R = 2^64: for x = hi 2^64 + lo < q 2^63, returns x 2^-64 mod q
// in [0, q).  m = lo (-q^-1) makes lo + m q = 0 mod 2^64 (carry out iff lo != 0), and
// (x + m q) / 2^64 < 1.5 q.
__device__ __forceinline__ u64 mont_reduce_lazy(u64 hi, u64 lo, u64 q, u64 mneg) {  // in [0, 2q)
    const u64 m = lo * mneg;
    return hi + mulhi(m, q) + (lo != 0 ? 1 : 0);
}
__device__ __forceinline__ u64 mont_reduce(u64 hi, u64 lo, u64 q, u64 mneg) {
    const u64 r = mont_reduce_lazy(hi, lo, q, mneg);
    return r >= q ? r - q : r;
}

__device__ __forceinline__ DPrime load_prime(const DPrime* tab, int i) {
    DPrime p;
    p.q = __ldg(&tab[i].q);
    p.mu = __ldg(&tab[i].mu);
    p.r64 = __ldg(&tab[i].r64);
    p.mneg = __ldg(&tab[i].mneg);
    p.s = __ldg(&tab[i].s);
    return p;
}

}  // namespace pft
