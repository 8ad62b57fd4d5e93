"""Bounds the device arithmetic relies on, checked with exact integers on the CPU.

Each check restates a claim made in the kernels' comments (the estimated Shoup quotient, the
Karatsuba sums of the basis conversion and the key inner product, the final reduction of the
uncorrected forward transform, the growth of uncorrected forward butterflies) and tests it at
the extreme inputs and on random ones.  These are statements about integers, independent of the
oracle and of the CUDA code."""
import random

import pytest

M64 = (1 << 64) - 1
RNG = random.Random(20261204)


def split30(a):
    return a & ((1 << 30) - 1), a >> 30


# ---- Karatsuba sums of 30-bit halves ------------------------------------------------------------
def karatsuba_terms(pairs):
    """S00, S11 exactly, and SM kept modulo 2^64 as a 64-bit accumulator would."""
    s00 = s11 = sm = 0
    for a, b in pairs:
        a0, a1 = split30(a)
        b0, b1 = split30(b)
        s00 += a0 * b0
        s11 += a1 * b1
        sm = (sm + (a0 + a1) * (b0 + b1)) & M64
    return s00, s11, sm


@pytest.mark.parametrize("terms", [1, 4, 8])
def test_karatsuba_middle_sum_exact_modulo_2_64(terms):
    """For up to 8 products of values below 2^60: S00 and S11 stay below 2^63, the middle sum
    S01 = sum(a0 b1 + a1 b0) stays below 2^64, so (SM - S00 - S11) mod 2^64 is S01 exactly even
    when SM itself wraps, and S00 + 2^30 S01 + 2^60 S11 is the exact sum of the products."""
    top = (1 << 60) - 1
    cases = [[(top, top)] * terms, [((1 << 30) - 1 | ((1 << 30) - 1) << 30, top)] * terms]
    cases += [[(RNG.getrandbits(60), RNG.getrandbits(60)) for _ in range(terms)] for _ in range(200)]
    wrapped = 0
    for pairs in cases:
        s00, s11, sm = karatsuba_terms(pairs)
        s01 = (sm - s00 - s11) & M64
        exact01 = sum(split30(a)[0] * split30(b)[1] + split30(a)[1] * split30(b)[0] for a, b in pairs)
        assert s00 < 1 << 63 and s11 < 1 << 63 and exact01 < 1 << 64
        assert s01 == exact01
        assert s00 + (s01 << 30) + (s11 << 60) == sum(a * b for a, b in pairs)
        wrapped += sum((split30(a)[0] + split30(a)[1]) * (split30(b)[0] + split30(b)[1]) for a, b in pairs) > M64
    if terms == 8:
        assert wrapped > 0  # the wrapping case is exercised


def test_montgomery_input_bound_of_the_sums():
    """8 products of residues below p < 2^60 (the key words and conversion constants carry the
    factor 2^64, i.e. are residues too) sum below 8 p^2 < p 2^63: the input range of the
    Montgomery reduction with R = 2^64."""
    p = (1 << 60) - 93
    assert 8 * (p - 1) ** 2 < p << 63


# ---- estimated Shoup quotient ---------------------------------------------------------------------
def mulhi_est(x, w):
    """xh wh + hi(xh wl) + hi(xl wh) in 32-bit pieces (the low x low product and the carries of
    the dropped low halves are not formed)."""
    xl, xh = x & 0xFFFFFFFF, x >> 32
    wl, wh = w & 0xFFFFFFFF, w >> 32
    return xh * wh + ((xh * wl) >> 32) + ((xl * wh) >> 32)


def test_estimated_shoup_quotient_and_product_range():
    """The estimate is the exact quotient floor(x w' / 2^64) or at most 2 below it, so the Shoup
    product x w - q_est q lies in [0, 4q) for any 64-bit x and w < q < 2^61."""
    for _ in range(3000):
        q = RNG.getrandbits(RNG.choice([30, 50, 60])) | 1
        w = RNG.randrange(q)
        wp = (w << 64) // q
        x = RNG.choice([RNG.getrandbits(64), M64, RNG.randrange(8 * q)])
        exact = (x * wp) >> 64
        est = mulhi_est(x, wp)
        assert exact - 2 <= est <= exact
        prod = x * w - est * q
        assert 0 <= prod < 4 * q
        assert prod % q == x * w % q


# ---- reduction of uncorrected forward outputs (below 66q) ----------------------------------------
def reduce_below66(x, q):
    s = q.bit_length() - 1
    mu = (1 << (64 + s)) // q
    r = mu >> 32
    xh = x >> (s - 24)
    assert xh < 1 << 32
    est = ((xh * r) >> 32) >> 24
    v = x - est * q
    assert 0 <= v < 2 * q
    return v - q if v >= q else v


@pytest.mark.parametrize("bits", [25, 30, 40, 50, 56])
def test_reduce_below66(bits):
    """For a prime of s + 1 >= 25 bits and x < 66q, the 32-bit estimate
    floor(floor(x / 2^(s-24)) floor(2^(s+32) / q) / 2^56) is floor(x / q) or one less, so one
    conditional subtraction gives the canonical residue."""
    for _ in range(2000):
        q = RNG.randrange(1 << (bits - 1), 1 << bits) | 1
        x = RNG.choice([RNG.randrange(66 * q), 66 * q - 1, 0, q - 1, q])
        assert reduce_below66(x, q) == x % q


# ---- growth of uncorrected forward butterflies ---------------------------------------------------
def test_uncorrected_forward_growth_bound():
    """Cooley-Tukey with the estimated quotient: X + WY and X - WY + 4q with WY in [0, 4q) grow by
    less than 4q per stage; from inputs in [0, 2q) the 16 stages of an N = 2^16 transform stay
    below 66q, which is below 2^63.1 for primes under 2^57 (no 64-bit overflow)."""
    bound = 2  # in units of q
    for _ in range(16):
        bound += 4
    assert bound == 66
    q = (1 << 57) - 1
    assert 66 * q < 2 ** 63.1 < 1 << 64
