"""Pins of the oracle's ring and RNS arithmetic (products, automorphism, CRT,
basis conversion, ModDown, rescale) against brute force, big integers and
closed forms."""
import math

import numpy as np
import pytest

from oracle import _lib as C
from oracle import ckks
from oracle import params as P

rng = np.random.default_rng(20240601)


def _rand(q, shape):
    return rng.integers(0, q, size=shape, dtype=np.uint64)


def _py_negacyclic(a, b, q):
    n = len(a)
    out = [0] * n
    for i in range(n):
        for j in range(n):
            k = i + j
            if k < n:
                out[k] += int(a[i]) * int(b[j])
            else:
                out[k - n] -= int(a[i]) * int(b[j])
    return [x % q for x in out]


@pytest.mark.parametrize("bits", [40, 60])
def test_schoolbook_matches_python_definition(bits):
    q = P.primes_of_bits(bits, 4, 1)[0]
    a, b = _rand(q, 16), _rand(q, 16)
    got = C.polymul_schoolbook(a[None], b[None], [q])[0]
    assert [int(x) for x in got] == _py_negacyclic(a, b, q)


@pytest.mark.parametrize("logn", [3, 5, 8, 10, 12])
def test_transform_product_matches_schoolbook(logn):
    qs = P.primes_of_bits(60, logn, 2) + P.primes_of_bits(40, logn, 1)
    a = np.stack([_rand(q, 1 << logn) for q in qs])
    b = np.stack([_rand(q, 1 << logn) for q in qs])
    assert np.array_equal(C.polymul(a, b, qs), C.polymul_schoolbook(a, b, qs))


def test_x_times_x_pow_n_minus_1_is_minus_one():
    n = 1 << 10
    q = P.primes_of_bits(50, 10, 1)[0]
    x = np.zeros((1, n), np.uint64)
    y = np.zeros((1, n), np.uint64)
    x[0, 1] = 1
    y[0, n - 1] = 1
    r = C.polymul(x, y, [q])[0]
    assert r[0] == q - 1 and not r[1:].any()


def test_large_product_spot_check():
    n = 1 << 16
    q = P.primes_of_bits(60, 16, 1)[0]
    a, b = _rand(q, n), _rand(q, n)
    c = C.polymul(a[None], b[None], [q])[0]
    for k in (0, 1, 12345, n - 1):
        assert int(c[k]) == C.polymul_coeff(a, b, q, k)


def test_eval_layout_definition_brute_force():
    logn, n = 4, 16
    q = P.primes_of_bits(40, logn, 1)[0]
    psi = P.root_2n(q, logn)
    a = _rand(q, n)
    got = C.eval_at(a, psi, q, logn, np.arange(n))
    for i in range(n):
        e = 2 * int(format(i, "0%db" % logn)[::-1], 2) + 1
        want = sum(int(a[j]) * pow(psi, e * j, q) for j in range(n)) % q
        assert int(got[i]) == want


@pytest.mark.parametrize("logn", [4, 6, 10])
def test_layout_interpolation_inverts_the_evaluation(logn):
    """interp_layout(A) evaluated at the layout points (the independent O(N^2) definition)
    gives back A; closed forms: the all-ones layout is the constant 1, the layout of the
    roots themselves is X."""
    n = 1 << logn
    q = P.primes_of_bits(50, logn, 1)[0]
    psi = P.root_2n(q, logn)
    A = _rand(q, n)
    a = C.interp_layout(A, psi, q, logn)
    assert np.array_equal(C.eval_at(a, psi, q, logn, np.arange(n)), A)
    one = C.interp_layout(np.ones(n, np.uint64), psi, q, logn)
    assert int(one[0]) == 1 and not np.any(one[1:])
    roots = np.array([pow(psi, 2 * int(format(i, "0%db" % logn)[::-1], 2) + 1, q) for i in range(n)], np.uint64)
    x = C.interp_layout(roots, psi, q, logn)
    assert int(x[1]) == 1 and int(x[0]) == 0 and not np.any(x[2:])


def test_automorphism_by_evaluation():
    # (a(X^g))(zeta) = a(zeta^g) at every root zeta = psi^e (e odd) of X^N + 1
    logn, n = 5, 32
    q = P.primes_of_bits(50, logn, 1)[0]
    psi = P.root_2n(q, logn)
    a = _rand(q, n)
    for g in (5, 25, pow(5, -1, 2 * n), 2 * n - 1):
        b = C.automorph(a[None], [q], g)[0]
        for e in (1, 3, 17, 2 * n - 1):
            lhs = sum(int(b[j]) * pow(psi, e * j, q) for j in range(n)) % q
            rhs = sum(int(a[j]) * pow(psi, e * g * j, q) for j in range(n)) % q
            assert lhs == rhs


def test_crt_round_trip():
    qs = P.primes_of_bits(60, 10, 2) + P.primes_of_bits(40, 10, 3)
    Q = math.prod(qs)
    xs = [int(v) for v in rng.integers(-(2 ** 62), 2 ** 62, size=64)]
    xs += [Q // 2, -(Q // 2) + 1, 0, 1, -1]
    x = np.array(xs, dtype=object)
    rows = np.stack([np.array([v % q for v in xs], np.uint64) for q in qs])
    assert list(ckks.crt_centered(rows, qs)) == xs
    small = np.array([v for v in xs if abs(v) < 2 ** 62], np.int64)
    assert list(ckks.crt_centered(C.reduce_signed(small, qs), qs)) == list(small)


@pytest.mark.parametrize("alpha", [1, 2, 4])
def test_bconv_invariant(alpha):
    n = 64
    src = P.primes_of_bits(50, 10, alpha)
    dst = P.primes_of_bits(60, 10, 3) + P.primes_of_bits(40, 10, 2)
    Qs = math.prod(src)
    x = np.stack([_rand(q, n) for q in src])
    x[:, 0] = 0
    x[:, 1] = [q - 1 for q in src]
    out = C.bconv(x, src, dst)
    for c in range(n):
        X = sum(int(x[i, c]) * (Qs // q) * pow(Qs // q, -1, q) for i, q in enumerate(src)) % Qs
        approx = sum((int(x[i, c]) * pow(Qs // q, -1, q) % q) * (Qs // q) for i, q in enumerate(src))
        u = (approx - X) // Qs
        assert (approx - X) % Qs == 0 and 0 <= u < alpha
        for m, d in enumerate(dst):
            assert int(out[m, c]) == (X + u * Qs) % d


def test_moddown_is_floor_minus_small_u():
    orc = ckks.Oracle(logn=6, n_limbs=3, n_special=2, alpha=2, first_bits=60, mid_bits=50, special_bits=60)
    l, n = 3, orc.N
    basis = orc.q[:l] + orc.p
    u = np.stack([_rand(q, n) for q in basis])
    out = orc.moddown(u, l)
    Qall, Q = math.prod(basis), math.prod(orc.q[:l])
    X = ckks.crt_centered(u, basis) % Qall
    got = ckks.crt_centered(out, orc.q[:l]) % Q
    for c in range(n):
        diff = (int(X[c]) // orc.Pprod - int(got[c])) % Q
        assert 0 <= diff < orc.k


@pytest.mark.parametrize("rounding", [True, False])
def test_rescale_exact_division(rounding):
    orc = ckks.Oracle(logn=8, n_limbs=4, n_special=1, alpha=1)
    l, n = 4, orc.N
    qs = orc.q[:l]
    c = np.stack([np.stack([_rand(q, n) for q in qs]) for _ in range(2)])
    c[:, :, 0] = 0
    for i, q in enumerate(qs):
        c[:, i, 1] = q - 1
    out = orc.rescale(ckks.Ciphertext(c, 2.0 ** 80), rounding=rounding)
    Q = math.prod(qs)
    p = qs[-1]
    for poly in range(2):
        C_int = ckks.crt_centered(c[poly], qs) % Q
        for kk in range(l - 1):
            want = [((int(v) + (p // 2 if rounding else 0)) // p) % qs[kk] for v in C_int]
            assert [int(x) for x in out.c[poly, kk]] == want
