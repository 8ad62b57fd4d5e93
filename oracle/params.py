"""Oracle parameter generation (test infrastructure only).

Prime chain, 2N-th roots and the Gaussian table, computed from their
definitions with Python integers and the ``decimal`` module.

Passages (PrivFT, arXiv 1908.06972):
  * Sec. 2.3: R_q = Z_q[X]/(X^N+1); the chain q_L > ... > q_1 with
    q_l = prod_{i<=l} p_i of word-sized primes.
  * Sec. 4.1 (implementation): the chain is ordered so that each prime is
    smaller than the one before it (p_i < p_{i-1}); rescale drops the last.
  * Sec. 5.4: sigma = 3.2 for the error distribution.
Readings where the paper is silent (prime rule, root rule, table layout) are
the documented sampler/parameter conventions of this project.
"""
from decimal import Decimal, getcontext

# HE-standard style bounds on log2(QP) for a uniform ternary secret at
# 128-bit classical security.
SECURE_LOG_QP = {10: 27, 11: 54, 12: 109, 13: 218, 14: 438, 15: 881, 16: 1772}

_MR_BASES = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37)


def is_prime(n):
    """Deterministic Miller-Rabin for n < 3.3e24 (bases: first 12 primes)."""
    if n < 2:
        return False
    for p in _MR_BASES:
        if n % p == 0:
            return n == p
    d, s = n - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for a in _MR_BASES:
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(s - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def primes_of_bits(bits, logn, count, exclude=()):
    """The first `count` primes among 2^bits - j*2N + 1, j = 1, 2, ...

    Each is = 1 mod 2N (so Z_q holds a primitive 2N-th root) and has exactly
    `bits` bits; the list is in the order found, i.e. descending.
    """
    step = 2 << logn
    out, j = [], 1
    exclude = set(exclude)
    while len(out) < count:
        c = (1 << bits) - j * step + 1
        if c < (1 << (bits - 1)):
            raise ValueError("not enough %d-bit primes for N=2^%d" % (bits, logn))
        if c not in exclude and is_prime(c):
            out.append(c)
        j += 1
    return out


def prime_chain(logn, n_limbs, n_special, first_bits, mid_bits, special_bits):
    """q_0 (first_bits), q_1..q_{L-1} (mid_bits, descending), then the special primes."""
    q0 = primes_of_bits(first_bits, logn, 1)
    mids = primes_of_bits(mid_bits, logn, n_limbs - 1, exclude=q0)
    special = primes_of_bits(special_bits, logn, n_special, exclude=q0 + mids)
    return q0 + mids, special


def root_2n(q, logn):
    """psi = x^((q-1)/2N) for the smallest quadratic non-residue x >= 2."""
    n2 = 2 << logn
    x = 2
    while pow(x, (q - 1) // 2, q) != q - 1:
        x += 1
    psi = pow(x, (q - 1) // n2, q)
    assert pow(psi, n2 // 2, q) == q - 1
    return psi


def gauss_cdt(sigma="3.2"):
    """32-bit cumulative table of |X| for the discrete Gaussian on [-tail, tail],
    tail = floor(6 sigma) (19 for sigma = 3.2).

    P(X = x) is proportional to exp(-x^2 / (2 sigma^2)); T[j] = floor(2^32 *
    P(|X| <= j)) for j = 0 .. tail-1.  A sample's magnitude is the number of
    entries its 32-bit draw reaches.
    """
    getcontext().prec = 60
    s = Decimal(sigma)
    tail = int((6 * s).to_integral_value(rounding="ROUND_FLOOR"))
    rho = [(-(Decimal(k * k)) / (2 * s * s)).exp() for k in range(tail + 1)]
    z = rho[0] + 2 * sum(rho[1:])
    out, acc = [], rho[0]
    for j in range(tail):
        if j > 0:
            acc += 2 * rho[j]
        out.append(int((acc / z * (Decimal(2) ** 32)).to_integral_value(rounding="ROUND_FLOOR")))
    return out
