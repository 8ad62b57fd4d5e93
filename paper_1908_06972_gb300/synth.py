"""Seeded synthetic inputs shaped like the paper's workloads (no CKKS arithmetic here).

* slot vectors: i.i.d. uniform complex values in [-1, 1]^2 (the micro-benchmark inputs);
* fastText weights: H (m x n) and O (n x c) with i.i.d. N(0, std^2) entries, standing
  in for trained fastText models (Sec. 5.5.1; trained models are not available);
* documents: lengths uniform in [w_min, w_max] tokens, token ids from a truncated
  Zipf law P(k) ~ (k + 1)^(-a), k < m, standing in for the paper's text datasets;
  the client vector is the normalised count vector v = (1/w) sum_i x_i (Sec. 3.1).
"""
import numpy as np


def slots(seed, n):
    rng = np.random.default_rng(seed)
    return rng.uniform(-1, 1, n) + 1j * rng.uniform(-1, 1, n)


def residues(seed, primes, n, polys=1):
    """Uniform residues [polys][len(primes)][n] (canonical, below each prime)."""
    rng = np.random.default_rng(seed)
    out = np.empty((polys, len(primes), n), np.uint64)
    for p in range(polys):
        for i, q in enumerate(primes):
            out[p, i] = rng.integers(0, int(q), n, dtype=np.uint64)
    return out


def fasttext_weights(seed, m, n, c, std=0.1):
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, std, (m, n)), rng.normal(0.0, std, (n, c))


def documents(seed, m, count, w_min=20, w_max=200, a=1.1):
    """Normalised count vectors [count][m] of Zipf(a) documents."""
    rng = np.random.default_rng(seed)
    k = np.arange(m)
    p = (k + 1.0) ** (-a)
    p /= p.sum()
    out = np.zeros((count, m))
    for d in range(count):
        w = int(rng.integers(w_min, w_max + 1))
        ids = rng.choice(m, size=w, p=p)
        out[d] = np.bincount(ids, minlength=m) / w
    return out


def batch_levels(count=64, lo=5, hi=30, seed=20241203):
    """Levels of a batch of ciphertexts, uniform in [lo, hi] (the mixed-level batch workload)."""
    rng = np.random.default_rng(seed)
    return [int(x) for x in rng.integers(lo, hi + 1, count)]
