"""Pins of the oracle's counter-based sampler against outside definitions.

ChaCha20 is checked against an independent library implementation (the
``cryptography`` package, RFC 8439 keystream); the Gaussian table against
mpmath; the distributions against their moments.
"""
import numpy as np
import pytest

from oracle import _lib as C
from oracle import params as P

SEED = (0x0123456789ABCDEF, 0xFEDCBA9876543210, 0x0F1E2D3C4B5A6978, 0x8877665544332211)


def _keystream_bytes(seed, nonce_words, nblocks):
    """RFC 8439 keystream from the cryptography package (counter starts at 0)."""
    cr = pytest.importorskip("cryptography.hazmat.primitives.ciphers")
    key = b"".join(int(s).to_bytes(8, "little") for s in seed)
    nonce16 = (0).to_bytes(4, "little") + b"".join(int(w).to_bytes(4, "little") for w in nonce_words)
    enc = cr.Cipher(cr.algorithms.ChaCha20(key, nonce16), mode=None).encryptor()
    return enc.update(b"\x00" * (64 * nblocks))


def test_chacha20_block_matches_rfc8439_library():
    words = np.frombuffer(_keystream_bytes(SEED, (7, 11, 13), 3), dtype="<u4")
    key = []
    for s in SEED:
        key += [s & 0xFFFFFFFF, s >> 32]
    for blk in range(3):
        got = C.chacha20_block(key, blk, [7, 11, 13])
        assert np.array_equal(got, words[16 * blk: 16 * blk + 16])


def test_word_stream_layout():
    # word w = block w/8, 32-bit words 2(w%8) (low) and 2(w%8)+1 (high), little endian
    ks = np.frombuffer(_keystream_bytes(SEED, (3, 5, 9), 4), dtype="<u8")
    got = C.stream_words(SEED, 3, 5, 9, 32)
    assert np.array_equal(got, ks)


def test_uniform_is_128bit_word_pair_mod_q():
    q = (1 << 60) - 93 * (1 << 13) + 1  # any modulus works for the layout check
    n = 64
    ks = np.frombuffer(_keystream_bytes(SEED, (2, 0, 4), 16), dtype="<u8")
    want = [((int(ks[2 * c + 1]) << 64) | int(ks[2 * c])) % q for c in range(n)]
    got = C.sample_uniform(SEED, 2, 0, 4, q, n)
    assert [int(x) for x in got] == want


def test_ternary_and_gauss_layout_and_moments():
    n = 1 << 16
    w = C.stream_words(SEED, 1, 0, 0, n)
    t = C.sample_ternary(SEED, 1, 0, 0, n)
    assert np.array_equal(t, (w % np.uint64(3)).astype(np.int64) - 1)
    frac = [np.mean(t == v) for v in (-1, 0, 1)]
    assert all(abs(f - 1 / 3) < 0.01 for f in frac)

    cdt = np.array(P.gauss_cdt("3.2"), np.uint32)
    g = C.sample_gauss(SEED, 3, 0, 0, n, cdt)
    w = C.stream_words(SEED, 3, 0, 0, n)
    top = (w >> np.uint64(32)).astype(np.uint64)
    mag = (top[:, None] >= cdt[None, :].astype(np.uint64)).sum(axis=1)
    sign = (w & np.uint64(1)).astype(bool)
    assert np.array_equal(g, np.where(sign, -mag, mag))
    assert abs(g.mean()) < 0.05
    assert abs(g.std() - 3.2) < 0.05
    assert np.abs(g).max() <= 19


def test_gauss_table_matches_mpmath():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    sigma = mp.mpf("3.2")
    rho = [mp.e ** (-(mp.mpf(k) ** 2) / (2 * sigma ** 2)) for k in range(20)]
    z = rho[0] + 2 * sum(rho[1:])
    want = []
    for j in range(19):
        cdf = (rho[0] + 2 * sum(rho[1: j + 1])) / z
        want.append(int(mp.floor(cdf * 2 ** 32)))
    assert P.gauss_cdt("3.2") == want
    # strictly increasing, and the last entry leaves a positive tail for |x| = 19
    assert all(a < b for a, b in zip(want, want[1:])) and want[-1] < 2 ** 32
