"""Build and load the oracle's C primitives (test infrastructure only).

The shared object is compiled with gcc from ``ckks_oracle.c`` into
``oracle/_build/`` on first use (or by ``build()``); nothing of the CUDA
library is involved.
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ckks_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force=False):
    """Compile the oracle C file (plain C, OpenMP over independent rows)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    tmp = _SO + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp", _SRC, "-o", tmp]
    subprocess.check_call(cmd)
    os.replace(tmp, _SO)
    return _SO


_u64p = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_u32p = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
_c = ctypes


def lib():
    global _lib
    with _lock:
        if _lib is None:
            so = build()
            L = ctypes.CDLL(so)
            L.orc_chacha20_block.argtypes = [_u32p, _c.c_uint32, _u32p, _u32p]
            L.orc_stream_words.argtypes = [_u64p, _c.c_uint32, _c.c_uint32, _c.c_uint32, _c.c_uint64, _u64p]
            L.orc_sample_uniform.argtypes = [_u64p, _c.c_uint32, _c.c_uint32, _c.c_uint32, _c.c_uint64, _c.c_int, _u64p]
            L.orc_sample_ternary.argtypes = [_u64p, _c.c_uint32, _c.c_uint32, _c.c_uint32, _c.c_int, _i64p]
            L.orc_sample_gauss.argtypes = [_u64p, _c.c_uint32, _c.c_uint32, _c.c_uint32, _c.c_int, _u32p, _c.c_int, _i64p]
            for name in ("orc_vadd", "orc_vsub", "orc_vmul", "orc_vscale", "orc_polymul", "orc_polymul_schoolbook"):
                getattr(L, name).argtypes = [_u64p, _u64p, _u64p, _c.c_int, _c.c_int, _u64p]
            L.orc_reduce_signed.argtypes = [_i64p, _u64p, _c.c_int, _c.c_int, _u64p]
            L.orc_polymul_coeff.argtypes = [_u64p, _u64p, _c.c_uint64, _c.c_int, _c.c_int]
            L.orc_polymul_coeff.restype = _c.c_uint64
            L.orc_automorph.argtypes = [_u64p, _u64p, _c.c_int, _c.c_int, _c.c_uint64, _u64p]
            L.orc_bconv.argtypes = [_u64p, _u64p, _c.c_int, _u64p, _c.c_int, _c.c_int, _u64p]
            L.orc_eval_at.argtypes = [_u64p, _c.c_uint64, _c.c_uint64, _c.c_int, _i64p, _c.c_int, _u64p]
            L.orc_interp_layout.argtypes = [_u64p, _c.c_uint64, _c.c_uint64, _c.c_int, _u64p]
            _lib = L
    return _lib


def _u64(x):
    return np.ascontiguousarray(x, dtype=np.uint64)


def _rows(x, n):
    x = _u64(x)
    return x.reshape(-1, n), x.size // n


def seed_arr(seed):
    return _u64(list(seed))


# ---- thin wrappers (row-batched) ---------------------------------------------------------

def stream_words(seed, dom, obj, sub, nwords):
    out = np.empty(nwords, np.uint64)
    lib().orc_stream_words(seed_arr(seed), dom, obj, sub, nwords, out)
    return out


def chacha20_block(key_words, counter, nonce_words):
    out = np.empty(16, np.uint32)
    lib().orc_chacha20_block(np.ascontiguousarray(key_words, np.uint32), counter,
                             np.ascontiguousarray(nonce_words, np.uint32), out)
    return out


def sample_uniform(seed, dom, obj, sub, q, n):
    out = np.empty(n, np.uint64)
    lib().orc_sample_uniform(seed_arr(seed), dom, obj, sub, int(q), n, out)
    return out


def sample_ternary(seed, dom, obj, sub, n):
    out = np.empty(n, np.int64)
    lib().orc_sample_ternary(seed_arr(seed), dom, obj, sub, n, out)
    return out


def sample_gauss(seed, dom, obj, sub, n, cdt):
    out = np.empty(n, np.int64)
    cdt = np.ascontiguousarray(cdt, np.uint32)
    lib().orc_sample_gauss(seed_arr(seed), dom, obj, sub, n, cdt, len(cdt), out)
    return out


def _binop(name, x, y, q):
    q = _u64(q)
    n = np.asarray(x).shape[-1]
    xr, rows = _rows(x, n)
    yr, rows2 = _rows(y, n)
    assert rows == rows2 == q.size, (rows, rows2, q.size)
    out = np.empty_like(xr)
    getattr(lib(), name)(xr, yr, q, rows, n, out)
    return out.reshape(np.asarray(x).shape)


def vadd(x, y, q):
    return _binop("orc_vadd", x, y, q)


def vsub(x, y, q):
    return _binop("orc_vsub", x, y, q)


def vmul(x, y, q):
    return _binop("orc_vmul", x, y, q)


def polymul(x, y, q):
    """Row-wise negacyclic product (the oracle's own textbook transform)."""
    return _binop("orc_polymul", x, y, q)


def polymul_schoolbook(x, y, q):
    return _binop("orc_polymul_schoolbook", x, y, q)


def vscale(x, s, q):
    q = _u64(q)
    n = np.asarray(x).shape[-1]
    xr, rows = _rows(x, n)
    out = np.empty_like(xr)
    lib().orc_vscale(xr, _u64(s), q, rows, n, out)
    return out.reshape(np.asarray(x).shape)


def reduce_signed(x, q):
    """Reduce one signed integer polynomial into each modulus of q -> [len(q)][n]."""
    q = _u64(q)
    x = np.ascontiguousarray(x, np.int64)
    out = np.empty((q.size, x.size), np.uint64)
    lib().orc_reduce_signed(x, q, q.size, x.size, out)
    return out


def polymul_coeff(a, b, q, k):
    a, b = _u64(a), _u64(b)
    return int(lib().orc_polymul_coeff(a, b, int(q), a.size, int(k)))


def automorph(x, q, g):
    q = _u64(q)
    n = np.asarray(x).shape[-1]
    xr, rows = _rows(x, n)
    out = np.empty_like(xr)
    lib().orc_automorph(xr, q, rows, n, int(g), out)
    return out.reshape(np.asarray(x).shape)


def bconv(x, src, dst):
    """Fast basis conversion of rows x (mod src primes) to the dst primes."""
    src, dst = _u64(src), _u64(dst)
    n = np.asarray(x).shape[-1]
    xr, rows = _rows(x, n)
    assert rows == src.size
    out = np.empty((dst.size, n), np.uint64)
    lib().orc_bconv(xr, src, src.size, dst, dst.size, n, out)
    return out


def eval_at(a, psi, q, logn, idx):
    """Entries idx of the library's evaluation-domain layout, by definition."""
    idx = np.ascontiguousarray(idx, np.int64)
    out = np.empty(idx.size, np.uint64)
    lib().orc_eval_at(_u64(a), int(psi), int(q), logn, idx, idx.size, out)
    return out


def interp_layout(A, psi, q, logn):
    """Coefficients of the polynomial whose library evaluation layout is A."""
    out = np.empty(1 << logn, np.uint64)
    lib().orc_interp_layout(_u64(A), int(psi), int(q), logn, out)
    return out
