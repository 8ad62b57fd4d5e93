"""Python binding of libprivft (GB300 RNS-CKKS for encrypted fastText, PrivFT arXiv 1908.06972).

Argument marshalling only: every function below calls the C entry point of the
same name declared in ``include/privft.h``; all arithmetic runs in the CUDA
kernels of the library.  Importing works without a GPU (so host-only utilities
such as ``pft_gen_primes`` can be called), but there is no CPU fallback: if the
shared library has not been built, every call raises ``NativeLibraryMissing``.

Handles are opaque ``ctypes.c_void_p`` values.  Errors raise ``PftError``.
"""
import ctypes
import os
from ctypes import CFUNCTYPE, POINTER, Structure, c_double, c_int, c_int32, c_int64, c_size_t, c_uint32, c_uint64, c_void_p

import numpy as np

from . import _build

_LIB = None

PFT_OK, PFT_ERR_ARG, PFT_ERR_LEVEL_MISMATCH, PFT_ERR_SCALE_MISMATCH, PFT_ERR_NO_KEY = 0, 1, 2, 3, 4
PFT_ERR_OOM, PFT_ERR_CUDA, PFT_ERR_TIMEOUT, PFT_ERR_SECURITY, PFT_ERR_NOT_IMPLEMENTED = 5, 6, 7, 8, 9
PFT_ALLOW_INSECURE = 1
PFT_COMPRESSED_KEYS = 2
PFT_ENC_PK, PFT_ENC_SK = 0, 1
PFT_NTT16_VARIANTS = 4  # N = 2^16 transform variants (pft_autotune, pft_set_transform_variant)


class NativeLibraryMissing(RuntimeError):
    pass


class PftError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("status %d: %s" % (code, msg))
        self.code = code


class pft_params(Structure):
    _fields_ = [("log_n", c_int), ("n_limbs", c_int), ("n_special", c_int), ("alpha", c_int),
                ("first_bits", c_int), ("mid_bits", c_int), ("special_bits", c_int),
                ("primes", POINTER(c_uint64)), ("scale", c_double), ("seed", c_uint64 * 4),
                ("sigma", c_double), ("flags", c_int)]


ALLOC_FN = CFUNCTYPE(c_void_p, c_size_t, c_void_p, c_void_p)
FREE_FN = CFUNCTYPE(None, c_void_p, c_void_p, c_void_p)


class pft_allocator(Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", c_void_p)]


class pft_server_done(Structure):
    _fields_ = [("tag", c_uint64), ("ring", c_int), ("level", c_int), ("scale", c_double),
                ("t_submit", c_double), ("t_done", c_double)]


class pft_job(Structure):
    _fields_ = [("op", c_int), ("a", c_void_p), ("b", c_void_p), ("p", c_void_p), ("out", c_void_p),
                ("after", c_int), ("wait_flag", c_void_p), ("wait_value", ctypes.c_uint32)]


PFT_JOB_ADD, PFT_JOB_SUB, PFT_JOB_MUL_PLAIN = 0, 1, 2


class pft_server_stats(Structure):
    _fields_ = [("waiting", c_int), ("active", c_int), ("exporting", c_int), ("max_active", c_int),
                ("completed", ctypes.c_long), ("iterations", ctypes.c_long), ("bytes_in_use", c_size_t),
                ("peak_bytes", c_size_t), ("budget", c_size_t)]


def build(force=False):
    """Compile the CUDA library (nvcc, sm_103a) into the package's _build folder."""
    return _build.build(force=force)


def lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(_build.SO):
            raise NativeLibraryMissing("libprivft.so is not built (run paper_1908_06972_gb300.build())")
        L = ctypes.CDLL(_build.SO)
        vp, ip, i, u32, u64, d = c_void_p, POINTER(c_int), c_int, c_uint32, POINTER(c_uint64), c_double
        pp = POINTER(c_void_p)
        sig = {
            "pft_ctx_create": [POINTER(pft_params), POINTER(pft_allocator), pp],
            "pft_ctx_destroy": [vp], "pft_set_stream": [vp, vp],
            "pft_ctx_info": [vp, ip, ip, ip, ip, u64],
            "pft_gen_primes": [i, i, i, u64, i, u64],
            "pft_gauss_cdt": [d, POINTER(c_uint32), i, ip],
            "pft_keygen": [vp, POINTER(c_int32), i, i], "pft_add_rotation_keys": [vp, POINTER(c_int32), i],
            "pft_key_export": [vp, u32, u64, c_size_t], "pft_secret_export": [vp, POINTER(c_int64), c_size_t],
            "pft_ct_create": [vp, pp], "pft_ct_destroy": [vp], "pft_pt_destroy": [vp],
            "pft_ct_level": [vp, ip], "pft_ct_scale": [vp, POINTER(c_double)], "pft_pt_level": [vp, ip],
            "pft_ct_data": [vp, POINTER(u64)],
            "pft_encode": [vp, POINTER(c_double), i, d, i, pp], "pft_decode": [vp, vp, POINTER(c_double), i],
            "pft_pt_import": [vp, u64, i, d, pp], "pft_pt_export": [vp, vp, u64, c_size_t],
            "pft_encrypt": [vp, vp, i, u32, pp], "pft_decrypt": [vp, vp, pp],
            "pft_ct_import": [vp, u64, i, d, pp], "pft_ct_export": [vp, vp, u64, c_size_t],
            "pft_ct_import_batch": [vp, pp, ip, POINTER(c_double), i, pp],
            "pft_ct_import_batch_into": [vp, pp, ip, POINTER(c_double), i, pp],
            "pft_ct_export_batch": [vp, pp, i, pp], "pft_ct_export_batch_async": [vp, pp, i, pp],
            "pft_add": [vp, vp, vp, vp], "pft_sub": [vp, vp, vp, vp], "pft_add_plain": [vp, vp, vp, vp],
            "pft_mul_plain": [vp, vp, vp, vp], "pft_mul_relin": [vp, vp, vp, vp],
            "pft_rescale": [vp, vp, vp], "pft_rotate": [vp, vp, c_int32, vp],
            "pft_add_batch": [vp, pp, pp, i, pp], "pft_mul_plain_batch": [vp, pp, pp, i, pp],
            "pft_mul_relin_batch": [vp, pp, pp, i, pp], "pft_rescale_batch": [vp, pp, i, pp],
            "pft_rotate_batch": [vp, pp, i, c_int32, pp],
            "pft_rotate_hoisted": [vp, vp, POINTER(c_int32), i, pp],
            "pft_dot_plain_batch": [vp, pp, pp, i, i, i, pp],
            "pft_drop_level": [vp, vp, i, vp], "pft_add_const": [vp, vp, d, vp],
            "pft_device_status": [vp], "pft_wait_selftest": [vp, ctypes.c_longlong],
            "pft_run_jobs": [vp, POINTER(pft_job), i, c_double], "pft_bfly_ceiling": [vp, POINTER(c_double)],
            "pft_mul_rates": [vp, POINTER(c_double), POINTER(c_double), POINTER(c_double)],
            "pft_autotune_report": [vp, ctypes.c_char_p, c_size_t, POINTER(c_size_t)],
            "pft_set_transform_plan": [vp, i],
            "pft_ct_copy_out": [vp, vp, c_void_p],
            "pft_ct_reduce_sum": [vp, c_void_p, i, d, i, vp],
            "pft_mul_const": [vp, vp, d, d, vp], "pft_ct_set_scale": [vp, d],
            "pft_ntt": [vp, c_void_p, i, i, i],
            "pft_rescale_noalloc": [vp, c_void_p, i, c_void_p],
            "pft_graph_begin": [vp], "pft_graph_end": [vp, pp], "pft_graph_launch": [vp, vp],
            "pft_graph_destroy": [vp],
            "pft_autotune": [vp, POINTER(c_double), i, ip], "pft_set_transform_variant": [vp, i],
            "pft_ft_model_create": [vp, POINTER(c_double), POINTER(c_double), i, i, i, i, pp],
            "pft_ft_model_import": [vp, pp, pp, i, i, i, pp], "pft_ft_model_destroy": [vp],
            "pft_ft_model_create_diag": [vp, POINTER(c_double), POINTER(c_double), i, i, i, i, pp],
            "pft_ft_model_import_diag": [vp, pp, vp, i, i, i, pp],
            "pft_fasttext_infer": [vp, vp, pp, i, vp], "pft_fasttext_infer_batch": [vp, vp, pp, i, i, pp],
            "pft_ft_enc_model_create": [vp, pp, pp, i, i, i, pp], "pft_ft_enc_model_get": [vp, vp, i, i, vp],
            "pft_ft_enc_model_levels": [vp, ip, ip], "pft_ft_enc_model_destroy": [vp],
            "pft_ft_enc_model_create_diag": [vp, pp, vp, vp, i, i, i, i, pp],
            "pft_fasttext_train_spec": [vp, vp, d, ip, ip, POINTER(c_double)],
            "pft_fasttext_train_forward": [vp, vp, pp, pp, i, pp], "pft_ft_tape_score": [vp, vp, i, vp],
            "pft_fasttext_train_backward": [vp, vp, pp, pp], "pft_ft_tape_destroy": [vp],
            "pft_fasttext_train_update": [vp, vp, pp, pp, d],
            "pft_fasttext_train_step": [vp, vp, pp, pp, i, d, pp, pp],
            "pft_server_create": [pp, pp, i, c_size_t, pp], "pft_server_destroy": [vp],
            "pft_server_submit": [vp, i, u64, i, d, u64, c_uint64], "pft_server_step": [vp, ip],
            "pft_server_drain": [vp], "pft_server_poll": [vp, POINTER(pft_server_done), i, ip],
            "pft_server_clock": [vp, POINTER(c_double)],
            "pft_server_get_stats": [vp, POINTER(pft_server_stats)],
            "pft_server_footprint": [vp, i, i, POINTER(c_size_t)],
            "pft_prof_start": [ctypes.c_char_p],
            "pft_prof_stop": [POINTER(c_double), POINTER(ctypes.c_longlong), POINTER(ctypes.c_longlong),
                              POINTER(c_double)],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = c_int
        L.pft_last_error.argtypes = [vp]
        L.pft_last_error.restype = ctypes.c_char_p
        L.pft_server_last_error.argtypes = [vp]
        L.pft_server_last_error.restype = ctypes.c_char_p
        _LIB = L
    return _LIB


def exported_symbols():
    """Names of the C entry points this binding declares (all must exist in the library)."""
    return ["pft_ctx_create", "pft_ctx_destroy", "pft_set_stream", "pft_last_error", "pft_ctx_info",
            "pft_gen_primes", "pft_gauss_cdt", "pft_keygen", "pft_add_rotation_keys", "pft_key_export",
            "pft_secret_export", "pft_ct_create", "pft_ct_destroy", "pft_pt_destroy", "pft_ct_level",
            "pft_ct_scale", "pft_pt_level", "pft_ct_data", "pft_encode", "pft_decode", "pft_pt_import",
            "pft_pt_export", "pft_encrypt", "pft_decrypt", "pft_ct_import", "pft_ct_export", "pft_add",
            "pft_sub", "pft_add_plain", "pft_mul_plain", "pft_mul_relin", "pft_rescale", "pft_rotate",
            "pft_add_batch", "pft_mul_plain_batch", "pft_mul_relin_batch", "pft_rescale_batch",
            "pft_rotate_batch", "pft_ntt", "pft_ft_model_create", "pft_ft_model_import",
            "pft_ft_model_destroy", "pft_fasttext_infer", "pft_fasttext_infer_batch",
            "pft_fasttext_train_step", "pft_prof_start", "pft_prof_stop", "pft_rescale_noalloc",
            "pft_ct_import_batch", "pft_ct_export_batch", "pft_graph_begin", "pft_graph_end",
            "pft_graph_launch", "pft_graph_destroy", "pft_autotune", "pft_set_transform_variant",
            "pft_rotate_hoisted", "pft_ft_model_create_diag", "pft_ft_model_import_diag",
            "pft_dot_plain_batch", "pft_server_create", "pft_server_destroy", "pft_server_last_error",
            "pft_server_submit", "pft_server_step", "pft_server_drain", "pft_server_poll", "pft_server_clock",
            "pft_server_get_stats", "pft_server_footprint", "pft_drop_level", "pft_add_const", "pft_mul_const",
            "pft_ct_set_scale", "pft_ft_enc_model_create", "pft_ft_enc_model_get", "pft_ft_enc_model_levels",
            "pft_ft_enc_model_destroy", "pft_fasttext_train_spec", "pft_fasttext_train_forward", "pft_ft_tape_score",
            "pft_fasttext_train_backward", "pft_ft_tape_destroy", "pft_fasttext_train_update",
            "pft_ct_export_batch_async", "pft_device_status", "pft_wait_selftest", "pft_ft_enc_model_create_diag",
            "pft_run_jobs", "pft_bfly_ceiling", "pft_ct_import_batch_into", "pft_mul_rates",
            "pft_autotune_report", "pft_set_transform_plan", "pft_ct_copy_out", "pft_ct_reduce_sum"]


def _check(rc, ctx=None):
    if rc != PFT_OK:
        msg = lib().pft_last_error(ctx).decode() if ctx else ""
        raise PftError(rc, msg)


def _u64p(a):
    return a.ctypes.data_as(POINTER(c_uint64))


def _arr(handles):
    return (c_void_p * max(1, len(handles)))(*[h.value if isinstance(h, c_void_p) else h for h in handles])


# ---- allocator backed by torch's caching allocator ---------------------------------------
_KEEP = []


def torch_allocator(device=0):
    """A pft_allocator whose memory comes from torch's CUDA caching allocator."""
    import torch

    def _alloc(nbytes, stream, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), device, int(stream or 0))
        except Exception:
            return None

    def _free(ptr, stream, user):
        if ptr:
            torch.cuda.caching_allocator_delete(ptr)

    a = pft_allocator(ALLOC_FN(_alloc), FREE_FN(_free), None)
    _KEEP.append(a)
    return a


# ---- context --------------------------------------------------------------------------------
def pft_ctx_create(log_n, n_limbs, n_special, alpha, first_bits=60, mid_bits=40, special_bits=60,
                   scale=2.0 ** 40, seed=(1, 2, 3, 4), sigma=3.2, flags=0, primes=None, allocator="torch",
                   stream=None):
    """Create a context; allocator "torch" (default), None (cudaMallocAsync) or a pft_allocator."""
    p = pft_params(log_n, n_limbs, n_special, alpha, first_bits, mid_bits, special_bits)
    keep = None
    if primes is not None:
        keep = np.ascontiguousarray(primes, np.uint64)
        p.primes = _u64p(keep)
    p.scale = scale
    p.seed = (c_uint64 * 4)(*[int(s) for s in seed])
    p.sigma = sigma
    p.flags = flags
    if allocator == "torch":
        allocator = torch_allocator()
    out = c_void_p()
    _check(lib().pft_ctx_create(ctypes.byref(p), ctypes.byref(allocator) if allocator is not None else None,
                                ctypes.byref(out)))
    if stream is None and allocator is not None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    if stream:
        _check(lib().pft_set_stream(out, c_void_p(stream)), out)
    del keep
    return out


def pft_ctx_destroy(ctx):
    _check(lib().pft_ctx_destroy(ctx))


def pft_set_stream(ctx, stream):
    _check(lib().pft_set_stream(ctx, c_void_p(stream)), ctx)


def pft_last_error(ctx):
    return lib().pft_last_error(ctx).decode()


def pft_ctx_info(ctx):
    n, L, k, a = c_int(), c_int(), c_int(), c_int()
    _check(lib().pft_ctx_info(ctx, ctypes.byref(n), ctypes.byref(L), ctypes.byref(k), ctypes.byref(a), None), ctx)
    primes = np.zeros(L.value + k.value, np.uint64)
    _check(lib().pft_ctx_info(ctx, None, None, None, None, _u64p(primes)), ctx)
    return {"N": n.value, "L": L.value, "k": k.value, "alpha": a.value, "primes": [int(x) for x in primes]}


def pft_gen_primes(log_n, bits, count, exclude=()):
    ex = np.ascontiguousarray(list(exclude) or [0], np.uint64)
    out = np.zeros(max(1, count), np.uint64)
    _check(lib().pft_gen_primes(log_n, bits, count, _u64p(ex), len(exclude), _u64p(out)))
    return [int(x) for x in out[:count]]


def pft_gauss_cdt(sigma=3.2):
    out = np.zeros(64, np.uint32)
    n = c_int()
    _check(lib().pft_gauss_cdt(sigma, out.ctypes.data_as(POINTER(c_uint32)), 64, ctypes.byref(n)))
    return [int(x) for x in out[: n.value]]


# ---- keys -------------------------------------------------------------------------------------
def pft_keygen(ctx, rot_steps=(), want_relin=True):
    steps = (c_int32 * max(1, len(rot_steps)))(*rot_steps)
    _check(lib().pft_keygen(ctx, steps, len(rot_steps), 1 if want_relin else 0), ctx)


def pft_add_rotation_keys(ctx, rot_steps):
    steps = (c_int32 * max(1, len(rot_steps)))(*rot_steps)
    _check(lib().pft_add_rotation_keys(ctx, steps, len(rot_steps)), ctx)


def pft_key_export(ctx, key_id):
    info = pft_ctx_info(ctx)
    beta = -(-info["L"] // info["alpha"])
    R = info["L"] + info["k"]
    out = np.zeros((beta, 2, R, info["N"]), np.uint64)
    _check(lib().pft_key_export(ctx, key_id, _u64p(out), out.size), ctx)
    return out


def pft_secret_export(ctx):
    n = pft_ctx_info(ctx)["N"]
    out = np.zeros(n, np.int64)
    _check(lib().pft_secret_export(ctx, out.ctypes.data_as(POINTER(c_int64)), n), ctx)
    return out


# ---- plaintexts / ciphertexts ----------------------------------------------------------------
def pft_ct_create(ctx):
    out = c_void_p()
    _check(lib().pft_ct_create(ctx, ctypes.byref(out)), ctx)
    return out


def pft_ct_destroy(ct):
    _check(lib().pft_ct_destroy(ct))


def pft_pt_destroy(pt):
    _check(lib().pft_pt_destroy(pt))


def pft_ct_level(ct):
    v = c_int()
    _check(lib().pft_ct_level(ct, ctypes.byref(v)))
    return v.value


def pft_ct_scale(ct):
    v = c_double()
    _check(lib().pft_ct_scale(ct, ctypes.byref(v)))
    return v.value


def pft_pt_level(pt):
    v = c_int()
    _check(lib().pft_pt_level(pt, ctypes.byref(v)))
    return v.value


def pft_ct_data(ct):
    p = POINTER(c_uint64)()
    _check(lib().pft_ct_data(ct, ctypes.byref(p)))
    return ctypes.cast(p, c_void_p).value


def pft_encode(ctx, z, scale, level):
    z = np.asarray(z, complex)
    buf = np.ascontiguousarray(np.stack([z.real, z.imag], axis=-1).reshape(-1), np.float64)
    out = c_void_p()
    _check(lib().pft_encode(ctx, buf.ctypes.data_as(POINTER(c_double)), z.size, scale, level, ctypes.byref(out)), ctx)
    return out


def pft_decode(ctx, pt, n_slots):
    buf = np.zeros(2 * n_slots, np.float64)
    _check(lib().pft_decode(ctx, pt, buf.ctypes.data_as(POINTER(c_double)), n_slots), ctx)
    return buf[0::2] + 1j * buf[1::2]


def pft_pt_import(ctx, coeffs, scale):
    coeffs = np.ascontiguousarray(coeffs, np.uint64)
    out = c_void_p()
    _check(lib().pft_pt_import(ctx, _u64p(coeffs), coeffs.shape[0], scale, ctypes.byref(out)), ctx)
    return out


def pft_pt_export(ctx, pt):
    n = pft_ctx_info(ctx)["N"]
    out = np.zeros((pft_pt_level(pt), n), np.uint64)
    _check(lib().pft_pt_export(ctx, pt, _u64p(out), out.size), ctx)
    return out


def pft_encrypt(ctx, pt, mode, nonce):
    out = c_void_p()
    _check(lib().pft_encrypt(ctx, pt, mode, nonce, ctypes.byref(out)), ctx)
    return out


def pft_decrypt(ctx, ct):
    out = c_void_p()
    _check(lib().pft_decrypt(ctx, ct, ctypes.byref(out)), ctx)
    return out


def pft_ct_import(ctx, coeffs, scale):
    coeffs = np.ascontiguousarray(coeffs, np.uint64)
    out = c_void_p()
    _check(lib().pft_ct_import(ctx, _u64p(coeffs), coeffs.shape[1], scale, ctypes.byref(out)), ctx)
    return out


def pft_ct_export(ctx, ct, out=None):
    n = pft_ctx_info(ctx)["N"] if out is None else out.shape[-1]
    if out is None:
        out = np.zeros((2, pft_ct_level(ct), n), np.uint64)
    _check(lib().pft_ct_export(ctx, ct, _u64p(out), out.size), ctx)
    return out


def pft_ct_import_batch(ctx, arrays, scales):
    """arrays: list of uint64 [2][l][N] host arrays (pinned for asynchronous copies)."""
    B = len(arrays)
    ptrs = (c_void_p * max(1, B))(*[a.ctypes.data for a in arrays])
    levels = (c_int * max(1, B))(*[a.shape[1] for a in arrays])
    sc = (c_double * max(1, B))(*scales)
    out = (c_void_p * max(1, B))()
    _check(lib().pft_ct_import_batch(ctx, ptrs, levels, sc, B, out), ctx)
    return [c_void_p(out[i]) for i in range(B)]


def pft_ct_import_batch_into(ctx, arrays, scales, cts):
    """Imports arrays[i] into the existing handle cts[i] (its buffer reused when large enough)."""
    B = len(arrays)
    ptrs = (c_void_p * max(1, B))(*[a.ctypes.data for a in arrays])
    levels = (c_int * max(1, B))(*[a.shape[1] for a in arrays])
    sc = (c_double * max(1, B))(*scales)
    _check(lib().pft_ct_import_batch_into(ctx, ptrs, levels, sc, B, _arr(cts)), ctx)


def pft_ct_export_batch(ctx, cts, arrays):
    """Exports cts[i] into the uint64 [2][l][N] host array arrays[i] (one synchronisation)."""
    ptrs = (c_void_p * max(1, len(arrays)))(*[a.ctypes.data for a in arrays])
    _check(lib().pft_ct_export_batch(ctx, _arr(cts), len(cts), ptrs), ctx)
    return arrays


def pft_ct_export_batch_async(ctx, cts, arrays):
    """Queues the export of cts[i] into arrays[i] (page-locked) on the context's stream without
    waiting; the arrays hold the results once that stream has reached this point."""
    ptrs = (c_void_p * max(1, len(arrays)))(*[a.ctypes.data for a in arrays])
    _check(lib().pft_ct_export_batch_async(ctx, _arr(cts), len(cts), ptrs), ctx)
    return arrays


# ---- operations -----------------------------------------------------------------------------
def _op(name, ctx, *args):
    _check(getattr(lib(), name)(ctx, *args), ctx)


def pft_add(ctx, a, b, out):
    _op("pft_add", ctx, a, b, out)


def pft_sub(ctx, a, b, out):
    _op("pft_sub", ctx, a, b, out)


def pft_add_plain(ctx, a, p, out):
    _op("pft_add_plain", ctx, a, p, out)


def pft_mul_plain(ctx, a, p, out):
    _op("pft_mul_plain", ctx, a, p, out)


def pft_mul_relin(ctx, a, b, out):
    _op("pft_mul_relin", ctx, a, b, out)


def pft_rescale(ctx, a, out):
    _op("pft_rescale", ctx, a, out)


def pft_rotate(ctx, a, step, out):
    _op("pft_rotate", ctx, a, c_int32(step), out)


def pft_add_batch(ctx, a, b, out):
    _op("pft_add_batch", ctx, _arr(a), _arr(b), len(a), _arr(out))


def pft_mul_plain_batch(ctx, a, p, out):
    _op("pft_mul_plain_batch", ctx, _arr(a), _arr(p), len(a), _arr(out))


def pft_mul_relin_batch(ctx, a, b, out):
    _op("pft_mul_relin_batch", ctx, _arr(a), _arr(b), len(a), _arr(out))


def pft_rescale_batch(ctx, a, out):
    _op("pft_rescale_batch", ctx, _arr(a), len(a), _arr(out))


def pft_rotate_batch(ctx, a, step, out):
    _op("pft_rotate_batch", ctx, _arr(a), len(a), c_int32(step), _arr(out))


def pft_device_status(ctx):
    """Raises PftError(PFT_ERR_TIMEOUT) if a bounded device wait expired since the last check."""
    _check(lib().pft_device_status(ctx), ctx)


def pft_wait_selftest(ctx, polls):
    _check(lib().pft_wait_selftest(ctx, int(polls)), ctx)


def pft_mul_rates(ctx):
    """Measured 32-bit multiply issue rates (ops/s, whole GPU): (low-word, high-word, widening)."""
    lo, hi, wide = c_double(), c_double(), c_double()
    _check(lib().pft_mul_rates(ctx, ctypes.byref(lo), ctypes.byref(hi), ctypes.byref(wide)), ctx)
    return lo.value, hi.value, wide.value


def pft_bfly_ceiling(ctx):
    """Butterflies per second of the transforms' butterfly arithmetic on register data."""
    v = c_double()
    _check(lib().pft_bfly_ceiling(ctx, ctypes.byref(v)), ctx)
    return v.value


def pft_run_jobs(ctx, jobs, wait_timeout_s=1.0):
    """One persistent launch over elementwise jobs of any contexts and levels.  Each job is a
    dict: op (PFT_JOB_*), a, b or p, out, optional after (index or -1), wait_flag (device
    address of a 32-bit word) and wait_value."""
    arr = (pft_job * max(1, len(jobs)))()
    for k, j in enumerate(jobs):
        h = lambda x: None if x is None else (x.value if isinstance(x, c_void_p) else x)  # noqa: E731
        arr[k] = pft_job(int(j["op"]), h(j["a"]), h(j.get("b")), h(j.get("p")), h(j["out"]), int(j.get("after", -1)),
                         j.get("wait_flag"), int(j.get("wait_value", 0)))
    _check(lib().pft_run_jobs(ctx, arr, len(jobs), float(wait_timeout_s)), ctx)


def pft_drop_level(ctx, a, level, out):
    _op("pft_drop_level", ctx, a, level, out)


def pft_add_const(ctx, a, value, out):
    _op("pft_add_const", ctx, a, float(value), out)


def pft_mul_const(ctx, a, value, const_scale, out):
    _op("pft_mul_const", ctx, a, float(value), float(const_scale), out)


def pft_ct_set_scale(ct, scale):
    _check(lib().pft_ct_set_scale(ct, float(scale)))


def pft_dot_plain_batch(ctx, cts, pts, K, outs, pts_shared=False):
    _op("pft_dot_plain_batch", ctx, _arr(cts), _arr(pts), K, len(outs), 1 if pts_shared else 0, _arr(outs))


def pft_rotate_hoisted(ctx, a, steps, outs):
    st = (c_int32 * max(1, len(steps)))(*steps)
    _op("pft_rotate_hoisted", ctx, a, st, len(steps), _arr(outs))


def pft_ntt(ctx, data_ptr, n_polys, n_limbs, inverse):
    """In-place transform of caller device memory (an int device pointer, e.g. tensor.data_ptr())."""
    _op("pft_ntt", ctx, c_void_p(data_ptr), n_polys, n_limbs, 1 if inverse else 0)


def pft_rescale_noalloc(ctx, in_ptr, level, out_ptr):
    """Rescale of raw device buffers (int device pointers) without any device allocation:
    for callers that cannot allocate device memory when they call the library.  The library
    uses a fixed 32 MiB array as working space (shared by all calls on a device)."""
    _op("pft_rescale_noalloc", ctx, c_void_p(in_ptr), level, c_void_p(out_ptr))


def pft_autotune(ctx):
    """Times the transform variants, keeps the fastest; returns (chosen index, times in us)."""
    us = (c_double * 16)()
    chosen = c_int()
    _check(lib().pft_autotune(ctx, us, 16, ctypes.byref(chosen)), ctx)
    return chosen.value, [us[i] for i in range(16)]


def pft_autotune_report(ctx):
    """The last autotuning search as a dict (parsed from the library's JSON text)."""
    import json
    n = c_size_t()
    _check(lib().pft_autotune_report(ctx, None, 0, ctypes.byref(n)), ctx)
    buf = ctypes.create_string_buffer(n.value + 1)
    _check(lib().pft_autotune_report(ctx, buf, n.value + 1, None), ctx)
    return json.loads(buf.value.decode())


def pft_ct_copy_out(ctx, ct, dev_ptr):
    """Copy ct's [2][l][N] words (evaluation layout) to caller device memory (int pointer)."""
    _check(lib().pft_ct_copy_out(ctx, ct, c_void_p(dev_ptr)), ctx)


def pft_ct_reduce_sum(ctx, dev_ptr, level, scale, n_terms, out):
    """out = the ciphertext whose words are the integer sums at dev_ptr reduced mod each prime."""
    _check(lib().pft_ct_reduce_sum(ctx, c_void_p(dev_ptr), level, scale, n_terms, out), ctx)


def pft_set_transform_plan(ctx, plan):
    _check(lib().pft_set_transform_plan(ctx, plan), ctx)


def pft_set_transform_variant(ctx, variant):
    _check(lib().pft_set_transform_variant(ctx, variant), ctx)


def pft_graph_begin(ctx):
    _check(lib().pft_graph_begin(ctx), ctx)


def pft_graph_end(ctx):
    out = c_void_p()
    _check(lib().pft_graph_end(ctx, ctypes.byref(out)), ctx)
    return out


def pft_graph_launch(ctx, graph):
    _check(lib().pft_graph_launch(ctx, graph), ctx)


def pft_graph_destroy(graph):
    _check(lib().pft_graph_destroy(graph))


def pft_ft_model_create(ctx, H, O, level):
    H = np.ascontiguousarray(H, np.float64)
    O = np.ascontiguousarray(O, np.float64)
    out = c_void_p()
    _check(lib().pft_ft_model_create(ctx, H.ctypes.data_as(POINTER(c_double)), O.ctypes.data_as(POINTER(c_double)),
                                     H.shape[0], H.shape[1], O.shape[1], level, ctypes.byref(out)), ctx)
    return out


def pft_ft_model_import(ctx, H_pts, O_pts, m, n, c):
    out = c_void_p()
    _check(lib().pft_ft_model_import(ctx, _arr(H_pts), _arr(O_pts), m, n, c, ctypes.byref(out)), ctx)
    return out


def pft_ft_model_create_diag(ctx, H, O, level):
    H = np.ascontiguousarray(H, np.float64)
    O = np.ascontiguousarray(O, np.float64)
    out = c_void_p()
    _check(lib().pft_ft_model_create_diag(ctx, H.ctypes.data_as(POINTER(c_double)),
                                          O.ctypes.data_as(POINTER(c_double)), H.shape[0], H.shape[1], O.shape[1],
                                          level, ctypes.byref(out)), ctx)
    return out


def pft_ft_model_import_diag(ctx, D_pts, P_pt, m, n, c):
    out = c_void_p()
    _check(lib().pft_ft_model_import_diag(ctx, _arr(D_pts), P_pt, m, n, c, ctypes.byref(out)), ctx)
    return out


def pft_ft_model_destroy(model):
    _check(lib().pft_ft_model_destroy(model))


def pft_fasttext_infer(ctx, model, v, scores):
    _op("pft_fasttext_infer", ctx, model, _arr(v), len(v), scores)


def pft_fasttext_infer_batch(ctx, model, v, n_chunks, scores):
    _op("pft_fasttext_infer_batch", ctx, model, _arr(v), n_chunks, len(scores), _arr(scores))


# ---- encrypted training (Sec. 4.2, Algorithm 5) ---------------------------------------------------
def pft_ft_enc_model_create(ctx, H, O, m, n, c):
    out = c_void_p()
    _check(lib().pft_ft_enc_model_create(ctx, _arr(H), _arr(O), m, n, c, ctypes.byref(out)), ctx)
    return out


def pft_ft_enc_model_create_diag(ctx, D, P, mask, m, n, c, lift_bits=0):
    out = c_void_p()
    _check(lib().pft_ft_enc_model_create_diag(ctx, _arr(D), P, mask, m, n, c, lift_bits, ctypes.byref(out)), ctx)
    return out


def pft_ft_enc_model_get(ctx, model, which, j, out):
    _op("pft_ft_enc_model_get", ctx, model, which, j, out)


def pft_ft_enc_model_levels(model):
    a, b = c_int(), c_int()
    _check(lib().pft_ft_enc_model_levels(model, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def pft_ft_enc_model_destroy(model):
    _check(lib().pft_ft_enc_model_destroy(model))


def pft_fasttext_train_spec(ctx, model, input_scale):
    """(document level, label level, label scale)."""
    dl, ll, ls = c_int(), c_int(), c_double()
    _check(lib().pft_fasttext_train_spec(ctx, model, float(input_scale), ctypes.byref(dl), ctypes.byref(ll),
                                         ctypes.byref(ls)), ctx)
    return dl.value, ll.value, ls.value


def pft_fasttext_train_forward(ctx, model, docs, labels):
    out = c_void_p()
    _check(lib().pft_fasttext_train_forward(ctx, model, _arr(docs), _arr(labels), len(docs), ctypes.byref(out)), ctx)
    return out


def pft_ft_tape_score(ctx, tape, b, out):
    _op("pft_ft_tape_score", ctx, tape, b, out)


def pft_fasttext_train_backward(ctx, tape, grad_H, grad_O):
    _op("pft_fasttext_train_backward", ctx, tape, _arr(grad_H), _arr(grad_O))


def pft_ft_tape_destroy(tape):
    _check(lib().pft_ft_tape_destroy(tape))


def pft_fasttext_train_update(ctx, model, grad_H, grad_O, eta):
    _op("pft_fasttext_train_update", ctx, model, _arr(grad_H), _arr(grad_O), float(eta))


def pft_fasttext_train_step(ctx, model, docs, labels, eta, grad_H=None, grad_O=None):
    gh = _arr(grad_H) if grad_H is not None else None
    go = _arr(grad_O) if grad_O is not None else None
    _op("pft_fasttext_train_step", ctx, model, _arr(docs), _arr(labels), len(docs), float(eta), gh, go)


# ---- request server -----------------------------------------------------------------------
def _scheck(rc, srv):
    if rc != PFT_OK:
        raise PftError(rc, lib().pft_server_last_error(srv).decode())


def pft_server_create(ctxs, models, budget_bytes=0):
    out = c_void_p()
    rc = lib().pft_server_create(_arr(ctxs), _arr(models), len(ctxs), budget_bytes, ctypes.byref(out))
    if rc != PFT_OK:
        raise PftError(rc, lib().pft_server_last_error(None).decode())
    return out


def pft_server_destroy(srv):
    _check(lib().pft_server_destroy(srv))


def pft_server_submit(srv, ring, coeffs, level, scale, out, tag):
    """coeffs: uint64 [chunks][2][level][N] (kept alive by the caller until the request is
    polled); out: uint64 array of 2 (level-2) N words, written on completion."""
    assert coeffs.dtype == np.uint64 and coeffs.flags.c_contiguous
    assert out.dtype == np.uint64 and out.flags.c_contiguous and out.flags.writeable
    _scheck(lib().pft_server_submit(srv, ring, _u64p(coeffs), level, scale, _u64p(out), tag), srv)


def pft_server_step(srv):
    n = c_int()
    _scheck(lib().pft_server_step(srv, ctypes.byref(n)), srv)
    return n.value


def pft_server_drain(srv):
    _scheck(lib().pft_server_drain(srv), srv)


def pft_server_poll(srv, max_n=256):
    """Completed requests: list of dicts (tag, ring, level, scale, t_submit, t_done)."""
    buf = (pft_server_done * max_n)()
    n = c_int()
    _scheck(lib().pft_server_poll(srv, buf, max_n, ctypes.byref(n)), srv)
    return [{f: getattr(buf[k], f) for f, _ in pft_server_done._fields_} for k in range(n.value)]


def pft_server_clock(srv):
    t = c_double()
    _scheck(lib().pft_server_clock(srv, ctypes.byref(t)), srv)
    return t.value


def pft_server_get_stats(srv):
    st = pft_server_stats()
    _scheck(lib().pft_server_get_stats(srv, ctypes.byref(st)), srv)
    return {f: getattr(st, f) for f, _ in pft_server_stats._fields_}


def pft_server_footprint(srv, ring, level):
    b = c_size_t()
    _scheck(lib().pft_server_footprint(srv, ring, level, ctypes.byref(b)), srv)
    return b.value


# ---- launch accounting ------------------------------------------------------------------------
def pft_prof_start(prefix=""):
    _check(lib().pft_prof_start(prefix.encode()))


def pft_prof_stop():
    """(device ms of the timed launches, their number, number of all launches, their algorithmic work)."""
    ms, n, tot, work = c_double(), ctypes.c_longlong(), ctypes.c_longlong(), c_double()
    _check(lib().pft_prof_stop(ctypes.byref(ms), ctypes.byref(n), ctypes.byref(tot), ctypes.byref(work)))
    return ms.value, n.value, tot.value, work.value
