"""ORACLE for the PrivFT RNS-CKKS hot path -- TEST INFRASTRUCTURE ONLY.

A plain, slow CPU restatement of what the GPU library computes: coefficient
form everywhere, 128-bit products reduced with `%`, textbook transforms,
Python integers for CRT.  Only tests/, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it; the product never does.

Modules:
  _lib      -- gcc-built C primitives (ChaCha20 sampler, modular rows,
               negacyclic products, automorphism, fast basis conversion,
               definitional evaluation of the library's transform layout)
  params    -- prime chain, 2N-th roots, Gaussian table, security bounds
  ckks      -- keygen, encode/decode, encrypt/decrypt, HADD/HMUL/HMULPLAIN,
               key switching (ModUp/ModDown), ROTATE, RESCALE, TotalSum
  fasttext  -- Algorithm 1 in FP64 and the encrypted inference sequence
"""
from . import _lib, params, ckks, fasttext  # noqa: F401
from ._lib import build  # noqa: F401
