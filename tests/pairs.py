"""Matched (GPU context, oracle) pairs built from the same parameters and seed."""
import numpy as np

from oracle import ckks


class Pair:
    def __init__(self, pft, logn, L, k, alpha, first_bits=60, mid_bits=40, special_bits=60, scale=2.0 ** 40,
                 seed=(0x5EED, 11, 22, 33), rot_steps=(), relin=True, insecure=True, gpu_keys=True, compressed=False):
        self.pft = pft
        self.orc = ckks.Oracle(logn, L, k, alpha, first_bits, mid_bits, special_bits, scale, seed,
                               compressed_keys=compressed)
        flags = (pft.PFT_ALLOW_INSECURE if insecure else 0) | (pft.PFT_COMPRESSED_KEYS if compressed else 0)
        self.ctx = pft.pft_ctx_create(logn, L, k, alpha, first_bits, mid_bits, special_bits, scale, seed,
                                      flags=flags)
        self.N = 1 << logn
        self.rot_steps = tuple(rot_steps)
        if gpu_keys:
            pft.pft_keygen(self.ctx, list(rot_steps), relin)
        self.orc.keygen(rot_steps, relin)
        self.handles = []

    # oracle objects -> GPU handles (coefficient form, identical integers)
    def ct(self, oct_):
        h = self.pft.pft_ct_import(self.ctx, oct_.c, oct_.scale)
        self.handles.append(("ct", h))
        return h

    def pt(self, opt):
        h = self.pft.pft_pt_import(self.ctx, opt.m, opt.scale)
        self.handles.append(("pt", h))
        return h

    def empty(self):
        h = self.pft.pft_ct_create(self.ctx)
        self.handles.append(("ct", h))
        return h

    def export(self, h):
        return self.pft.pft_ct_export(self.ctx, h)

    def assert_equal(self, h, oct_, what=""):
        got = self.export(h)
        assert got.shape == oct_.c.shape, (what, got.shape, oct_.c.shape)
        bad = np.argwhere(got != oct_.c)
        assert bad.size == 0, "%s: %d mismatching words, first at %s" % (what, len(bad), bad[:3].tolist())
        assert self.pft.pft_ct_scale(h) == oct_.scale, what

    def close(self):
        for kind, h in self.handles:
            (self.pft.pft_ct_destroy if kind == "ct" else self.pft.pft_pt_destroy)(h)
        self.handles = []
        self.pft.pft_ctx_destroy(self.ctx)
