"""Encrypted fastText training behind ``torch.autograd`` (Sec. 4.2, Algorithm 5).

The weights stay in the library as ciphertexts (``pft_ft_enc_model``).  Autograd sees one
scalar anchor tensor per weight matrix: the forward pass of ``EncryptedFastText.loss`` runs
the encrypted forward pass (``pft_fasttext_train_forward``) and returns a placeholder, since
the loss itself is encrypted and the server cannot read it; ``backward`` runs the library's
homomorphic adjoint (``pft_fasttext_train_backward``) and leaves the encrypted gradients on
the model (``grad_H``, ``grad_O``: ciphertext handles); ``EncryptedSGD.step`` applies the
update (``pft_fasttext_train_update``).  Argument marshalling only: every step runs in the
library's kernels.
"""
import torch

from . import (pft_add_batch, pft_ct_create, pft_ct_destroy, pft_fasttext_train_backward,
               pft_fasttext_train_forward, pft_fasttext_train_spec, pft_fasttext_train_update,
               pft_ft_enc_model_create, pft_ft_enc_model_create_diag, pft_ft_enc_model_destroy,
               pft_ft_enc_model_get, pft_ft_enc_model_levels, pft_ft_tape_destroy)


class EncryptedFastText:
    """H (m x n) and O (n x c) as ciphertexts: H[j] = column j over the vocabulary slots,
    O[j] = row j in slots 0..c-1 one level below H (the handles are copied).  `diag` builds
    the rotation-light layout instead: H_cts = the n diagonals, O_cts = [P], plus the mask
    and the documents' lift (bits)."""

    def __init__(self, ctx, H_cts, O_cts, m, n, c, mask=None, lift_bits=0):
        self.ctx, self.n = ctx, n
        if mask is None:
            self.model = pft_ft_enc_model_create(ctx, H_cts, O_cts, m, n, c)
            self.n_o = n
        else:
            self.model = pft_ft_enc_model_create_diag(ctx, H_cts, O_cts[0], mask, m, n, c, lift_bits)
            self.n_o = 1
        self.anchor_H = torch.zeros((), dtype=torch.float64, requires_grad=True)
        self.anchor_O = torch.zeros((), dtype=torch.float64, requires_grad=True)
        self.grad_H = self.grad_O = None

    @classmethod
    def diag(cls, ctx, D_cts, P_ct, mask, m, n, c, lift_bits=0):
        return cls(ctx, D_cts, [P_ct], m, n, c, mask=mask, lift_bits=lift_bits)

    def parameters(self):
        return [self.anchor_H, self.anchor_O]

    def spec(self, input_scale):
        """(document level, label level, label scale) for documents at input_scale."""
        return pft_fasttext_train_spec(self.ctx, self.model, input_scale)

    def levels(self):
        return pft_ft_enc_model_levels(self.model)

    def loss(self, docs, labels):
        """Encrypted loss of a minibatch (documents and labels w = y - 1/4 as handles);
        the returned tensor is a placeholder for autograd."""
        return _FastTextLoss.apply(self.anchor_H, self.anchor_O, self, list(docs), list(labels))

    def weight(self, which, j):
        """A copy of H_j (which = 0) or O_j (which = 1) as a new ciphertext handle."""
        out = pft_ct_create(self.ctx)
        pft_ft_enc_model_get(self.ctx, self.model, which, j, out)
        return out

    def _add_grads(self, gH, gO):
        if self.grad_H is None:
            self.grad_H, self.grad_O = gH, gO
            return
        pft_add_batch(self.ctx, self.grad_H, gH, self.grad_H)
        pft_add_batch(self.ctx, self.grad_O, gO, self.grad_O)
        for h in gH + gO:
            pft_ct_destroy(h)

    def zero_grad(self):
        for h in (self.grad_H or []) + (self.grad_O or []):
            pft_ct_destroy(h)
        self.grad_H = self.grad_O = None
        for a in self.parameters():
            a.grad = None

    def close(self):
        self.zero_grad()
        if self.model is not None:
            pft_ft_enc_model_destroy(self.model)
            self.model = None


class _FastTextLoss(torch.autograd.Function):
    @staticmethod
    def forward(fctx, anchor_H, anchor_O, model, docs, labels):
        fctx.model = model
        fctx.docs = docs  # the tape reads the documents again in the backward pass
        fctx.tape = pft_fasttext_train_forward(model.ctx, model.model, docs, labels)
        return anchor_H.new_zeros(())

    @staticmethod
    def backward(fctx, grad_out):
        if float(grad_out) != 1.0:
            raise ValueError("the encrypted loss can only be differentiated with an upstream gradient of 1")
        m = fctx.model
        gH = [pft_ct_create(m.ctx) for _ in range(m.n)]
        gO = [pft_ct_create(m.ctx) for _ in range(m.n_o)]
        try:
            pft_fasttext_train_backward(m.ctx, fctx.tape, gH, gO)
        except Exception:
            for h in gH + gO:
                pft_ct_destroy(h)
            raise
        finally:
            pft_ft_tape_destroy(fctx.tape)
            fctx.tape = None
        m._add_grads(gH, gO)
        # the anchors carry no value: the gradients are the ciphertexts left on the model
        return torch.zeros_like(m.anchor_H), torch.zeros_like(m.anchor_O), None, None, None


class EncryptedSGD:
    """Minibatch SGD (Algorithm 5): H <- H - lr dH, O <- O - lr dO on the ciphertexts."""

    def __init__(self, model, lr):
        self.model, self.lr = model, float(lr)

    def step(self):
        m = self.model
        if m.grad_H is None:
            raise RuntimeError("no gradients: call loss.backward() first")
        pft_fasttext_train_update(m.ctx, m.model, m.grad_H, m.grad_O, self.lr)

    def zero_grad(self):
        self.model.zero_grad()
