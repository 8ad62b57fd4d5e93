"""Summing ciphertexts across data-parallel ranks (the gradient exchange of Sec. 4.2).

The paper trains with the minibatch split over GPUs, so the ranks' encrypted gradients must
be added.  A ciphertext's words are canonical residues below their limb's prime q; R of them sum
to less than R (q - 1), so when R (q - 1) < 2^64 for every prime of the level the integer sum of
the words is exact and one all-reduce (SUM over int64 words: two's-complement addition is the
same as unsigned 64-bit addition) followed by a reduction modulo each prime gives the sum of the
ciphertexts.  Otherwise the words are gathered and added modulo q one rank at a time.

This module is the collective plumbing only: the reduction and the additions run in the
library's kernels (pft_ct_reduce_sum, pft_add); on a CPU process group the same host logic runs
with the caller's reducer (the tests pass the oracle's)."""
import numpy as np

SUM, GATHER = "sum", "gather"


def exchange_plan(n_ranks, primes):
    """SUM when n_ranks canonical residues of every prime add up below 2^64, else GATHER."""
    return SUM if all(n_ranks * (int(q) - 1) < (1 << 64) for q in primes) else GATHER


def sum_words(words, group=None, plan=None, primes=None, reduce_mod=None):
    """Sum of `words` (an int64 tensor holding uint64 words) over the ranks of `group`.

    plan SUM: one all-reduce; the result holds the exact integer sums (as uint64 bit patterns),
    still to be reduced modulo the primes.  plan GATHER: all-gather, then the modular sum
    reduce_mod(acc, part) rank by rank (acc and part canonical); returns the canonical sum.
    Returns (tensor, plan)."""
    import torch.distributed as dist

    n = dist.get_world_size(group)
    if plan is None:
        plan = exchange_plan(n, primes)
    if plan == SUM:
        out = words.clone()
        dist.all_reduce(out, op=dist.ReduceOp.SUM, group=group)
        return out, SUM
    parts = [words.new_empty(words.shape) for _ in range(n)]
    dist.all_gather(parts, words, group=group)
    acc = parts[0]
    for p in parts[1:]:
        acc = reduce_mod(acc, p)
    return acc, GATHER


def allreduce_ciphertexts(pft, ctx, cts, group=None):
    """Replaces every ciphertext of `cts` (same levels and scales on every rank, on the
    context's device) by its sum over the ranks of `group`, through the library's kernels."""
    import torch
    import torch.distributed as dist

    info = pft.pft_ctx_info(ctx)
    n, primes = info["N"], [int(q) for q in info["primes"]]
    ranks = dist.get_world_size(group)
    for ct in cts:
        level, scale = pft.pft_ct_level(ct), pft.pft_ct_scale(ct)
        buf = torch.empty((2, level, n), dtype=torch.int64, device="cuda")
        pft.pft_ct_copy_out(ctx, ct, buf.data_ptr())
        torch.cuda.synchronize()
        if exchange_plan(ranks, primes[:level]) == SUM:
            dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)
            pft.pft_ct_reduce_sum(ctx, buf.data_ptr(), level, scale, ranks, ct)
        else:
            parts = [torch.empty_like(buf) for _ in range(ranks)]
            dist.all_gather(parts, buf, group=group)
            tmp = pft.pft_ct_create(ctx)
            try:
                pft.pft_ct_reduce_sum(ctx, parts[0].data_ptr(), level, scale, 1, ct)
                for p in parts[1:]:
                    pft.pft_ct_reduce_sum(ctx, p.data_ptr(), level, scale, 1, tmp)
                    pft.pft_add(ctx, ct, tmp, ct)
            finally:
                pft.pft_ct_destroy(tmp)


def as_uint64(t):
    """numpy uint64 view of an int64 tensor (CPU)."""
    return t.numpy().view(np.uint64)
