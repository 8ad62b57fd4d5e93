"""Host-side pieces of bench.py that its reported numbers rest on: the FP64 references used for
the accuracy figures agree with the oracle's independent ones (the scores of Algorithm 1 and
the gradients of the degree-3 loss, themselves checked by finite differences), and the
whole-job throughput counts every rank's units over the slowest rank's time."""
import numpy as np

import bench
from oracle import fasttext as OF
from paper_1908_06972_gb300 import synth


def test_fp64_scores_match_the_oracle():
    H, O = synth.fasttext_weights(5, 300, 8, 3)
    V = synth.documents(6, 300, 4, 20, 60)
    for v in V:
        assert np.allclose(bench.fp64_scores(v, H, O), OF.plain_scores(v, H, O), rtol=0, atol=1e-15)


def test_fp64_training_gradients_match_the_oracle():
    rng = np.random.default_rng(7)
    V = synth.documents(8, 200, 5, 20, 60)
    Y = np.eye(4)[rng.integers(0, 4, 5)]
    H, O = rng.normal(0, 0.1, (200, 6)), rng.normal(0, 0.1, (6, 4))
    gH, gO = bench.fp64_train_grads(V, Y, H, O)
    rH, rO = OF.train_grads_plain(V, Y, H, O)
    assert np.allclose(gH, rH, rtol=0, atol=1e-14) and np.allclose(gO, rO, rtol=0, atol=1e-14)


def test_throughput_counts_every_rank():
    assert bench.throughput(64 * 5, 1, 2.0) == 160.0
    assert bench.throughput(64 * 5, 8, 2.0) == 8 * 160.0
