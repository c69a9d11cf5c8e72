"""Pins of the neighbourhood-quality measures (R_NX, recall) by their limits."""
import numpy as np

from paper_2509_07681_gb300.quality import recall, rnx_auc, rnx_curve


def test_rnx_perfect_and_random():
    rng = np.random.default_rng(0)
    N, K = 400, 20
    exact = np.array([rng.permutation(np.delete(np.arange(N), i))[:K] for i in range(N)])
    assert np.allclose(rnx_curve(exact, exact, N), 1.0)
    assert abs(rnx_auc(exact, exact, N) - 1.0) < 1e-12
    rand = np.array([rng.permutation(np.delete(np.arange(N), i))[:K] for i in range(N)])
    assert abs(rnx_auc(rand, exact, N)) < 0.03
    assert recall(exact, exact) == 1.0
    assert recall(rand, exact) < 0.1


def test_recall_ignores_order():
    a = np.array([[1, 2, 3, 4]])
    b = np.array([[4, 3, 9, 1]])
    assert recall(a, b) == 0.75
