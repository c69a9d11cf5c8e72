"""Pins of the neighbourhood-quality measures (R_NX, recall) by their limits."""
import numpy as np

from paper_2509_07681_gb300.quality import recall, rnx_auc, rnx_curve, rnx_points


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


def test_rnx_points_average_to_the_curve():
    rng = np.random.default_rng(1)
    N, K = 300, 16
    exact = np.array([rng.permutation(np.delete(np.arange(N), i))[:K] for i in range(N)])
    est = exact.copy()
    est[::3, K // 2:] = (est[::3, K // 2:] + 7) % N  # a third of the rows lose half their tail
    per = rnx_points(est, exact, N)
    np.testing.assert_allclose(per.mean(0), rnx_curve(est, exact, N), rtol=1e-12, atol=1e-15)
    assert np.all(per[1::3] == 1.0) and per[::3, -1].max() < 1.0
