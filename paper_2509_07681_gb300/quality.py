"""Neighbourhood-quality measures used to assess whole runs (host-side numpy).

* ``recall``: mean fraction of the exact k nearest neighbours found.
* ``rnx_curve`` / ``rnx_auc``: R_NX(K) and its area under the log-K curve
  (Lee, Peluffo-Ordonez, Verleysen 2015), the quality measure of the paper's
  Fig. 4 / Fig. 6 / Fig. 7 (Section 3 describes it in words):
      Q_NX(K) = (1 / (K N)) sum_i |nu_i^K  n  n_i^K|
      R_NX(K) = ((N - 1) Q_NX(K) - K) / (N - 1 - K)
      AUC     = sum_K R_NX(K) / K  /  sum_K 1 / K
  R_NX is 0 for random neighbour sets and 1 for perfect retrieval.
"""
from __future__ import annotations

import numpy as np

__all__ = ["recall", "rnx_curve", "rnx_auc", "rnx_points", "overlap_counts"]


def overlap_counts(est: np.ndarray, exact: np.ndarray, K: int) -> np.ndarray:
    """|est_i[:K] n exact_i[:K]| for every row i (rows are neighbour index lists)."""
    a = np.sort(np.asarray(est)[:, :K], axis=1)
    b = np.sort(np.asarray(exact)[:, :K], axis=1)
    cnt = np.zeros(a.shape[0], dtype=np.int64)
    for r in range(a.shape[0]):
        cnt[r] = np.intersect1d(a[r], b[r], assume_unique=True).size
    return cnt


def recall(est: np.ndarray, exact: np.ndarray, k: int | None = None) -> float:
    """Mean fraction of the exact k-NN present in the estimated lists (order ignored)."""
    est = np.asarray(est)
    exact = np.asarray(exact)
    if k is None:
        k = min(est.shape[1], exact.shape[1])
    # vectorised membership: sort each row, then test membership per row
    e = np.sort(est[:, :k], axis=1)
    x = exact[:, :k]
    pos = np.empty_like(x)
    for r in range(x.shape[0]):
        pos[r] = np.searchsorted(e[r], x[r])
    pos = np.minimum(pos, k - 1)
    hit = np.take_along_axis(e, pos, axis=1) == x
    return float(hit.sum()) / float(x.size)


def rnx_curve(est: np.ndarray, exact: np.ndarray, n_points: int, kmax: int | None = None) -> np.ndarray:
    """R_NX(K) for K = 1..kmax, where est/exact are ordered neighbour lists of a
    subset (or all) of the points and n_points is the dataset size N."""
    est = np.asarray(est)
    exact = np.asarray(exact)
    if kmax is None:
        kmax = min(est.shape[1], exact.shape[1])
    N = int(n_points)
    out = np.zeros(kmax)
    for K in range(1, kmax + 1):
        q = overlap_counts(est, exact, K).sum() / (K * est.shape[0])
        out[K - 1] = ((N - 1) * q - K) / (N - 1 - K)
    return out


def rnx_auc(est: np.ndarray, exact: np.ndarray, n_points: int, kmax: int | None = None) -> float:
    r = rnx_curve(est, exact, n_points, kmax)
    K = np.arange(1, len(r) + 1)
    return float((r / K).sum() / (1.0 / K).sum())


def rnx_points(est: np.ndarray, exact: np.ndarray, n_points: int, kmax: int | None = None) -> np.ndarray:
    """Per-point R_NX: row i, column K-1 holds ((N - 1) |nu_i^K n n_i^K| / K - K) / (N - 1 - K),
    whose mean over the rows is rnx_curve. Its spread across points is the
    band of the paper's Fig. 7."""
    est = np.asarray(est)
    exact = np.asarray(exact)
    if kmax is None:
        kmax = min(est.shape[1], exact.shape[1])
    N = int(n_points)
    out = np.zeros((est.shape[0], kmax))
    for K in range(1, kmax + 1):
        q = overlap_counts(est, exact, K) / K
        out[:, K - 1] = ((N - 1) * q - K) / (N - 1 - K)
    return out
