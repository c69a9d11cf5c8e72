"""The error band of distances to reduced-precision rows, on the CPU.

A candidate row x_c held as x~_c (BF16, or FP8-E4M3 times a per-row scale)
carries E >= ||x_c - x~_c||. For any own row x_i, expanding
||(x_i - x~_c) - (x_c - x~_c)||^2 and applying Cauchy-Schwarz gives
|d2 - d~2| <= 2 ||x_i - x~_c|| E + E^2, with d2 = ||x_i - x_c||^2 and
d~2 = ||x_i - x~_c||^2. The tests check the inequality on random rows and
that it is tight (reached when x_i - x~_c is parallel to x_c - x~_c), so a
band narrower than this formula would let a neighbour be missed."""
import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")


def _fp8_rows(X):
    """E4M3 codes of X / s (round to nearest even, saturating at 448) times
    s, with s = max|x| / 448 per row (1 for a zero row)."""
    s = np.abs(X).max(1, keepdims=True) / 448.0
    s[s == 0] = 1.0
    s = s.astype(np.float32)
    q = torch.from_numpy((X / s).astype(np.float32)).clamp(-448, 448).to(torch.float8_e4m3fn)
    return q.to(torch.float32).numpy().astype(np.float64) * s


def _rows(rng, n, D):
    # offsets, spread scales and tiny entries (FP8 subnormal range)
    X = rng.standard_normal((n, D)) * np.exp(rng.uniform(-3, 3, (n, 1))) + rng.uniform(-20, 20, (n, 1))
    X[:, ::7] *= 1e-3
    return X.astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("fmt", ["bf16", "fp8"])
def test_band_bounds_the_distance_error(fmt):
    rng = np.random.default_rng(80)
    D = 50
    Xc = _rows(rng, 400, D)
    Xq = O.bf16(Xc) if fmt == "bf16" else _fp8_rows(Xc)
    E = np.linalg.norm(Xc - Xq, axis=1)
    assert np.all(E > 0)
    # the stored bound is well below the worst case of the format
    worst = (2.0 ** -8 if fmt == "bf16" else 2.0 ** -4) * np.linalg.norm(Xq, axis=1)
    assert np.median(E / worst) < 0.7
    Xi = Xc[rng.permutation(400)] + rng.standard_normal((400, D)) * 0.1
    dt = np.linalg.norm(Xi - Xq, axis=1)
    d2 = np.sum((Xi - Xc) ** 2, axis=1)
    band = 2 * dt * E + E ** 2
    assert np.all(np.abs(d2 - dt ** 2) <= band * (1 + 1e-12))


@pytest.mark.parametrize("fmt", ["bf16", "fp8"])
def test_band_is_reached_for_aligned_errors(fmt):
    """x_i = x~_c - t (x_c - x~_c) / E puts x_i - x~_c against the rounding
    error: d2 = (t + E)^2 and d~2 = t^2, so d2 - d~2 = 2 t E + E^2 exactly."""
    rng = np.random.default_rng(81)
    Xc = _rows(rng, 50, 32)
    Xq = O.bf16(Xc) if fmt == "bf16" else _fp8_rows(Xc)
    e = Xc - Xq
    E = np.linalg.norm(e, axis=1)
    t = rng.uniform(0.5, 5.0, 50)
    Xi = Xq - (t / E)[:, None] * e
    dt = np.linalg.norm(Xi - Xq, axis=1)
    d2 = np.sum((Xi - Xc) ** 2, axis=1)
    band = 2 * dt * E + E ** 2
    np.testing.assert_allclose(d2 - dt ** 2, band, rtol=1e-9)
