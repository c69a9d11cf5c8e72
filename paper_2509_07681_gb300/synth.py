"""Seeded synthetic workloads for the FUnc-SNE step.

This module only draws input data (numpy PCG64, seed 0 by default). It holds
none of the method's arithmetic, so both the CUDA path and the CPU oracle may
use it. The paper evaluates on MNIST, RNA-seq and ImageNet/EVA features (its
Section 4); none of those are available, so each workload below is a stand-in
with the shape, size and cluster structure of the paper's use:

* ``blobs``      -- isotropic Gaussian mixture, the paper's "Gaussian blobs"
                    (Fig. 6/7): N=2000, D=50, 10 clusters.
* ``pixels``     -- MNIST-shaped data (N=70000, D=784, values k/255 in [0,1],
                    ~50% zeros) from 10 blobs in a 20-d latent pushed through a
                    random ReLU map (stand-in for the MNIST runs of Fig. 3).
* ``spectrum``   -- N=1,000,000, D=50 with feature variance ~1/j over 50
                    anisotropic clusters of Zipf sizes (stand-in for the usual
                    "PCA to 50 components" preprocessing of Section 3).
* ``swissroll``  -- D=128, 32 Gaussian clusters on a swiss roll in dims 0-2
                    (dynamic-dataset workload; drawn in batches).
* ``lowrank``    -- N=2,000,000, D=256 low-rank (30-d latent) mixture plus
                    N(0, 0.1^2) noise (stand-in for the 192-PC ImageNet run).
"""
from __future__ import annotations

import math

import numpy as np

__all__ = ["blobs", "pixels", "spectrum", "swissroll", "lowrank", "integer_grid",
           "WORKLOADS", "make"]


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def blobs(n: int = 2000, dim: int = 50, n_clusters: int = 10, centre_std: float = 4.0,
          sigma: float = 1.0, seed: int = 0) -> np.ndarray:
    """Equal-weight isotropic Gaussian mixture; centres ~ N(0, centre_std^2 I)."""
    g = _rng(seed)
    centres = g.standard_normal((n_clusters, dim)) * centre_std
    lab = np.arange(n) % n_clusters
    g.shuffle(lab)
    x = centres[lab] + sigma * g.standard_normal((n, dim))
    return np.ascontiguousarray(x, dtype=np.float32)


def pixels(n: int = 70000, dim: int = 784, latent: int = 10 * 2, n_clusters: int = 10,
           seed: int = 0) -> np.ndarray:
    """uint8/255-valued rows: round(255 * clip(relu(z W), 0, 1)) / 255.

    z comes from ``n_clusters`` blobs in a ``latent``-d space (centres N(0,16 I),
    sigma 1); W ~ N(0, s^2) with s chosen so the pre-activation std is ~0.5,
    which leaves about half of the pixels at zero.
    """
    g = _rng(seed)
    centres = g.standard_normal((n_clusters, latent)) * 4.0
    lab = np.arange(n) % n_clusters
    g.shuffle(lab)
    z = centres[lab] + g.standard_normal((n, latent))
    s = 0.5 / math.sqrt(latent * 17.0)
    w = g.standard_normal((latent, dim)) * s
    out = np.empty((n, dim), dtype=np.float32)
    step = 8192
    for a in range(0, n, step):
        pre = z[a:a + step] @ w
        q = np.rint(255.0 * np.clip(pre, 0.0, 1.0))
        out[a:a + step] = (q / 255.0).astype(np.float32)
    return out


def _zipf_sizes(n: int, k: int) -> np.ndarray:
    wts = 1.0 / np.arange(1, k + 1)
    sizes = np.floor(n * wts / wts.sum()).astype(np.int64)
    sizes[0] += n - sizes.sum()
    return sizes


def spectrum(n: int = 1_000_000, dim: int = 50, n_clusters: int = 50, seed: int = 0) -> np.ndarray:
    """Zipf-sized anisotropic clusters, then feature j (1-based) scaled by 1/sqrt(j).

    Each cluster: centre ~ N(0, 16 I); samples = centre + (e * s) Q^T with
    e ~ N(0, I), s_j ~ U[0.25, 1] and Q a random rotation (QR of a Gaussian).
    """
    g = _rng(seed)
    sizes = _zipf_sizes(n, n_clusters)
    scale = 1.0 / np.sqrt(np.arange(1, dim + 1, dtype=np.float64))
    out = np.empty((n, dim), dtype=np.float32)
    pos = 0
    for c in range(n_clusters):
        centre = g.standard_normal(dim) * 4.0
        q, r = np.linalg.qr(g.standard_normal((dim, dim)))
        q = q * np.sign(np.diag(r))
        s = g.uniform(0.25, 1.0, size=dim)
        m = int(sizes[c])
        e = g.standard_normal((m, dim)) * s
        out[pos:pos + m] = ((centre + e @ q.T) * scale).astype(np.float32)
        pos += m
    perm = g.permutation(n)
    return np.ascontiguousarray(out[perm])


def swissroll(n: int = 200_000, dim: int = 128, n_clusters: int = 32, seed: int = 0,
              batch: int = 0) -> np.ndarray:
    """Gaussian clusters on a swiss roll in dims 0-2, isotropic noise elsewhere.

    Cluster k sits at roll parameter t_k = 1.5 pi + 3 pi k / (n_clusters - 1)
    and height h_k ~ U(0, 21), i.e. centre (t cos t, h, t sin t, 0, ...).
    Noise std 0.5 in dims 0-2 and 0.1 in the rest. ``batch`` selects an
    independent draw from the same generator (for later insertions); the
    cluster geometry depends on ``seed`` only.
    """
    g = _rng(seed)
    t = 1.5 * math.pi + 3.0 * math.pi * np.arange(n_clusters) / (n_clusters - 1)
    h = g.uniform(0.0, 21.0, size=n_clusters)
    centres = np.zeros((n_clusters, dim))
    centres[:, 0] = t * np.cos(t)
    centres[:, 1] = h
    centres[:, 2] = t * np.sin(t)
    gb = _rng(seed * 1_000_003 + 7919 * (batch + 1))
    lab = gb.integers(0, n_clusters, size=n)
    noise = gb.standard_normal((n, dim)) * 0.1
    noise[:, :3] *= 5.0
    return np.ascontiguousarray(centres[lab] + noise, dtype=np.float32)


def lowrank(n: int = 2_000_000, dim: int = 256, latent: int = 30, n_comp: int = 100,
            seed: int = 0) -> np.ndarray:
    """z from a ``latent``-d mixture (centres N(0, 4 I), sigma 1) mapped by a random
    orthonormal latent x dim matrix, plus N(0, 0.1^2) noise. Returned as float32;
    the workload stores it in bfloat16."""
    g = _rng(seed)
    centres = g.standard_normal((n_comp, latent)) * 2.0
    q, _ = np.linalg.qr(g.standard_normal((dim, latent)))
    basis = q.T  # latent x dim, orthonormal rows
    out = np.empty((n, dim), dtype=np.float32)
    step = 65536
    for a in range(0, n, step):
        m = min(step, n - a)
        lab = g.integers(0, n_comp, size=m)
        z = centres[lab] + g.standard_normal((m, latent))
        out[a:a + m] = (z @ basis + 0.1 * g.standard_normal((m, dim))).astype(np.float32)
    return out


def integer_grid(n: int, dim: int, high: int = 4, seed: int = 0) -> np.ndarray:
    """Small-integer coordinates: every squared distance is an exact small
    integer in float32 and float64, so distance ties are exact on both sides."""
    g = _rng(seed)
    return g.integers(0, high, size=(n, dim)).astype(np.float32)


# name -> (generator, keyword arguments, method parameters)
WORKLOADS = {
    "blobs-2k": (blobs, dict(n=2000, dim=50),
                 dict(d=2, k_hd=32, k_ld=16, n_neg=16, alpha=1.0, perplexity=30.0)),
    "pixels-70k": (pixels, dict(n=70000, dim=784),
                   dict(d=2, k_hd=32, k_ld=16, n_neg=16, alpha=1.0, perplexity=30.0)),
    "spectrum-1m": (spectrum, dict(n=1_000_000, dim=50),
                    dict(d=16, k_hd=32, k_ld=32, n_neg=32, alpha=1.0, perplexity=30.0)),
    "swissroll-200k": (swissroll, dict(n=200_000, dim=128),
                       dict(d=8, k_hd=32, k_ld=16, n_neg=16, alpha=1.0, perplexity=30.0)),
    "lowrank-2m": (lowrank, dict(n=2_000_000, dim=256),
                   dict(d=32, k_hd=64, k_ld=32, n_neg=32, alpha=0.7, perplexity=50.0)),
}


def make(name: str, n: int | None = None, seed: int = 0):
    """Return (X float32 N x D, method parameters) for a named workload,
    optionally with a different N (same generator, same structure)."""
    gen, kw, params = WORKLOADS[name]
    kw = dict(kw)
    if n is not None:
        kw["n"] = n
    kw["seed"] = seed
    return gen(**kw), dict(params)
