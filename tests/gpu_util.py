"""Helpers shared by the GPU parity tests: build/load the library, run the
oracle from a GPU-exported state, and compare neighbour sets allowing only
FP32-vs-FP64 near-ties at the list boundary."""
from __future__ import annotations

import numpy as np

import oracle as O
from paper_2509_07681_gb300 import funcsne as F
from paper_2509_07681_gb300.build import build

# FP32 squared distances carry a relative error below (D + 4) 2^-24; two
# candidates whose FP64 distances differ by less than this band may be
# ordered differently by the two sides (the oracle calls them ambiguous).
def fp32_band(D: int) -> float:
    return 4.0 * (D + 4) * 2.0 ** -24


def lib():
    build()
    return F.load()


def oracle_from_state(X, st, params, **opts):
    o = O.OracleState(X, params["d"], params["k_hd"], params["k_ld"], params["n_neg"], params["alpha"],
                      params["perplexity"], seed=params.get("seed", 0), init=False, **opts)
    o.load(Y=st["Y"], V=st["V"], hd_idx=st["hd_idx"], ld_idx=st["ld_idx"], beta=st["beta"], P=st["P"],
           Zhat=st["Zhat"], E=st["E"], t=st["t"])
    return o


def compare_sets(gpu_idx, ref_idx, points, ref_rows, band):
    """gpu_idx / ref_idx: N x k lists. ref_rows: FP64 coordinates defining the
    distances. Returns (n_exact_mismatch, n_ambiguous). A row differs
    'ambiguously' when every element of the symmetric difference lies within
    the relative FP32 band of the reference list's k-th distance."""
    bad = 0
    amb = 0
    for i in points:
        a = set(gpu_idx[i].tolist())
        b = set(ref_idx[i].tolist())
        if a == b:
            continue
        diff = np.array(sorted(a ^ b))
        d_ref = ((ref_rows[ref_idx[i]] - ref_rows[i]) ** 2).sum(1)
        kth = d_ref.max()
        dd = ((ref_rows[diff] - ref_rows[i]) ** 2).sum(1)
        if np.all(np.abs(dd - kth) <= band * max(kth, 1e-300)):
            amb += 1
        else:
            bad += 1
    return bad, amb


def rel_err_rows(a, b):
    """Per-row ||a - b|| / ||b||, with rows of zero norm compared absolutely."""
    num = np.linalg.norm(a - b, axis=1)
    den = np.linalg.norm(b, axis=1)
    floor = 1e-6 * max(den.max(), 1e-300)
    return num / np.maximum(den, floor)
