"""Helpers shared by the GPU parity tests: build/load the library, run the
oracle from a GPU-exported state, compare neighbour sets allowing only
FP32-vs-FP64 near-ties at the list boundary, and check the GPU's bandwidth
calibration (Eq. 1) against the oracle's with tolerances derived from the
two sides' stopping rules."""
from __future__ import annotations

import math

import numpy as np

import oracle as O
from paper_2509_07681_gb300 import funcsne as F
from paper_2509_07681_gb300.build import build

U32 = 2.0 ** -24          # unit roundoff of binary32 (round to nearest)
GPU_BISECT_TOL = 1e-5     # the kernels stop when |H - ln perp| < 1e-5, evaluated in FP32


# FP32 squared distances carry a relative error below (D + 4) 2^-24; two
# candidates whose FP64 distances differ by less than this band may be
# ordered differently by the two sides (the oracle calls them ambiguous).
def fp32_band(D: int) -> float:
    return 4.0 * (D + 4) * 2.0 ** -24


def lib():
    build()
    return F.load()


def oracle_from_state(X, st, params, d2=True, **opts):
    o = O.OracleState(X, params["d"], params["k_hd"], params["k_ld"], params["n_neg"], params["alpha"],
                      params["perplexity"], seed=params.get("seed", 0), init=False, **opts)
    o.load(Y=st["Y"], V=st["V"], hd_idx=st["hd_idx"], ld_idx=st["ld_idx"], beta=st["beta"], P=st["P"],
           Zhat=st["Zhat"], E=st["E"], t=st["t"], d2=d2, fresh_lo=st.get("fresh_lo"),
           fresh_until=st.get("fresh_until"))
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


def _row_d2(X, i, idx):
    xi = np.asarray(X[i], dtype=np.float64)
    return ((np.asarray(X[idx], dtype=np.float64) - xi) ** 2).sum(1)


def oracle_calibration(X, rows, hd_idx, beta_prev, perplexity):
    """The oracle's bandwidth and P_{.|i} (Eq. 1) of each point in `rows`,
    from its HD list hd_idx[i] (FP64 distances from X) by the oracle's own
    bisection, warm-started at beta_prev[i] as the method does (Section 3).
    Returns (beta (n,), P (n, k))."""
    k = hd_idx.shape[1]
    beta = np.zeros(len(rows))
    P = np.zeros((len(rows), k))
    for a, i in enumerate(rows):
        beta[a], P[a], _ = O.bisect(_row_d2(X, i, hd_idx[i]), perplexity, beta0=float(beta_prev[i]))
    return beta, P


def check_calibration(X, rows, hd_idx, beta_gpu, P_gpu, beta_or, P_or, perplexity, D):
    """Checks the GPU's calibration of the points `rows` against the oracle's
    (beta_or, P_or aligned with `rows`; beta_gpu, P_gpu indexed by point).

    The GPU stops when |H - ln perp| < 1e-5 with H evaluated in FP32 from FP32
    distances; the oracle when it is below 1e-9 in FP64. Hence, per row:
      1. H(beta_gpu) over the FP64 distances is within 1e-5 of ln perp, plus
         the first-order effect of the FP32 distance errors on H
         (dH/dsh_j = -beta^2 p_j (sh_j - mu), sh = d2 - d2_min, mu = E_p[sh])
         and the FP32 evaluation error of ln S + beta U / S;
      2. beta_gpu - beta_or is the entropy error divided by the slope
         |dH/dbeta| = beta Var_p(sh) (the smaller of the slopes at both ends);
      3. each P_{j|i} differs from the oracle's by at most the first-order
         change of Eq. 1 under that beta difference (|dp_j/dbeta| =
         p_j |sh_j - mu|), under the distance errors, and under the FP32
         evaluation of exp2 and the normalisation.
    When ln k <= ln perp, P must be uniform (beta = 0) on both sides.
    Returns the worst ratio of error to bound for (entropy, beta, P)."""
    band = fp32_band(D)
    k = hd_idx.shape[1]
    lp = math.log(perplexity)
    worst = np.zeros(3)
    for a, i in enumerate(rows):
        if math.log(k) <= lp:
            assert beta_gpu[i] == 0.0 and beta_or[a] == 0.0, i
            np.testing.assert_array_equal(P_gpu[i], np.float32(1.0) / np.float32(k))
            continue
        d2 = _row_d2(X, i, hd_idx[i])
        sh = d2 - d2.min()
        dsh = band * (d2 + d2.min())       # bound on the FP32 error of each shifted distance
        b = float(beta_gpu[i])
        H, Pg = O.entropy(d2, b)
        mu = float((Pg * sh).sum())
        var = float((Pg * sh * sh).sum()) - mu * mu
        eps_dist = b * b * float((Pg * np.abs(sh - mu) * dsh).sum())
        # FP32 sums of k exponentials, the ratio U / S and logf (1 ulp)
        eps_arith = 2 * U32 * (k + 8 + 3 * b * mu) * (1 + b * mu) + 4 * U32 * math.log(k)
        tol_h = GPU_BISECT_TOL + eps_dist + eps_arith
        eh = abs(H - lp)
        assert eh <= tol_h, (i, H, lp, tol_h)
        bo = float(beta_or[a])
        _, Po = O.entropy(d2, bo)
        mu_o = float((Po * sh).sum())
        var_o = float((Po * sh * sh).sum()) - mu_o * mu_o
        slope = min(b * var, bo * var_o)
        db = abs(b - bo)
        if slope > 0:
            tol_b = 1.05 * (eh + 1e-9) / slope + 2 * U32 * b
            assert db <= tol_b, (i, b, bo, tol_b)
            worst[1] = max(worst[1], db / tol_b)
        worst[0] = max(worst[0], eh / tol_h)
        tol_p = 1.25 * P_or[a] * (np.abs(sh - mu_o) * db + b * (dsh + float((P_or[a] * dsh).sum()))
                                  + 2 * U32 * (k + 12 + 3 * b * (sh + mu_o))) + 1e-30
        ep = np.abs(P_gpu[i].astype(np.float64) - P_or[a])
        assert np.all(ep <= tol_p), (i, int(np.argmax(ep / tol_p)), float(np.max(ep / tol_p)))
        worst[2] = max(worst[2], float(np.max(ep / tol_p)))
    return worst


def gpu_list_oracle(X, st0, st1, params, rows=None, **opts):
    """The oracle at iteration t holding the GPU's lists of t+1, with the
    oracle's own calibration (warm-started from beta_t) of every point whose
    HD list changed, so its forces are comparable with the GPU's on every
    row. rows: only these points are calibrated (the rows a sampled force
    check reads); None means all.
    Returns (oracle, changed rows, beta_or, P_or)."""
    changed = np.any(st1["hd_idx"] != st0["hd_idx"], axis=1)
    cal = np.nonzero(changed)[0] if rows is None else np.asarray(rows)[changed[np.asarray(rows)]]
    beta_or, P_or = oracle_calibration(X, cal, st1["hd_idx"], st0["beta"], params["perplexity"])
    mix = dict(st0)
    mix["hd_idx"], mix["ld_idx"] = st1["hd_idx"], st1["ld_idx"]
    mix["beta"] = st0["beta"].astype(np.float64)
    mix["P"] = st0["P"].astype(np.float64)
    mix["beta"][cal] = beta_or
    mix["P"][cal] = P_or
    o = oracle_from_state(X, mix, params, d2=rows is None, **opts)
    return o, cal, beta_or, P_or


def attraction_term_norms(Y, hd_idx, P, alpha):
    """Per point, the sum of the norms of the attraction terms that reach it
    (its own list and the lists that hold it). Any FP32 summation order of
    those terms errs by at most about (terms + a few) 2^-24 times this sum,
    so rows whose attraction cancels strongly need an absolute bound."""
    N, k = hd_idx.shape
    Y = Y.astype(np.float64)
    dy = Y[:, None, :] - Y[hd_idx]
    r2 = (dy * dy).sum(-1)
    mag = 4.0 * (P / (2.0 * N)) / (1.0 + r2 / alpha) * np.sqrt(r2)
    s = mag.sum(1)
    np.add.at(s, hd_idx.ravel(), mag.ravel())
    cnt = np.full(N, k, dtype=np.int64)
    np.add.at(cnt, hd_idx.ravel(), 1)
    return s, cnt


def align_to(gpu_idx, ref_idx, ref_vals):
    """ref_vals (rows aligned with ref_idx) reordered to the order of gpu_idx;
    the two lists must hold the same set in each row."""
    out = np.empty(ref_vals.shape, dtype=np.float64)
    for r in range(len(gpu_idx)):
        pos = {int(j): a for a, j in enumerate(ref_idx[r])}
        out[r] = ref_vals[r][[pos[int(j)] for j in gpu_idx[r]]]
    return out


FORCE_RTOL = 1e-4


def check_after_refinement(X, st, st1, att, rep, s1, params, lr, momentum=0.8, gamma_e=0.1, gamma_z=0.1,
                           label="", coin=True, **opts):
    """Everything one GPU iteration computes after its neighbour refinement,
    checked on every row against the oracle run from the GPU's lists of t+1
    (st: exported state t; st1: state t+1; att, rep: the GPU's forces of the
    iteration; s1: its stats; the HD refinement ran):
      * the flag count equals the number of changed HD lists, and E follows
        from it (coin=False: an iteration that refined only the insertion
        window, which leaves E as it was);
      * beta and P of every changed row against the oracle's warm-started
        calibration (check_calibration); unchanged rows keep theirs;
      * attraction and repulsion of every row within 1e-4 relative;
      * Z_t within 1e-5, Zhat_{t+1} = (1 - gamma_z) Zhat_t + gamma_z Z_t;
      * V_{t+1} = momentum V_t - lr (A - R) within the force errors and FP32
        rounding, and Y_{t+1} = Y_t + V_{t+1} rounded once.
    Returns a dict of the measured worst errors."""
    N, D = X.shape
    X64 = np.asarray(X, dtype=np.float64)
    o1, cal, beta_or, P_or = gpu_list_oracle(X, st, st1, params, **opts)
    changed = np.zeros(N, bool)
    changed[cal] = True
    assert s1["last_n_new"] == len(cal)
    if coin:
        assert st1["E"] == (1.0 - gamma_e) * st["E"] + gamma_e * (len(cal) / N)  # same FP64 expression
    else:
        assert st1["E"] == st["E"]
    worst = check_calibration(X64, cal, st1["hd_idx"], st1["beta"], st1["P"], beta_or, P_or,
                              params["perplexity"], D)
    np.testing.assert_array_equal(st1["P"][~changed], st["P"][~changed])
    np.testing.assert_array_equal(st1["beta"][~changed], st["beta"][~changed])
    A, R, zt, _ = o1.forces(zhat=st["Zhat"], t=st["t"])
    ea = rel_err_rows(att.astype(np.float64), A)
    er = rel_err_rows(rep.astype(np.float64), R)
    Y0 = st["Y"].astype(np.float64)
    S, cnt = attraction_term_norms(Y0, st1["hd_idx"], o1.P, params["alpha"])
    cond = S / np.maximum(np.linalg.norm(A, axis=1), 1e-300)
    w = int(np.argmax(ea))
    res = dict(calibrated=len(cal), entropy=worst[0], beta=worst[1], P=worst[2], att_max=float(ea.max()),
               att_q999=float(np.quantile(ea, 0.999)), att_cancel=float(cond[w]), att_terms=int(cnt[w]),
               rep_max=float(er.max()))
    print(f"{label}: calibrated rows {len(cal)}, worst error/bound entropy {worst[0]:.3f} beta {worst[1]:.3f} "
          f"P {worst[2]:.3f}; attraction rel err max {ea.max():.2e} (row {w}, cancellation {cond[w]:.1f}, "
          f"terms {cnt[w]}) q99.9 {res['att_q999']:.2e}; repulsion max {er.max():.2e}")
    assert ea.max() < FORCE_RTOL, (ea.max(), cond[w])
    assert er.max() < FORCE_RTOL, er.max()
    assert abs(s1["last_Z"] - zt) <= 1e-5 * zt
    assert abs(st1["Zhat"] - ((1.0 - gamma_z) * st["Zhat"] + gamma_z * zt)) <= 1e-5 * st1["Zhat"]
    V1 = momentum * st["V"].astype(np.float64) - lr * (A - R)
    dv = np.linalg.norm(st1["V"] - V1, axis=1)
    tol_v = lr * (np.linalg.norm(att - A, axis=1) + np.linalg.norm(rep - R, axis=1)) + \
        8 * U32 * (momentum * np.linalg.norm(st["V"], axis=1) +
                   lr * (np.linalg.norm(A, axis=1) + np.linalg.norm(R, axis=1)))
    assert np.all(dv <= 1.01 * tol_v + 1e-30)
    Y1 = Y0 + st1["V"].astype(np.float64)
    assert np.all(np.abs(st1["Y"] - Y1) <= U32 * np.abs(Y1) + 1e-38)
    return res
