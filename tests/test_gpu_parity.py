"""GPU parity of the FUnc-SNE iteration (phase kernels) against the FP64 oracle,
through the C ABI. One iteration from the same state and Philox streams:
neighbour index sets bit-exact (FP32/FP64 near-ties at the list boundary
are reported, never silently accepted beyond a handful), forces within
1e-4 relative per point, bandwidths within the bisection tolerance."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2509_07681_gb300 import funcsne as F
from paper_2509_07681_gb300 import synth
from paper_2509_07681_gb300.quality import recall, rnx_auc

from gpu_util import (align_to, check_after_refinement, check_calibration, compare_sets, fp32_band, lib,
                      oracle_from_state, rel_err_rows)

pytestmark = pytest.mark.gpu

@pytest.fixture(scope="module", autouse=True)
def _lib():
    lib()


CASES = {
    # blobs workload: N=2000, D=50, d=2, k_hd=32, k_ld=16, n_neg=16, alpha=1
    "blobs-2k": (lambda: synth.blobs(n=2000, dim=50),
                 dict(d=2, k_hd=32, k_ld=16, n_neg=16, alpha=1.0, perplexity=30.0)),
    # ragged: N not a multiple of the warps per block, D not a multiple of 4,
    # d padded 3 -> 4, n_neg > 32, heavy tails
    "ragged": (lambda: synth.blobs(n=997, dim=7, n_clusters=4, seed=3),
               dict(d=3, k_hd=20, k_ld=10, n_neg=40, alpha=0.5, perplexity=12.0)),
    # two registers per lane for the HD list (k_hd = 64), d = 32, light tails
    "k64-d32": (lambda: synth.lowrank(n=1500, dim=33, latent=8, n_comp=10, seed=4),
                dict(d=32, k_hd=64, k_ld=32, n_neg=32, alpha=0.7, perplexity=50.0)),
    # the 1M-point workload's shape at small N: d=16, k 32/32, n_neg 32
    "spectrum-shape": (lambda: synth.spectrum(n=3000, dim=50, n_clusters=12, seed=5),
                       dict(d=16, k_hd=32, k_ld=32, n_neg=32, alpha=1.0, perplexity=30.0)),
    # pixel rows: D=784 (multiples of 1/255, about half zeros), d=2
    "pixels-shape": (lambda: synth.pixels(n=2500, dim=784, seed=10),
                     dict(d=2, k_hd=32, k_ld=16, n_neg=16, alpha=1.0, perplexity=30.0)),
    # dynamic-dataset shape: D=128, d=8
    "swissroll-shape": (lambda: synth.swissroll(n=2500, dim=128, seed=6),
                        dict(d=8, k_hd=32, k_ld=16, n_neg=16, alpha=100.0, perplexity=30.0)),
    # smallest N for k_hd = 32 (every other point is listed), D = 1, d = 1,
    # a single negative sample
    "n33-D1-d1": (lambda: synth.blobs(n=33, dim=1, n_clusters=2, seed=7),
                  dict(d=1, k_hd=32, k_ld=16, n_neg=1, alpha=1.0, perplexity=20.0)),
    # more LD than HD neighbours, tiny n_neg
    "kld-gt-khd": (lambda: synth.blobs(n=400, dim=5, n_clusters=3, seed=8),
                   dict(d=2, k_hd=8, k_ld=24, n_neg=3, alpha=1.0, perplexity=5.0)),
    # perplexity above k_hd: no bandwidth reaches it, P is uniform
    "uniform-P": (lambda: synth.blobs(n=500, dim=9, n_clusters=3, seed=9),
                  dict(d=2, k_hd=10, k_ld=8, n_neg=8, alpha=1.0, perplexity=10.5)),
}


def _make(X, params, seed=0, **opts):
    m = F.FuncSNE(X, params["d"], params["k_hd"], params["k_ld"], params["n_neg"], params["alpha"],
                  params["perplexity"], seed=seed)
    for k, v in opts.items():
        m.set_option(k, v)
    return m


def test_initial_state_matches_oracle():
    X = synth.blobs(n=2000, dim=50)
    p = CASES["blobs-2k"][1]
    with _make(X, p) as m:
        st = m.export_state()
    o = O.OracleState(X, p["d"], p["k_hd"], p["k_ld"], p["n_neg"], p["alpha"], p["perplexity"], seed=0)
    # initial lists are integer draws from Philox: identical element by element
    np.testing.assert_array_equal(np.sort(st["hd_idx"], 1), np.sort(o.hd_idx, 1))
    np.testing.assert_array_equal(st["ld_idx"], o.ld_idx)
    assert np.max(rel_err_rows(st["Y"].astype(np.float64), o.Y)) < 1e-5
    np.testing.assert_allclose(st["beta"], o.beta, rtol=2e-3)
    assert abs(st["Zhat"] - o.Zhat) <= 1e-5 * o.Zhat
    assert st["E"] == 1.0 and st["t"] == 0


@pytest.mark.parametrize("case", list(CASES))
def test_one_iteration_matches_oracle(case):
    """One iteration from the same state. Neighbour sets: the oracle's own
    step, bit-exact up to counted FP32/FP64 near-ties. Everything after the
    refinement is then checked on every row, unconditionally: the oracle is
    given the GPU's lists of t+1 and calibrates every changed row itself
    (Eq. 1, warm start), and its attraction, repulsion, Z_t, Zhat, V and Y
    are compared with the GPU's; the GPU's beta and P against the oracle's
    within the bounds the two stopping rules imply."""
    gen, p = CASES[case]
    X = gen()
    N, D = X.shape
    m = _make(X, p, hd_mode=1)
    m.step(4)
    m.sync()
    st = m.export_state()
    o = oracle_from_state(X, st, p, hd_mode=1)
    att, rep = m.debug_step()
    st1 = m.export_state()
    s1 = m.stats()
    lr = m.get_option("lr")
    m.close()
    out = o.step()
    X64 = X.astype(np.float64)
    band = fp32_band(D)
    bad, amb = compare_sets(st1["hd_idx"], o.hd_idx, range(N), X64, band)
    assert bad == 0, f"{bad} HD sets differ beyond FP32 near-ties"
    assert amb <= max(2, N // 500)
    Y0 = st["Y"].astype(np.float64)
    badl, ambl = compare_sets(st1["ld_idx"], o.ld_idx, range(N), Y0, band)
    assert badl == 0, f"{badl} LD sets differ beyond FP32 near-ties"
    assert ambl <= max(2, N // 500)
    # LD lists come out ordered by (d2, idx) at Y_t on both sides: where the
    # sets agree, the order agrees too unless two neighbours are FP32 near-ties
    for i in range(N):
        a, b = st1["ld_idx"][i], o.ld_idx[i]
        if set(a.tolist()) != set(b.tolist()) or np.array_equal(a, b):
            continue
        d2 = ((Y0[b] - Y0[i]) ** 2).sum(1)
        ties = np.diff(d2) <= band * np.maximum(d2[1:], 1e-300)
        wrong = np.nonzero(a != b)[0]
        assert all(ties[max(w - 1, 0):w + 1].any() for w in wrong), (i, a, b)
    assert s1["last_coin"] == 1 and out["coin"]

    # the flag count differs from the oracle's own step only on near-tie rows
    assert abs(s1["last_n_new"] - out["n_new"]) <= amb
    check_after_refinement(X, st, st1, att, rep, s1, p, lr, label=case)


@pytest.mark.parametrize("dim,k_hd", [(50, 32), (200, 32), (200, 64)])
@pytest.mark.parametrize("precision", [F.BF16, F.FP8])
def test_reduced_precision_sets_equal_fp32(precision, dim, k_hd):
    """BF16 / FP8 rows with the exact FP32 re-rank give the FP32 path's sets
    and distances bit for bit (D = 200: the reduced-precision rows and the
    FP32 rows are read by different numbers of lanes per row; k_hd = 64: the
    two-register list, whose BF16 pass batches its loads)."""
    X = synth.spectrum(n=4000, dim=dim, n_clusters=12, seed=7)
    p = dict(CASES["spectrum-shape"][1], k_hd=k_hd)
    m = _make(X, p, hd_mode=1)
    m.step(3)
    st = m.export_state()
    m.step(1)
    ref = m.export_state()
    m.import_state(st)
    m.set_option("precision", precision)
    m.step(1)
    got = m.export_state()
    s = m.stats()
    np.testing.assert_array_equal(got["hd_idx"], ref["hd_idx"])
    np.testing.assert_array_equal(got["hd_d2"], ref["hd_d2"])
    np.testing.assert_array_equal(got["ld_idx"], ref["ld_idx"])
    assert s["cand_scored"] > 0 and s["cand_reranked"] <= s["cand_scored"]
    m.close()


@pytest.mark.parametrize("precision", [F.BF16, F.FP8])
def test_reduced_precision_bands_hold_on_hard_rows(precision):
    """Rows that stress the stored rounding-error bound: a large common
    offset (every candidate falls inside its band and is re-ranked), one
    huge coordinate per row (the FP8 scale pushes the other values towards
    subnormal codes), values halfway between BF16 neighbours (rounding ties)
    and identical all-zero rows (distance-0 ties broken by index). The sets
    and distances still equal the FP32 path's bit for bit."""
    rng = np.random.default_rng(71)
    n, D = 3000, 40
    X = synth.blobs(n=n, dim=D, n_clusters=6, seed=71)
    X[: n // 3] += 1000.0
    X[n // 3: 2 * n // 3, 0] = (1e4 * (1.0 + rng.random(n // 3))).astype(np.float32)
    ties = 1.0 + (2 * rng.integers(0, 64, (n // 6, D)) + 1) * 2.0 ** -8
    X[2 * n // 3: 2 * n // 3 + n // 6] = ties.astype(np.float32)
    X[-12:] = 0.0
    p = dict(d=2, k_hd=16, k_ld=8, n_neg=8, alpha=1.0, perplexity=8.0)
    m = _make(X, p, hd_mode=1)
    m.step(3)
    st = m.export_state()
    m.step(1)
    ref = m.export_state()
    m.import_state(st)
    m.set_option("precision", precision)
    m.step(1)
    got = m.export_state()
    s = m.stats()
    np.testing.assert_array_equal(got["hd_idx"], ref["hd_idx"])
    np.testing.assert_array_equal(got["hd_d2"], ref["hd_d2"])
    np.testing.assert_array_equal(got["ld_idx"], ref["ld_idx"])
    # the offset block alone sends a third of the candidates to the re-rank
    assert s["cand_reranked"] >= 0.25 * s["cand_scored"]
    m.close()


def test_integer_ties_are_broken_by_index():
    """Small-integer data: FP32 and FP64 distances are exact, ties are exact,
    and both sides must order them by index: bit-exact lists, no ambiguity."""
    X = synth.integer_grid(1200, 6, high=3, seed=8)
    p = dict(d=2, k_hd=24, k_ld=12, n_neg=16, alpha=1.0, perplexity=10.0)
    m = _make(X, p, hd_mode=1)
    m.step(2)
    st = m.export_state()
    o = oracle_from_state(X, st, p, hd_mode=1)
    m.debug_step()
    st1 = m.export_state()
    o.step()
    np.testing.assert_array_equal(st1["hd_idx"], o.hd_idx)
    np.testing.assert_array_equal(st1["hd_d2"], o.hd_d2.astype(np.float32))
    m.close()


def test_no_hd_refinement_keeps_lists_and_p():
    X = synth.blobs(n=1000, dim=20, seed=9)
    p = dict(d=2, k_hd=16, k_ld=8, n_neg=8, alpha=1.0, perplexity=8.0)
    m = _make(X, p, hd_mode=2)
    st = m.export_state()
    m.step(3)
    st1 = m.export_state()
    np.testing.assert_array_equal(st1["hd_idx"], st["hd_idx"])
    np.testing.assert_array_equal(st1["P"], st["P"])
    assert st1["E"] == st["E"] and st1["t"] == 3
    m.close()


def test_adaptive_coin_and_smoothing_match_oracle():
    X = synth.blobs(n=1500, dim=30, seed=10)
    p = dict(d=2, k_hd=16, k_ld=8, n_neg=8, alpha=1.0, perplexity=8.0)
    m = _make(X, p)
    m.step(40)
    for _ in range(5):
        st = m.export_state()
        o = oracle_from_state(X, st, p)
        m.step(1)
        s = m.stats()
        out = o.step()
        assert s["last_coin"] == int(out["coin"])
        if s["last_n_new"] == out["n_new"]:
            assert m.export_state()["E"] == o.E
    m.close()


def test_coin_floor_and_smoothing_options_match_oracle():
    """Adaptive refinement with a non-default floor and smoothing rates: the
    coin, E (integer counts, FP64 with explicit rounding) and Zhat follow the
    oracle from the same state."""
    X = synth.blobs(n=1500, dim=30, seed=12)
    p = dict(d=2, k_hd=16, k_ld=8, n_neg=8, alpha=1.0, perplexity=8.0)
    opts = dict(coin_floor=0.3, gamma_e=0.25, gamma_z=0.5)
    m = _make(X, p, **opts)
    for k, v in opts.items():
        assert m.get_option(k) == v
    m.step(30)
    coins = []
    for _ in range(6):
        st = m.export_state()
        o = oracle_from_state(X, st, p, **opts)
        m.step(1)
        s = m.stats()
        out = o.step()
        assert s["last_coin"] == int(out["coin"])
        coins.append(out["coin"])
        st1 = m.export_state()
        if s["last_n_new"] == out["n_new"]:
            assert st1["E"] == o.E
        assert abs(st1["Zhat"] - o.Zhat) <= 1e-4 * o.Zhat
    for k, v in (("coin_floor", 1.5), ("gamma_e", 0.0), ("gamma_z", -0.1)):
        with pytest.raises(F.FuncSNEError):
            m.set_option(k, v)
    m.close()


def test_exact_knn_matches_bruteforce():
    X = synth.spectrum(n=5000, dim=50, n_clusters=8, seed=11)
    with _make(X, CASES["spectrum-shape"][1]) as m:
        q = np.arange(0, 5000, 37)
        idx, d2 = m.exact_knn(q, 40)
    ref, rd = O.query_knn(X, q, 40)
    bad, amb = compare_sets(idx, ref, range(len(q)), X.astype(np.float64), fp32_band(50))
    assert bad == 0 and amb <= 1


def test_whole_run_blobs_recall_and_structure():
    """500 iterations of the blobs workload: the HD lists converge to the exact
    KNN and the embedding keeps the clusters (statistics, not bit parity)."""
    X = synth.blobs(n=2000, dim=50)
    p = CASES["blobs-2k"][1]
    with _make(X, p) as m:
        m.step(500)
        m.sync()
        hd = m.knn(F.SPACE_HD, with_d2=False)
        Y = m.embedding()
        s = m.stats()
    exact, _ = O.bruteforce_knn(X, 128)
    assert recall(hd, exact[:, :32]) > 0.99
    ld, _ = O.bruteforce_knn(Y, 128)
    from paper_2509_07681_gb300.quality import rnx_curve
    r = rnx_curve(ld, exact, len(X))
    assert r[99] > 0.5
    assert math.isfinite(s["Zhat"]) and s["error_word"] == 0


@pytest.mark.parametrize("rounds", [64, 0, 5, 200])
def test_insertion_matches_oracle(rounds):
    """funcsne_insert (mean placement) against the oracle from the same state:
    the new points' HD/LD lists, positions and bandwidths, the scalars, and
    the next iteration over the grown state; with the default 64, no, 5 and
    200 neighbour-of-neighbour rounds."""
    X = synth.blobs(n=2600, dim=30, n_clusters=6, seed=15)
    p = dict(d=2, k_hd=16, k_ld=8, n_neg=8, alpha=1.0, perplexity=8.0)
    m = _make(X[:2000], p, hd_mode=1)
    m.set_option("insert_rounds", rounds)
    m.step(30)
    st = m.export_state()
    o = oracle_from_state(X[:2000], st, p, hd_mode=1)
    first = m.insert(X[2000:])
    o.insert(X[2000:], rounds=rounds)
    assert first == 2000 and m.N == 2600
    st1 = m.export_state()
    new = range(2000, 2600)
    X64 = X.astype(np.float64)
    bad, amb = compare_sets(st1["hd_idx"], o.hd_idx, new, X64, fp32_band(30))
    assert bad == 0 and amb <= 2
    # rows whose sets agree (all but the counted near-ties): position, cold
    # calibration (Eq. 1) and LD seeding against the oracle
    same = [i for i in new if set(st1["hd_idx"][i].tolist()) == set(o.hd_idx[i].tolist())]
    assert len(same) >= len(new) - amb
    ys = np.array(same)
    assert np.max(rel_err_rows(st1["Y"][ys].astype(np.float64), o.Y[ys])) < 1e-5
    check_calibration(X64, ys, st1["hd_idx"], st1["beta"], st1["P"], o.beta[ys],
                      align_to(st1["hd_idx"][ys], o.hd_idx[ys], o.P[ys]), p["perplexity"], 30)
    for i in same:
        assert set(st1["ld_idx"][i].tolist()) == set(o.ld_idx[i].tolist())
    assert abs(st1["Zhat"] - o.Zhat) <= 1e-5 * o.Zhat and st1["E"] == o.E
    # old points are untouched
    np.testing.assert_array_equal(st1["hd_idx"][:2000], st["hd_idx"])
    np.testing.assert_array_equal(st1["Y"][:2000], st["Y"])
    # one more iteration over the grown state, checked on every row
    o2 = oracle_from_state(X, st1, p, hd_mode=1)
    att, rep = m.debug_step()
    st2 = m.export_state()
    s2 = m.stats()
    lr = m.get_option("lr")
    m.close()
    o2.step()
    bad, amb = compare_sets(st2["hd_idx"], o2.hd_idx, range(2600), X64, fp32_band(30))
    assert bad == 0 and amb <= 3
    check_after_refinement(X, st1, st2, att, rep, s2, p, lr, label=f"insert {rounds} rounds", hd_mode=1)


def test_insertion_grows_repeatedly_and_keeps_stepping():
    X = synth.swissroll(n=3000, dim=16, n_clusters=8, seed=16)
    p = dict(d=8, k_hd=32, k_ld=16, n_neg=16, alpha=1.0, perplexity=30.0)
    m = _make(X[:1000], p)
    m.step(20)
    for b in range(4):
        lo = 1000 + 500 * b
        assert m.insert(X[lo:lo + 500]) == lo
        m.step(10)
    m.sync()
    assert m.N == 3000 and m.stats()["N"] == 3000
    hd = m.knn(F.SPACE_HD, with_d2=False)
    assert hd.min() >= 0 and hd.max() < 3000
    assert np.isfinite(m.embedding()).all()
    m.close()


@pytest.mark.parametrize("hd_mode", [2, 0])
def test_insertion_window_matches_oracle(hd_mode):
    """Option fresh_iters: after an insertion, the new points refine their HD
    lists in every iteration of the window, also when the coin does not
    fire (hd_mode 2: never; 0: the adaptive coin). Each iteration from the
    same state as the oracle: HD and LD sets, the window's bounds, and
    everything after the refinement on every row; the old points' HD lists
    change only in iterations whose coin fired."""
    X = synth.blobs(n=2600, dim=24, n_clusters=6, seed=17)
    p = dict(d=2, k_hd=16, k_ld=8, n_neg=8, alpha=1.0, perplexity=8.0)
    m = _make(X[:2000], p, hd_mode=1)
    m.step(20)
    m.set_option("hd_mode", hd_mode)
    m.set_option("fresh_iters", 5)
    m.set_option("insert_rounds", 2)
    m.step(10)
    m.insert(X[2000:])
    st = m.export_state()
    assert st["fresh_lo"] == 2000 and st["fresh_until"] == st["t"] + 5
    lr = m.get_option("lr")
    X64 = X.astype(np.float64)
    for it in range(6):
        o = oracle_from_state(X, st, p, hd_mode=hd_mode, fresh_iters=5)
        att, rep = m.debug_step()
        st1 = m.export_state()
        s1 = m.stats()
        out = o.step()
        assert s1["last_coin"] == int(out["coin"])
        bad, amb = compare_sets(st1["hd_idx"], o.hd_idx, range(2600), X64, fp32_band(24))
        assert bad == 0 and amb <= 3
        badl, _ = compare_sets(st1["ld_idx"], o.ld_idx, range(2600), st["Y"].astype(np.float64), fp32_band(24))
        assert badl == 0
        if not out["coin"]:
            np.testing.assert_array_equal(st1["hd_idx"][:2000], st["hd_idx"][:2000])
            if it < 5:
                assert np.any(st1["hd_idx"][2000:] != st["hd_idx"][2000:])
            else:  # the window has closed
                np.testing.assert_array_equal(st1["hd_idx"], st["hd_idx"])
        check_after_refinement(X, st, st1, att, rep, s1, p, lr, label=f"window it {it}", coin=out["coin"],
                               hd_mode=hd_mode, fresh_iters=5)
        st = st1
    m.close()


def _host_copy(X, fmt):
    """The reduced-precision copy of each row as the library makes it:
    BF16 round to nearest even; FP8-E4M3 codes of x / s (FP32 division,
    round to nearest even, saturating at 448) times s = max|x| / 448 in FP32
    (s = 1 for a zero row)."""
    torch = pytest.importorskip("torch")
    X32 = X.astype(np.float32)
    if fmt == "bf16":
        return O.bf16(X32.astype(np.float64))
    m = np.abs(X32).max(1, keepdims=True)
    s = np.where(m > 0, m / np.float32(448.0), np.float32(1.0)).astype(np.float32)
    q = torch.from_numpy((X32 / s).astype(np.float32)).clamp(-448, 448).to(torch.float8_e4m3fn)
    return (q.to(torch.float32).numpy() * s).astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("fmt", ["bf16", "fp8"])
def test_row_error_bounds_cover_the_quantisation_error(fmt):
    """The bound E_i >= ||x_i - x~_i|| stored with each reduced-precision row
    (it widens the distance band, so the exact re-rank sees every candidate
    that can enter): never below the exact error norm of the row's copy,
    and within 1e-4 of it. Rows of spread scales, offsets, tiny entries and
    a zero row."""
    rng = np.random.default_rng(81)
    N, D = 1200, 50
    X = rng.standard_normal((N, D)) * np.exp(rng.uniform(-12, 12, (N, 1))) + rng.uniform(-5, 5, (N, 1))
    X[:, ::9] *= 1e-3
    X[7] = 0.0
    X = X.astype(np.float32)
    p = CASES["blobs-2k"][1]
    with F.FuncSNE(X, p["d"], p["k_hd"], p["k_ld"], p["n_neg"], p["alpha"], p["perplexity"], seed=0,
                   precision=F.BF16 if fmt == "bf16" else F.FP8) as m:
        E = m.row_bounds().astype(np.float64)
    exact = np.sqrt(((X.astype(np.float64) - _host_copy(X, fmt)) ** 2).sum(1))
    assert np.all(E >= exact)
    assert np.all(E <= exact * (1 + 1e-4) + 1e-38)
    assert E[7] == 0.0
