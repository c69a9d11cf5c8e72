"""Pins of the FP64 CPU oracle against facts that do not come from the oracle:
published known-answer vectors, closed forms, brute force, finite
differences, conservation laws and limiting cases of the paper's equations.
"""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2509_07681_gb300 import synth
from paper_2509_07681_gb300.quality import recall, rnx_auc, rnx_curve

HERE = os.path.dirname(os.path.abspath(__file__))


# ---------------------------------------------------------------- Philox
def _kat_rows():
    rows = []
    with open(os.path.join(HERE, "golden", "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            w = [int(x, 16) for x in line.split()]
            rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,out", _kat_rows())
def test_philox_known_answers(ctr, key, out):
    assert O.philox(ctr, key).tolist() == out


# ---------------------------------------------------------------- bisection (Eq. 1)
def test_bisection_hits_target_entropy():
    g = np.random.default_rng(1)
    for _ in range(50):
        k = int(g.integers(8, 65))
        d2 = np.sort(g.exponential(3.0, size=k) + g.uniform(0, 5))
        perp = float(g.uniform(2.0, k - 1.5))
        beta, P, it = O.bisect(d2, perp)
        # entropy evaluated independently of the oracle's routine
        p = np.exp(-beta * (d2 - d2.min()))
        p /= p.sum()
        H = -(p * np.log(p)).sum()
        assert abs(H - math.log(perp)) < 1e-6
        assert abs(P.sum() - 1.0) < 1e-12
        np.testing.assert_allclose(P, p, rtol=1e-9, atol=1e-15)


def test_bisection_two_point_closed_form():
    # two neighbours at distances 0 and c: p = 1/(1+exp(-beta c)), binary entropy
    from scipy.optimize import brentq
    c = 2.5
    for perp in [1.2, 1.5, 1.9]:
        beta, P, _ = O.bisect([0.0, c], perp)

        def h(b):
            e = math.exp(-b * c)
            p1, p2 = 1.0 / (1.0 + e), e / (1.0 + e)
            return -(p1 * math.log(p1) + p2 * math.log(p2)) - math.log(perp)
        ref = brentq(h, 1e-12, 20.0, xtol=1e-14)
        assert abs(beta - ref) < 1e-6 * max(1.0, ref)


def test_bisection_degenerate_cases():
    # equal distances: every beta gives H = ln k; a reachable target is impossible
    # when perplexity >= k, which must give the uniform distribution.
    beta, P, _ = O.bisect(np.full(16, 3.0), 30.0)
    assert beta == 0.0 and np.allclose(P, 1 / 16)
    beta, P, _ = O.bisect(np.linspace(0, 1, 16), 16.0)
    assert beta == 0.0 and np.allclose(P, 1 / 16)
    h, p = O.entropy(np.full(8, 1.0), 5.0)
    assert abs(h - math.log(8)) < 1e-12


def test_entropy_monotone_in_beta():
    d2 = np.sort(np.random.default_rng(2).exponential(1.0, 32))
    hs = [O.entropy(d2, b)[0] for b in np.geomspace(1e-3, 1e3, 40)]
    assert all(a >= b - 1e-12 for a, b in zip(hs, hs[1:]))
    assert abs(hs[0] - math.log(32)) < 1e-2


def test_warm_start_agrees_with_cold_start():
    d2 = np.sort(np.random.default_rng(3).exponential(2.0, 32))
    b0, P0, _ = O.bisect(d2, 10.0)
    b1, P1, _ = O.bisect(d2, 10.0, beta0=b0 * 3.7)
    assert abs(b1 - b0) < 1e-6 * b0
    np.testing.assert_allclose(P0, P1, rtol=1e-6)


# ---------------------------------------------------------------- top-k merge
def _lex_knn(X, i, k):
    d2 = ((X - X[i]) ** 2).sum(1)
    d2[i] = np.inf
    order = np.lexsort((np.arange(len(X)), d2))
    return order[:k], d2[order[:k]]


@pytest.mark.parametrize("gen", ["gauss", "integer"])
def test_merge_with_all_candidates_is_exact_knn(gen):
    rng = np.random.default_rng(4)
    N, D, k = 200, 7, 8
    X = rng.standard_normal((N, D)) if gen == "gauss" else synth.integer_grid(N, D, high=3, seed=4)
    X = X.astype(np.float64)
    for i in range(0, N, 13):
        old = rng.choice(np.delete(np.arange(N), i), size=k, replace=False).astype(np.int32)
        old_d2 = ((X[old] - X[i]) ** 2).sum(1)
        o = np.lexsort((old, old_d2))
        old, old_d2 = old[o], old_d2[o]
        cand = np.arange(N)
        cand_d2 = ((X - X[i]) ** 2).sum(1)
        ni, nd, ch = O.topk_merge(i, old, old_d2, cand, cand_d2)
        ref_i, ref_d = _lex_knn(X, i, k)
        assert ni.tolist() == ref_i.tolist()
        np.testing.assert_array_equal(nd, ref_d)
        assert ch == (set(ref_i.tolist()) != set(old.tolist()))


def test_merge_drops_self_duplicates_and_keeps_order_when_unchanged():
    old = np.array([5, 3, 9], dtype=np.int32)
    od = np.array([1.0, 2.0, 3.0])
    # candidates: self (0), a duplicate of an old entry, a repeated candidate, and far ones
    ni, nd, ch = O.topk_merge(0, old, od, [0, 3, 7, 7, 8], [0.0, 0.5, 9.0, 9.0, 8.0])
    assert ni.tolist() == [5, 3, 9] and not ch
    ni, nd, ch = O.topk_merge(0, old, od, [7, 7, 2], [1.5, 1.5, 2.0])
    # tie at d2=2.0 between old 3 and candidate 2: smaller index first
    assert ni.tolist() == [5, 7, 2] and ch


# ---------------------------------------------------------------- candidates
def _state(N=300, D=10, d=2, kh=16, kl=8, nneg=8, alpha=1.0, perp=8.0, seed=5, **kw):
    X = synth.blobs(n=N, dim=D, n_clusters=5, seed=seed)
    return O.OracleState(X, d, kh, kl, nneg, alpha, perp, seed=seed, **kw)


def test_ld_merge_reorders_every_time():
    # hand example: 7 enters, 9 (a listed point) and 4 (too far) do not; the
    # list comes out ordered by (d2, idx)
    ni, nd, ch = O.ld_merge(0, [5, 9, 2], [1.0, 3.0, 2.0], [7, 9, 4], [0.5, 9.9, 2.5])
    assert ni.tolist() == [7, 5, 2] and nd.tolist() == [0.5, 1.0, 2.0] and ch
    # nothing enters: the same set, re-ordered under the new distances
    ni, nd, ch = O.ld_merge(0, [3, 1, 2], [0.3, 0.1, 0.2], [4, 5], [0.9, 0.8])
    assert ni.tolist() == [1, 2, 3] and not ch
    # random cases against the plain definition
    rng = np.random.default_rng(12)
    for _ in range(300):
        k = int(rng.integers(1, 12))
        pool = rng.permutation(40)[: k + 12]
        old = pool[:k]
        cand = rng.choice(np.concatenate([pool, [0]]), size=int(rng.integers(1, 20)))
        d = {int(j): float(rng.integers(0, 6)) + 0.01 * j for j in np.concatenate([pool, [0]])}
        od = np.array([d[int(j)] for j in old])
        cd = np.array([d[int(j)] for j in cand])
        ni, nd, ch = O.ld_merge(0, old, od, cand, cd)
        keep = [j for s, j in enumerate(cand.tolist()) if j != 0 and j not in old.tolist() and j not in cand[:s].tolist()]
        union = sorted(set(old.tolist()) | set(keep), key=lambda j: (d[j], j))[:k]
        assert ni.tolist() == union
        assert ch == (set(union) != set(old.tolist()))


def test_initial_lists_distinct_and_valid():
    st = _state()
    for lists, k in [(st.hd_idx, st.k_hd), (st.ld_idx, st.k_ld)]:
        for i in range(st.N):
            row = lists[i]
            assert len(set(row.tolist())) == k
            assert i not in row
            assert row.min() >= 0 and row.max() < st.N
    # HD lists ordered by (d2, idx) with exact distances
    for i in range(0, st.N, 17):
        d2 = ((st.X[st.hd_idx[i]] - st.X[i]) ** 2).sum(1)
        assert np.all(np.diff(d2) >= 0)
    # tiny N: k = N - 1 forces every other point into the list
    st2 = _state(N=17, kh=16, kl=16, perp=4.0)
    for i in range(17):
        assert sorted(st2.hd_idx[i].tolist()) == [j for j in range(17) if j != i]


def test_candidates_come_from_their_sources():
    st = _state()
    for i in range(0, st.N, 7):
        c = st.hd_candidates(i)
        nn_hd = set(st.hd_idx[st.hd_idx[i]].ravel().tolist())
        nn_ld = set(st.ld_idx[st.ld_idx[i]].ravel().tolist())
        assert set(c[:16].tolist()) <= nn_hd
        assert set(c[16:20].tolist()) <= set(st.ld_idx[i].tolist())
        assert set(c[20:24].tolist()) <= nn_ld
        assert all(0 <= x < st.N and x != i for x in c[24:])
        c = st.ld_candidates(i)
        assert set(c[:16].tolist()) <= nn_ld
        assert set(c[16:24].tolist()) <= set(st.hd_idx[i].tolist())
        assert all(0 <= x < st.N and x != i for x in c[24:])


def test_random_candidates_are_uniform():
    # chi-square over many iterations: the random slots cover the other points uniformly
    st = _state(N=40, kh=8, kl=8)
    counts = np.zeros(40)
    for t in range(400):
        st.set(t=t)
        c = st.hd_candidates(3)
        for x in c[24:]:
            counts[x] += 1
    assert counts[3] == 0
    exp = counts.sum() / 39
    chi2 = (((counts - exp) ** 2) / exp)[np.arange(40) != 3].sum()
    assert chi2 < 80  # 38 dof: p ~ 1e-4


# ---------------------------------------------------------------- gradient (Eq. 4-6)
@pytest.mark.parametrize("alpha", [0.5, 1.0, 3.0])
def test_exact_gradient_matches_finite_differences(alpha):
    st = _state(N=40, D=6, d=3, kh=8, kl=6, perp=5.0)
    rng = np.random.default_rng(6)
    Y = rng.standard_normal((40, 3))
    Pd = st.dense_p()
    G = O.exact_grad(Pd, Y, alpha)
    h = 1e-6
    for i in range(0, 40, 9):
        for c in range(3):
            Yp, Ym = Y.copy(), Y.copy()
            Yp[i, c] += h
            Ym[i, c] -= h
            fd = (O.kl_divergence(Pd, Yp, alpha) - O.kl_divergence(Pd, Ym, alpha)) / (2 * h)
            assert abs(fd - G[i, c]) <= 1e-6 * max(1.0, np.abs(G).max())


def test_dense_p_symmetric_and_normalised():
    st = _state()
    Pd = st.dense_p()
    np.testing.assert_allclose(Pd, Pd.T, rtol=0, atol=1e-18)
    assert abs(Pd.sum() - 1.0) < 1e-12
    assert np.all(np.diag(Pd) == 0)


@pytest.mark.parametrize("alpha", [0.5, 1.0, 2.0])
def test_exhaustive_split_equals_exact_gradient(alpha):
    """Eq. 6's three-term split, with the rest summed exhaustively and the exact Z,
    must reproduce Eq. 5 over the sparse symmetrised P."""
    st = _state(N=120, D=8, d=2, kh=12, kl=8, alpha=alpha, perp=6.0, neg_mode=1)
    rng = np.random.default_rng(7)
    st.Y[...] = rng.standard_normal(st.Y.shape)
    z = O.exact_z(st.Y, alpha)
    A, R, zt, _ = st.forces(zhat=z)
    assert abs(zt - z) <= 1e-12 * z
    G = O.exact_grad(st.dense_p(), st.Y, alpha)
    np.testing.assert_allclose(A - R, G, rtol=0, atol=1e-12 * np.abs(G).max())
    # momentum conservation: both parts sum to zero over points
    assert np.abs(A.sum(0)).max() < 1e-12 * np.abs(A).max() * st.N
    assert np.abs(G.sum(0)).max() < 1e-12 * np.abs(G).max() * st.N


def test_alpha_one_is_tsne_gradient():
    """alpha = 1 reduces Eq. 5 to the t-SNE gradient of Eq. 3."""
    st = _state(N=60, D=5, d=2, kh=8, kl=6, perp=5.0)
    Y = np.random.default_rng(8).standard_normal((60, 2))
    Pd = st.dense_p()
    G = O.exact_grad(Pd, Y, 1.0)
    diff = Y[:, None, :] - Y[None, :, :]
    r2 = (diff ** 2).sum(-1)
    num = 1.0 / (1.0 + r2)
    np.fill_diagonal(num, 0.0)
    Q = num / num.sum()
    G3 = 4.0 * (((Pd - Q) * num)[:, :, None] * diff).sum(1)
    np.testing.assert_allclose(G, G3, rtol=1e-10, atol=1e-14)


def test_large_alpha_is_gaussian_kernel_sne():
    """alpha -> infinity: w -> exp(-r2) and w^{1/alpha} -> 1 (symmetric SNE)."""
    st = _state(N=50, D=5, d=2, kh=8, kl=6, perp=5.0)
    Y = 0.5 * np.random.default_rng(9).standard_normal((50, 2))
    Pd = st.dense_p()
    G = O.exact_grad(Pd, Y, 1e7)
    diff = Y[:, None, :] - Y[None, :, :]
    w = np.exp(-(diff ** 2).sum(-1))
    np.fill_diagonal(w, 0.0)
    Q = w / w.sum()
    Gs = 4.0 * ((Pd - Q)[:, :, None] * diff).sum(1)
    np.testing.assert_allclose(G, Gs, rtol=1e-4, atol=1e-6 * np.abs(Gs).max())


def test_negative_sampling_is_unbiased():
    """Averaged over independent Philox streams, the sampled repulsion and Z
    approach the exhaustive values (Monte-Carlo, 4 sigma)."""
    st = _state(N=80, D=6, d=2, kh=8, kl=6, nneg=4, perp=5.0)
    st.Y[...] = np.random.default_rng(10).standard_normal(st.Y.shape)
    ex = st.copy()
    ex.set(neg_mode=1)
    z = O.exact_z(st.Y, st.alpha)
    A0, R0, z0, _ = ex.forces(zhat=z)
    Rs, Zs = [], []
    for t in range(3000):
        _, R, zt, _ = st.forces(zhat=z, t=t)
        Rs.append(R)
        Zs.append(zt)
    Rs = np.array(Rs)
    Zs = np.array(Zs)
    assert abs(Zs.mean() - z0) < 4 * Zs.std() / math.sqrt(len(Zs))
    m = Rs.mean(0)
    se = Rs.std(0) / math.sqrt(len(Rs)) + 1e-15
    assert np.mean(np.abs(m - R0) < 4 * se) > 0.99


# ---------------------------------------------------------------- step
def test_step_invariants():
    st = _state(N=300, hd_mode=1)
    for _ in range(5):
        old_hd = st.hd_idx.copy()
        out = st.step()
        assert out["coin"]
        changed = np.array([set(a.tolist()) != set(b.tolist()) for a, b in zip(old_hd, st.hd_idx)])
        np.testing.assert_array_equal(changed, out["flags"].astype(bool))
        assert out["n_new"] == changed.sum()
        for i in range(st.N):
            assert len(set(st.hd_idx[i].tolist())) == st.k_hd and i not in st.hd_idx[i]
            assert len(set(st.ld_idx[i].tolist())) == st.k_ld and i not in st.ld_idx[i]
            assert abs(st.P[i].sum() - 1) < 1e-9
        # HD distances never increase position-wise as a set: the k-th distance is monotone
    assert st.t == 5


def test_hd_kth_distance_never_increases():
    st = _state(N=300, hd_mode=1)
    kth = st.hd_d2[:, -1].copy()
    for _ in range(5):
        st.step()
        assert np.all(st.hd_d2[:, -1] <= kth + 1e-12)
        kth = st.hd_d2[:, -1].copy()


def test_coin_probability_follows_smoothed_fraction():
    st = _state(N=50)
    st.set(E=0.0)
    fired = 0
    for t in range(4000):
        st.set(t=t)
        fired += st.coin()
    assert abs(fired / 4000 - 0.05) < 0.012
    st.set(E=1.0)
    assert all(st.coin() for _ in range(3))


def test_coin_floor_sets_the_refinement_probability():
    """Floor f: the coin fires with probability f + (1 - f) E; f = 1 always
    fires and f = 0 with E = 0 never does."""
    st = _state(N=50, coin_floor=0.3)
    st.set(E=0.5)
    fired = 0
    for t in range(4000):
        st.set(t=t)
        fired += st.coin()
    # p = 0.65, standard error 0.0075
    assert abs(fired / 4000 - 0.65) < 0.03
    st.set(coin_floor=0.0, E=0.0)
    assert not any(st.set(t=t) or st.coin() for t in range(2000))
    st.set(coin_floor=1.0)
    assert all(st.set(t=t) or st.coin() for t in range(2000))


@pytest.mark.parametrize("gamma_e,gamma_z", [(1.0, 0.5), (0.5, 1.0)])
def test_smoothing_rates_reach_the_last_values(gamma_e, gamma_z):
    """A rate of 1 keeps only the last value: E becomes the step's fraction
    of points with new HD neighbours, and with exhaustive negatives Zhat
    becomes the exact sum of w over all ordered pairs at the step's starting
    embedding. The other rate (0.5) averages old and new halves."""
    X = synth.blobs(n=200, dim=6, n_clusters=3, seed=62)
    st = O.OracleState(X, 2, 10, 6, 4, 0.8, 5.0, seed=62, neg_mode=1, hd_mode=1, gamma_e=gamma_e,
                       gamma_z=gamma_z)
    for _ in range(4):
        Y0, E0, Z0 = st.Y.copy(), st.E, st.Zhat
        out = st.step()
        frac, z = out["n_new"] / 200, O.exact_z(Y0, 0.8)
        assert out["coin"]
        assert st.E == pytest.approx(frac if gamma_e == 1 else 0.5 * (E0 + frac), rel=1e-15, abs=0)
        assert st.Zhat == pytest.approx(z if gamma_z == 1 else 0.5 * (Z0 + z), rel=1e-10)


def test_whole_run_finds_neighbours_and_structure():
    """Approximate method: statistics only. A short run on Gaussian blobs must
    reach high HD-KNN recall and an embedding that keeps the clusters
    (R_NX at the cluster scale) and part of the local structure."""
    X = synth.blobs(n=600, dim=20, n_clusters=6, seed=11)
    st = O.OracleState(X, 2, 16, 8, 8, 1.0, 10.0, seed=11, exaggeration=4.0, exag_iters=100)
    for _ in range(300):
        st.step()
    exact, _ = O.bruteforce_knn(X, 128)
    assert recall(st.hd_idx, exact[:, :16]) > 0.99
    ld_exact, _ = O.bruteforce_knn(st.Y, 128)
    r = rnx_curve(ld_exact, exact, len(X))
    assert r[99] > 0.6
    assert rnx_auc(ld_exact, exact, len(X), kmax=16) > 0.15


# ---------------------------------------------------------------- insertion
def test_insertion_lists_placement_and_scalars():
    X = synth.blobs(n=700, dim=12, n_clusters=5, seed=13)
    st = O.OracleState(X[:600], 2, 16, 12, 8, 1.0, 8.0, seed=13)
    for _ in range(60):
        st.step()
    z0, e0 = st.Zhat, st.E
    first = st.insert(X[600:])
    assert first == 600 and st.N == 700
    new = np.arange(600, 700)
    for i in new:
        row = st.hd_idx[i]
        assert len(set(row.tolist())) == 16 and row.max() < 600 and row.min() >= 0
        d2 = ((st.X[row] - st.X[i]) ** 2).sum(1)
        assert np.all(np.diff(d2) >= 0)
        # mean placement over the listed HD neighbours
        np.testing.assert_allclose(st.Y[i], st.Y[row].mean(0), rtol=1e-12, atol=1e-15)
        assert np.all(st.V[i] == 0)
        assert st.ld_idx[i].tolist() == row[:12].tolist()
        assert abs(st.P[i].sum() - 1) < 1e-9
    assert abs(st.Zhat - z0 * (700 * 699) / (600 * 599)) <= 1e-12 * st.Zhat
    assert st.E == max(e0, 100 / 700)
    # the default 64 neighbour-of-neighbour rounds from a random start find a
    # large share of the exact neighbours among the existing points (random
    # lists would find about 16/600 of them); later iterations refine the rest
    ex, _ = O.bruteforce_knn(X[:600], 16)
    exact_new = []
    for i in new:
        d2 = ((X[:600].astype(np.float64) - X[i]) ** 2).sum(1)
        exact_new.append(np.lexsort((np.arange(600), d2))[:16])
    assert recall(st.hd_idx[new], np.array(exact_new)) > 0.4
    # the state keeps stepping
    out = st.step()
    assert np.isfinite(st.Y).all() and out["A"].shape == (700, 2)


def test_insertion_rounds():
    """Zero rounds keep the k_hd random starting points (ordered); each
    round is a greedy top-k merge, so the k-th distance never grows with
    more rounds on the same draws, and many rounds reach the exact
    neighbours of well-separated data."""
    X = synth.blobs(n=900, dim=10, n_clusters=4, seed=17)
    base = O.OracleState(X[:800], 2, 12, 6, 6, 1.0, 6.0, seed=17)
    for _ in range(20):
        base.step()
    new = np.arange(800, 900)
    kth, rec = [], []
    exact = np.array([np.lexsort((np.arange(800), ((X[:800].astype(np.float64) - X[i]) ** 2).sum(1)))[:12]
                      for i in new])
    for rounds in (0, 1, 4, 24):
        st = base.copy()
        st.insert(X[800:], rounds=rounds)
        if rounds == 0:
            for i in new:
                w = [O.philox([st.t, i, 5, l], [17, 0])[0] for l in range(12)]
                offs = []
                for u in w:
                    o = (int(u) * 800) >> 32
                    while o in offs:
                        o = (o + 1) % 800
                    offs.append(o)
                assert set(st.hd_idx[i].tolist()) == set(offs)
        d2 = np.array([((st.X[st.hd_idx[i]] - st.X[i]) ** 2).sum(1).max() for i in new])
        kth.append(d2)
        rec.append(recall(st.hd_idx[new], exact))
    for a, b in zip(kth, kth[1:]):
        assert np.all(b <= a + 1e-12)
    assert rec[0] < 0.1 and rec[-1] > 0.9 and rec[-1] >= rec[2] >= rec[1]


def test_fresh_window_refines_only_recent_points():
    """With the coin off (hd_mode 2), an insertion opens a window of
    fresh_iters iterations in which exactly the new points refine their HD
    lists: each new point's list of t+1 is the top-k merge of its list of t
    with its 32 candidates (recomputed here from the state of t), the other
    points' lists stay, E stays, and changed points are recalibrated to the
    target entropy. After the window nothing changes; a second insertion
    inside a window keeps the older points in it; a removal closes it."""
    X = synth.blobs(n=960, dim=10, n_clusters=4, seed=18)
    st = O.OracleState(X[:800], 2, 12, 6, 6, 1.0, 6.0, seed=18, hd_mode=2, fresh_iters=4)
    for _ in range(5):
        st.step()
    st.insert(X[800:900], rounds=0)
    assert st.fresh_lo == 800 and st.fresh_until == st.t + 4
    for it in range(4):
        pre = st.copy()
        e0 = st.E
        out = st.step()
        np.testing.assert_array_equal(st.hd_idx[:800], pre.hd_idx[:800])
        assert st.E == e0 and not out["coin"]
        changed = 0
        for i in range(800, 900):
            cand = pre.hd_candidates(i)
            cd2 = ((pre.X[cand] - pre.X[i]) ** 2).sum(1)
            od2 = ((pre.X[pre.hd_idx[i]] - pre.X[i]) ** 2).sum(1)
            ni, _, ch = O.topk_merge(i, pre.hd_idx[i], od2, cand, cd2)
            np.testing.assert_array_equal(st.hd_idx[i], ni)
            if ch:
                changed += 1
                h, _ = O.entropy(((st.X[ni] - st.X[i]) ** 2).sum(1), st.beta[i])
                assert abs(h - np.log(6.0)) < 1e-8
        assert changed > 0 or it > 0
    before = st.hd_idx.copy()
    st.step()
    np.testing.assert_array_equal(st.hd_idx, before)  # window closed
    st.step()
    st.insert(X[900:930], rounds=0)
    assert st.fresh_lo == 900
    st.step()
    st.insert(X[930:], rounds=0)  # inside the open window: it keeps point 900 on
    assert st.fresh_lo == 900 and st.fresh_until == st.t + 4
    st.remove(np.array([3, 950]))
    assert st.fresh_until == st.t and st.fresh_lo == st.N


def test_insertion_with_more_ld_than_hd_neighbours():
    X = synth.blobs(n=300, dim=6, n_clusters=3, seed=14)
    st = O.OracleState(X[:250], 2, 8, 12, 4, 1.0, 5.0, seed=14)
    st.insert(X[250:])
    for i in range(250, 300):
        row = st.ld_idx[i]
        assert len(set(row.tolist())) == 12 and row.max() < 250
        assert row[:8].tolist() == st.hd_idx[i].tolist()


# ---------------------------------------------------------------- live changes
def test_perplexity_change_recalibrates_every_point():
    X = synth.blobs(n=400, dim=8, n_clusters=4, seed=40)
    st = O.OracleState(X, 2, 16, 8, 8, 1.0, 6.0, seed=40)
    for _ in range(10):
        st.step()
    sets = [set(r.tolist()) for r in st.hd_idx]
    st.set_perplexity(11.0)
    for i in range(400):
        assert set(st.hd_idx[i].tolist()) == sets[i]
        P = st.P[i]
        assert abs(P.sum() - 1) < 1e-12
        H = -np.sum(P[P > 0] * np.log(P[P > 0]))
        assert abs(H - np.log(11.0)) < 1e-8
        # P follows Eq. 1 with the point's beta over the shifted distances
        d2 = st.hd_d2[i]
        q = np.exp(-st.beta[i] * (d2 - d2[0]))
        np.testing.assert_allclose(P, q / q.sum(), rtol=1e-12, atol=1e-15)


def test_drifted_rows_refresh_list_distances():
    X = synth.blobs(n=300, dim=6, n_clusters=3, seed=41)
    st = O.OracleState(X, 2, 12, 6, 6, 1.0, 5.0, seed=41)
    for _ in range(8):
        st.step()
    ids = np.array([3, 77, 150])
    rows = X[ids] + 2.5
    st.update_rows(ids, rows)
    X2 = X.astype(np.float64).copy()
    X2[ids] = rows
    for i in range(300):
        d2 = ((X2[st.hd_idx[i]] - X2[i]) ** 2).sum(1)
        np.testing.assert_allclose(st.hd_d2[i], d2, rtol=1e-14)
        assert np.all(np.diff(d2) >= 0)
        assert abs(st.P[i].sum() - 1) < 1e-12


def test_removal_renumbers_replaces_and_recalibrates():
    X = synth.blobs(n=500, dim=8, n_clusters=4, seed=42)
    st = O.OracleState(X, 2, 12, 8, 6, 1.0, 6.0, seed=42)
    for _ in range(10):
        st.step()
    before = st.copy()
    ids = np.array([0, 5, 17, 250, 499])
    keep = np.setdiff1d(np.arange(500), ids)
    new_of = -np.ones(500, dtype=np.int64)
    new_of[keep] = np.arange(len(keep))
    z0, e0 = st.Zhat, st.E
    n = st.remove(ids)
    assert n == 495 and st.N == 495 and st.X.shape == (495, 8)
    np.testing.assert_array_equal(st.X, X[keep].astype(np.float64))
    np.testing.assert_array_equal(st.Y, before.Y[keep])
    np.testing.assert_array_equal(st.V, before.V[keep])
    assert abs(st.Zhat - z0 * (495 * 494) / (500 * 499)) <= 1e-12 * z0
    assert st.E == max(e0, 5 / 500)
    for n_i, o_i in enumerate(keep):
        for lst_new, lst_old, k, salt in ((st.hd_idx, before.hd_idx, 12, 0), (st.ld_idx, before.ld_idx, 8, 1024)):
            row = lst_new[n_i]
            assert len(set(row.tolist())) == k and row.min() >= 0 and row.max() < 495 and n_i not in row
            kept_old = [new_of[j] for j in lst_old[o_i] if new_of[j] >= 0]
            assert set(kept_old) <= set(row.tolist())
        # the replacement rule, re-derived for the LD list (its order is kept)
        old = before.ld_idx[o_i]
        row = [int(new_of[j]) for j in old]
        for e in range(8):
            if row[e] >= 0:
                continue
            w = O.philox([st.t, n_i, 11, 1024 + e], [42, 0])[0]
            j = (int(w) * 494) >> 32
            j += j >= n_i
            while j in row:
                j = (j + 1) % 495
                if j == n_i:
                    j = (j + 1) % 495
            row[e] = j
        assert row == st.ld_idx[n_i].tolist()
        d2 = ((st.X[st.hd_idx[n_i]] - st.X[n_i]) ** 2).sum(1)
        np.testing.assert_allclose(st.hd_d2[n_i], d2, rtol=1e-14)
        assert abs(st.P[n_i].sum() - 1) < 1e-12
    st.step()
    assert np.isfinite(st.Y).all()


def test_jump_start_projects_instead_of_stepping():
    """While t < jump_iters: Y is a centred random linear projection of X with
    per-dimension std 1e-4, renewed at t = 0 and t = jump_iters / 2 (two
    parts), V stays 0; afterwards the gradient moves Y."""
    X = synth.blobs(n=300, dim=12, n_clusters=3, seed=60)
    st = O.OracleState(X, 3, 12, 8, 8, 1.0, 6.0, seed=60, jump_iters=6, jump_parts=2)
    Xc = st.X - st.X.mean(0)
    ys = []
    for t in range(8):
        st.step()
        ys.append(st.Y.copy())
        if t < 6:
            assert np.all(st.V == 0)
            np.testing.assert_allclose(st.Y.std(0), 1e-4, rtol=1e-9)
            np.testing.assert_allclose(st.Y.mean(0), 0.0, atol=1e-18)
            # Y is linear in the centred data
            M, res, *_ = np.linalg.lstsq(Xc, st.Y, rcond=None)
            assert np.abs(Xc @ M - st.Y).max() < 1e-12 * np.abs(st.Y).max()
    for t in (1, 2, 4, 5):
        np.testing.assert_array_equal(ys[t], ys[t - 1])
    assert not np.allclose(ys[3], ys[2])          # the second projection at t = 3
    assert not np.allclose(ys[7], ys[6]) and np.any(st.V != 0)


def test_implosion_scales_and_reestimates_z():
    """Scaling Y and V by f; with exhaustive negatives the new Zhat is the
    exact sum of w over all ordered pairs at the scaled embedding."""
    X = synth.blobs(n=200, dim=6, n_clusters=3, seed=61)
    st = O.OracleState(X, 2, 10, 6, 4, 0.8, 5.0, seed=61, neg_mode=1)
    for _ in range(5):
        st.step()
    Y0, V0 = st.Y.copy(), st.V.copy()
    st.scale(0.1)
    np.testing.assert_array_equal(st.Y, Y0 * 0.1)
    np.testing.assert_array_equal(st.V, V0 * 0.1)
    assert abs(st.Zhat - O.exact_z(st.Y, 0.8)) <= 1e-10 * st.Zhat


# ---------------------------------------------------------------- learned placement (MLP)
def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(20).standard_normal(20000) * np.exp(np.random.default_rng(21).uniform(-20, 20, 20000))
    x[:5] = [1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -(1.0 + 2 ** -8), 0.0, 65504.0]
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(O.bf16(x), ref)
    assert O.lib().oracle_bf16(1.0 + 2 ** -8) == 1.0  # tie to even


def test_mlp_gradient_matches_finite_differences():
    rng = np.random.default_rng(22)
    D, H, d, B = 6, 10, 3, 7
    th = O.mlp_init(D, H, d, 5) + 0.05 * rng.standard_normal(O.mlp_size(D, H, d))
    X = rng.standard_normal((B, D))
    T = rng.standard_normal((B, d))
    loss, g, _ = O.mlp_grad(th, X, T, H, round_bf16=False)
    h = 1e-6
    for e in rng.choice(len(th), 40, replace=False):
        tp, tm = th.copy(), th.copy()
        tp[e] += h
        tm[e] -= h
        fd = (O.mlp_grad(tp, X, T, H, False)[0] - O.mlp_grad(tm, X, T, H, False)[0]) / (2 * h)
        assert abs(fd - g[e]) <= 1e-6 * max(1.0, abs(g).max())


def test_mlp_forward_is_the_composition_of_layers():
    # an independent numpy restatement of the network for one input
    rng = np.random.default_rng(23)
    D, H, d = 4, 6, 2
    th = O.mlp_init(D, H, d, 3)
    W1 = th[:H * D].reshape(H, D)
    b1 = th[H * D:H * D + H]
    o = H * D + H
    W2 = th[o:o + H * H].reshape(H, H)
    b2 = th[o + H * H:o + H * H + H]
    o += H * H + H
    W3 = th[o:o + d * H].reshape(d, H)
    b3 = th[o + d * H:]
    x = rng.standard_normal((5, D))
    ref = np.maximum(np.maximum(x @ W1.T + b1, 0) @ W2.T + b2, 0) @ W3.T + b3
    np.testing.assert_allclose(O.mlp_forward(th, x, H, d, round_bf16=False), ref, rtol=1e-12, atol=1e-14)


def test_mlp_magnitudes_bound_and_equal_without_cancellation():
    """oracle_mlp_grad_mag: with nonnegative weights, biases and inputs and
    negative targets nothing cancels and every ReLU is open, so the
    magnitudes equal the gradient and outputs themselves; with signed
    parameters they bound them (triangle inequality)."""
    rng = np.random.default_rng(26)
    D, H, d, B = 5, 9, 3, 11
    n = O.mlp_size(D, H, d)
    th = np.abs(rng.standard_normal(n)) * 0.3
    X = np.abs(rng.standard_normal((B, D)))
    T = -np.abs(rng.standard_normal((B, d))) - 0.5
    _, g, out = O.mlp_grad(th, X, T, H, round_bf16=False)
    gm, om = O.mlp_grad_mag(th, X, T, H)
    np.testing.assert_allclose(gm, g, rtol=1e-12, atol=0)
    np.testing.assert_allclose(om, out, rtol=1e-12, atol=0)
    th = rng.standard_normal(n) * 0.3
    X = rng.standard_normal((B, D))
    T = rng.standard_normal((B, d))
    _, g, out = O.mlp_grad(th, X, T, H, round_bf16=False)
    gm, om = O.mlp_grad_mag(th, X, T, H)
    assert np.all(np.abs(g) <= gm * (1 + 1e-12)) and np.all(np.abs(out) <= om * (1 + 1e-12))
    assert np.mean(np.abs(g) < 0.5 * gm) > 0.1  # signed terms do cancel


def test_mlp_standardisation_and_target_scaling():
    """Closed forms: a feature a + b z (z with mean 0 and population variance
    1) has mean a and std |b|; a constant feature gets std 1; standardised
    inputs are bfloat16 values within one bfloat16 rounding of z; targets
    have RMS 1 (exactly 1 for s computed from them) and all-zero targets keep
    s = 1."""
    z = np.array([-1.5, -0.5, 0.5, 1.5, 0.0, 0.0])
    z = (z - z.mean()) / z.std()
    X = np.stack([3.0 + 2.0 * z, -1.0 - 0.25 * z, np.full(6, 7.0)], axis=1)
    mean, std = O.mlp_stats(X)
    np.testing.assert_allclose(mean, [3.0, -1.0, 7.0], rtol=0, atol=1e-12)
    np.testing.assert_allclose(std, [2.0, 0.25, 1.0], rtol=1e-12)
    xin = O.mlp_inputs(X, np.arange(6), mean, std)
    np.testing.assert_array_equal(xin, O.bf16(xin))
    np.testing.assert_allclose(xin[:, 0], z, rtol=2 ** -8, atol=1e-6)
    np.testing.assert_allclose(xin[:, 1], -z, rtol=2 ** -8, atol=1e-6)
    np.testing.assert_array_equal(xin[:, 2], 0.0)
    Y = np.random.default_rng(31).standard_normal((50, 3))
    T, sc = O.mlp_targets(Y, np.arange(10, 40))
    assert abs(np.sqrt(np.mean(T * T)) - 1.0) < 1e-12
    np.testing.assert_allclose(T * sc, Y[10:40], rtol=1e-14)
    T0, s0 = O.mlp_targets(np.zeros((5, 2)), np.arange(5))
    assert s0 == 1.0 and np.all(T0 == 0)


def test_mlp_init_ranges():
    D, H, d = 50, 256, 8
    th = O.mlp_init(D, H, d, 0)
    W1 = th[:H * D]
    a = np.sqrt(6 / D)
    assert np.abs(W1).max() < a and abs(W1.mean()) < 0.02 * a
    assert abs(W1.var() - a * a / 3) < 0.05 * a * a / 3
    assert np.all(th[H * D:H * D + H] == 0)
    assert np.all(th.astype(np.float32).astype(np.float64) == th)  # binary32 values


def test_adam_first_step_closed_form():
    g = np.array([0.3, -2.0, 1e-9, 0.0])
    th = np.zeros(4)
    m = np.zeros(4)
    v = np.zeros(4)
    O.adam(th, g, m, v, 1, lr=1e-3, eps=1e-8)
    # first step: m_hat = g, v_hat = g^2, so the update is lr g / (|g| + eps)
    np.testing.assert_allclose(th, -1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)


def test_mlp_training_fits_a_smooth_map():
    rng = np.random.default_rng(24)
    D, H, d, B = 8, 32, 2, 256
    A = rng.standard_normal((D, d))
    X = rng.standard_normal((4 * B, D))
    T = np.tanh(X @ A)
    th = O.mlp_init(D, H, d, 1)
    m = np.zeros_like(th)
    v = np.zeros_like(th)
    losses = []
    for step in range(1, 301):
        b = rng.choice(len(X), B, replace=False)
        loss, g, _ = O.mlp_grad(th, O.bf16(X[b]), T[b], H, round_bf16=True)
        losses.append(loss)
        O.adam(th, g, m, v, step, lr=3e-3)
    assert np.mean(losses[-20:]) < 0.2 * np.mean(losses[:5])


def test_sampled_forces_equal_full_forces():
    st = _state(N=250, D=8, d=3, kh=12, kl=8, nneg=40, perp=6.0)
    st.Y[...] = np.random.default_rng(25).standard_normal(st.Y.shape)
    A, R, _, _ = st.forces(zhat=123.0, t=7)
    pts = np.array([0, 5, 17, 249, 100])
    As, Rs = st.forces_points(pts, zhat=123.0, t=7)
    np.testing.assert_allclose(As, A[pts], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(Rs, R[pts], rtol=1e-12, atol=1e-15)


def test_results_do_not_depend_on_the_thread_count():
    """The oracle runs its per-point loops on several threads; every sum
    keeps a fixed index order, so one and four threads give the same bits."""
    X = synth.spectrum(n=1500, dim=12, n_clusters=6, seed=27)
    runs = []
    for nt in (1, 4):
        O.set_threads(nt)
        st = O.OracleState(X, 3, 16, 12, 20, 0.8, 9.0, seed=27, hd_mode=0, fresh_iters=3)
        outs = [st.step() for _ in range(6)]
        st.insert(synth.spectrum(n=100, dim=12, n_clusters=6, seed=28), rounds=4)
        outs += [st.step() for _ in range(3)]
        runs.append((st, outs))
    O.set_threads(0)
    (a, oa), (b, ob) = runs
    for name in ("Y", "V", "hd_idx", "ld_idx", "beta", "P"):
        np.testing.assert_array_equal(getattr(a, name), getattr(b, name))
    assert a.Zhat == b.Zhat and a.E == b.E
    for x, y in zip(oa, ob):
        np.testing.assert_array_equal(x["A"], y["A"])
        np.testing.assert_array_equal(x["z"], y["z"])
