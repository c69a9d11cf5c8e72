"""GPU parity of the live changes of the point set against the oracle, from
the same exported state: a new perplexity, drifted rows of X, removed
points (renumbering and replacement draws are integer work: bit-exact), and
an iteration after each. Also insertions below a grown capacity after a
change of storage precision."""
import numpy as np
import pytest

from paper_2509_07681_gb300 import funcsne as F
from paper_2509_07681_gb300 import synth

from gpu_util import (align_to, check_after_refinement, check_calibration, compare_sets, fp32_band, lib,
                      oracle_from_state, rel_err_rows)

pytestmark = pytest.mark.gpu

P = dict(d=2, k_hd=16, k_ld=8, n_neg=8, alpha=1.0, perplexity=8.0)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    lib()


def _run(X, steps=15, **opts):
    m = F.FuncSNE(X, P["d"], P["k_hd"], P["k_ld"], P["n_neg"], P["alpha"], P["perplexity"], seed=0, hd_mode=1,
                  **opts)
    m.step(steps)
    m.sync()
    return m


def _check_calibration(st, o, rows):
    """Same HD sets (the lists are kept), rows ordered by distance, and the
    cold calibration of every point (Eq. 1) against the oracle's within the
    bounds the two stopping rules imply."""
    for i in range(len(st["hd_idx"])):
        assert set(st["hd_idx"][i].tolist()) == set(o.hd_idx[i].tolist())
        d2 = ((rows[st["hd_idx"][i]] - rows[i]) ** 2).sum(1)
        assert np.all(np.diff(d2) >= -fp32_band(rows.shape[1]) * d2[-1])
    allr = np.arange(len(st["hd_idx"]))
    check_calibration(rows, allr, st["hd_idx"], st["beta"], st["P"], o.beta,
                      align_to(st["hd_idx"], o.hd_idx, o.P), o.perplexity, rows.shape[1])


def _one_more_iteration(m, X, st, hd_mode=1):
    """One iteration after the change: sets against the oracle's own step,
    then everything after the refinement on every row."""
    o = oracle_from_state(X, st, P, hd_mode=hd_mode)
    att, rep = m.debug_step()
    o.step()
    st1 = m.export_state()
    bad, amb = compare_sets(st1["hd_idx"], o.hd_idx, range(len(X)), o.X, fp32_band(X.shape[1]))
    assert bad == 0 and amb <= 3
    check_after_refinement(X, st, st1, att, rep, m.stats(), P, m.get_option("lr"), momentum=m.get_option("momentum"),
                           label="after change", hd_mode=hd_mode)


def test_perplexity_change_matches_oracle():
    X = synth.blobs(n=1500, dim=20, n_clusters=5, seed=50)
    m = _run(X)
    st = m.export_state()
    o = oracle_from_state(X, st, P, hd_mode=1)
    m.set_option("perplexity", 12.0)
    assert m.get_option("perplexity") == 12.0
    o.set_perplexity(12.0)
    st1 = m.export_state()
    _check_calibration(st1, o, X.astype(np.float64))
    assert st1["Zhat"] == st["Zhat"] and st1["E"] == st["E"] and st1["t"] == st["t"]
    with pytest.raises(F.FuncSNEError):
        m.set_option("perplexity", 17.5)
    m.close()


def test_drifted_rows_match_oracle():
    X = synth.blobs(n=1500, dim=20, n_clusters=5, seed=51)
    m = _run(X, precision=F.BF16)
    st = m.export_state()
    o = oracle_from_state(X, st, P, hd_mode=1)
    ids = np.array([4, 99, 700, 1499])
    rows = X[ids][::-1] + 0.5
    m.update_points(ids, rows)
    o.update_rows(ids, rows)
    X2 = X.copy()
    X2[ids] = rows
    st1 = m.export_state()
    _check_calibration(st1, o, X2.astype(np.float64))
    # the BF16 copy follows the new rows: one iteration equals FP32's
    ref = m.export_state()
    m.step(1)
    b = m.export_state()
    m.set_option("precision", F.FP32)
    m.import_state(ref)
    m.step(1)
    a = m.export_state()
    np.testing.assert_array_equal(a["hd_idx"], b["hd_idx"])
    with pytest.raises(F.FuncSNEError):
        m.update_points(np.array([3, 3]), X[:2])
    with pytest.raises(F.FuncSNEError):
        bad = X[:1].copy()
        bad[0, 0] = np.nan
        m.update_points(np.array([5]), bad)
    m.close()


@pytest.mark.parametrize("precision", [F.FP32, F.FP8])
def test_removal_matches_oracle(precision):
    X = synth.blobs(n=1600, dim=20, n_clusters=5, seed=52)
    m = _run(X, precision=precision)
    st = m.export_state()
    o = oracle_from_state(X, st, P, hd_mode=1)
    rng = np.random.default_rng(3)
    ids = np.sort(rng.choice(1600, 100, replace=False))
    ids = np.unique(np.concatenate([ids, [0, 1599]]))
    keep = np.setdiff1d(np.arange(1600), ids)
    m.remove(ids[::-1].copy())
    n = o.remove(ids)
    assert m.N == n == len(keep) and m.stats()["N"] == n
    st1 = m.export_state()
    # renumbering and replacement draws: bit-exact
    np.testing.assert_array_equal(st1["ld_idx"], o.ld_idx)
    np.testing.assert_array_equal(np.sort(st1["hd_idx"], 1), np.sort(o.hd_idx, 1))
    np.testing.assert_array_equal(st1["Y"], st["Y"][keep])
    np.testing.assert_array_equal(st1["V"], st["V"][keep])
    assert abs(st1["Zhat"] - o.Zhat) <= 1e-12 * o.Zhat and st1["E"] == o.E
    Xk = X[keep]
    _check_calibration(st1, o, Xk.astype(np.float64))
    _one_more_iteration(m, Xk, st1)
    with pytest.raises(F.FuncSNEError):
        m.remove(np.arange(m.N - 10))
    m.close()


def test_insertion_below_grown_capacity_after_precision_change():
    """Capacity grows on the first insertion; the BF16 copy created after it
    must cover the capacity, so the second insertion (no growth) fits."""
    X = synth.blobs(n=2600, dim=24, n_clusters=6, seed=53)
    m = _run(X[:2000])
    m.insert(X[2000:2100])
    m.set_option("precision", F.BF16)
    m.insert(X[2100:2600])
    m.step(5)
    m.sync()
    st = m.export_state()
    assert m.N == 2600 and np.isfinite(st["Y"]).all()
    m.step(1)
    b = m.export_state()
    m.set_option("precision", F.FP32)
    m.import_state(st)
    m.step(1)
    a = m.export_state()
    np.testing.assert_array_equal(a["hd_idx"], b["hd_idx"])
    m.close()


def test_checkpoint_resume(tmp_path):
    """save() / load_checkpoint(): the resumed handle's next iteration gives
    the same lists as the original's (the lists do not depend on the order of
    the force atomics) and nearly the same positions."""
    X = synth.blobs(n=1800, dim=20, n_clusters=5, seed=54)
    m = _run(X, precision=F.BF16)
    m.set_option("momentum", 0.7)
    m.remove(np.array([3, 4, 5]))
    m.step(3)
    m.sync()
    path = str(tmp_path / "ckpt.npz")
    m.save(path)
    m2 = F.FuncSNE.load_checkpoint(path)
    assert m2.N == m.N and m2.get_option("momentum") == 0.7 and m2.get_option("precision") == F.BF16
    np.testing.assert_array_equal(m2.data(), m.data())
    a, b = m.export_state(), m2.export_state()
    for k in ("hd_idx", "ld_idx", "Y", "V"):
        np.testing.assert_array_equal(a[k], b[k])
    assert a["t"] == b["t"] and a["Zhat"] == b["Zhat"] and a["E"] == b["E"]
    m.step(1)
    m2.step(1)
    a, b = m.export_state(), m2.export_state()
    np.testing.assert_array_equal(a["hd_idx"], b["hd_idx"])
    np.testing.assert_array_equal(a["ld_idx"], b["ld_idx"])
    np.testing.assert_allclose(a["Y"], b["Y"], rtol=1e-4, atol=1e-5 * np.abs(a["Y"]).max())
    m.close()
    m2.close()


def test_jump_start_matches_oracle():
    """Jump start: at t = 0 and t = 3 (jump_iters 6, two parts) the embedding
    is the oracle's random linear projection; in between no gradient moves
    it; afterwards the gradient steps resume."""
    X = synth.blobs(n=1500, dim=20, n_clusters=5, seed=55)
    m = F.FuncSNE(X, P["d"], P["k_hd"], P["k_ld"], P["n_neg"], P["alpha"], P["perplexity"], seed=0, hd_mode=1,
                  jump_iters=6, jump_parts=2)
    st = m.export_state()
    o = oracle_from_state(X, st, P, hd_mode=1, jump_iters=6, jump_parts=2)
    ys = []
    for t in range(7):
        m.step(1)
        o.step()
        g = m.export_state()
        if t in (0, 3):
            assert np.max(rel_err_rows(g["Y"].astype(np.float64), o.Y)) < 1e-5
        if t < 6:
            assert np.all(g["V"] == 0)
        ys.append(g["Y"])
    np.testing.assert_array_equal(ys[1], ys[0])
    np.testing.assert_array_equal(ys[5], ys[3])
    assert not np.array_equal(ys[3], ys[2]) and not np.array_equal(ys[6], ys[5])
    m.close()


def test_implosion_matches_oracle():
    X = synth.blobs(n=1500, dim=20, n_clusters=5, seed=56)
    m = _run(X, steps=20)
    st = m.export_state()
    o = oracle_from_state(X, st, P, hd_mode=1)
    m.scale_embedding(0.1)
    o.scale(0.1)
    g = m.export_state()
    assert np.max(rel_err_rows(g["Y"].astype(np.float64), o.Y)) < 1e-6
    assert abs(g["Zhat"] - o.Zhat) <= 1e-5 * o.Zhat and g["Zhat"] > st["Zhat"]
    with pytest.raises(F.FuncSNEError):
        m.scale_embedding(0.0)
    m.step(2)
    assert np.isfinite(m.embedding()).all()
    m.close()


def test_alpha_annealing_snapshots():
    """anneal(): one snapshot per tail weight; lowering alpha during the run
    changes the forces (the snapshots differ) and keeps the run finite."""
    X = synth.blobs(n=1200, dim=12, n_clusters=4, seed=57)
    m = _run(X, steps=30)
    snaps = m.anneal([1.0, 0.5, 0.25], 10)
    assert len(snaps) == 3 and all(s.shape == (1200, 2) for s in snaps)
    assert m.get_option("alpha") == 0.25
    assert all(np.isfinite(s).all() for s in snaps) and not np.array_equal(snaps[1], snaps[2])
    m.close()


@pytest.mark.parametrize("d", [2, 3])
def test_async_embedding_readout(d):
    """get_embedding_async snapshots Y after the steps queued before it: the
    copy equals a synchronous read taken at the same point, though more steps
    run while it is in flight; back-to-back read-outs into two buffers (the
    second waits on the device for the first) each hold their own step."""
    import torch
    X = synth.blobs(n=3000, dim=20, n_clusters=5, seed=58)
    m = F.FuncSNE(X, d, 16, 8, 8, 1.0, 8.0, seed=0)
    bufs = [torch.empty((3000, d), dtype=torch.float32).pin_memory() for _ in range(2)]
    m.step(3)
    m.embedding_async(bufs[0])
    ref = m.embedding()
    m.step(5)
    m.wait_embedding()
    np.testing.assert_array_equal(bufs[0].numpy(), ref)
    assert not np.array_equal(m.embedding(), ref)
    refs = []
    for k in range(4):
        m.step(1)
        m.embedding_async(bufs[k % 2])
        refs.append(m.embedding())
        if k % 2:
            m.wait_embedding()
            np.testing.assert_array_equal(bufs[0].numpy(), refs[k - 1])
            np.testing.assert_array_equal(bufs[1].numpy(), refs[k])
    part = torch.zeros((100, d), dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    m.embedding_async(part)
    m.sync()
    np.testing.assert_array_equal(part.cpu().numpy(), m.embedding()[:100])
    m.close()


def test_pitched_copies_round_trip():
    """Rows of D = 30 floats live in rows of 32 on the device and LD rows of
    d = 3 in rows of 4: copies between them and host or device buffers of
    the caller (staged through a contiguous device buffer when a host side
    is pitched) return the caller's values exactly."""
    import torch
    X = synth.blobs(n=2000, dim=30, n_clusters=4, seed=59)
    Xn = X[1500:]
    m = F.FuncSNE(X[:1500], 3, 16, 8, 8, 1.0, 8.0, seed=0)
    np.testing.assert_array_equal(m.data(), X[:1500])
    m.step(3)
    st = m.export_state()
    m.import_state(st)
    np.testing.assert_array_equal(m.export_state()["Y"], st["Y"])
    np.testing.assert_array_equal(m.embedding(), st["Y"])
    m.insert(Xn[:200])
    dev = torch.from_numpy(Xn[200:]).cuda()
    torch.cuda.synchronize()
    m.insert(dev)
    np.testing.assert_array_equal(m.data(), X)
    out = torch.empty((2000, 30), dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    m.data(out=out)
    np.testing.assert_array_equal(out.cpu().numpy(), X)
    m.close()
    # a device tensor as the input of create
    Xd = torch.from_numpy(X).cuda()
    torch.cuda.synchronize()
    m2 = F.FuncSNE(Xd, 3, 16, 8, 8, 1.0, 8.0, seed=0)
    np.testing.assert_array_equal(m2.data(), X)
    m2.close()


def test_bounded_device_wait_is_reported_and_context_survives():
    """Failure detection without a fault: a device wait on an mbarrier that
    nothing arrives on gives up after its poll limit and sets the error bit
    the tensor-core kernels use; funcsne_sync reports it, and the CUDA
    context stays usable for a new handle."""
    X = synth.blobs(n=1000, dim=20, n_clusters=4, seed=60)
    m = F.FuncSNE(X, 2, 16, 8, 8, 1.0, 8.0, seed=0)
    m.step(2)
    m.sync()
    with pytest.raises(F.FuncSNEError):
        m.debug_bounded_wait(0)
    m.debug_bounded_wait(1000)
    with pytest.raises(F.FuncSNEError, match="timed out"):
        m.sync()
    m.close()
    m2 = F.FuncSNE(X, 2, 16, 8, 8, 1.0, 8.0, seed=0)
    m2.step(3)
    m2.sync()
    assert np.isfinite(m2.embedding()).all()
    m2.close()


def test_allocation_failure_is_reported_and_the_library_stays_usable():
    """Failure detection without a fault: allocation failures injected on the
    host (funcsne_debug_fail_alloc) at several points of funcsne_create and
    of an insertion's capacity growth return FUNCSNE_E_OOM; a failed create
    leaves nothing behind, a failed insertion leaves the handle's points and
    state as they were, and both the handle and new handles keep working."""
    X = synth.blobs(n=1400, dim=20, n_clusters=4, seed=61)
    failed = 0
    for after in (0, 1, 3, 6, 10):
        F.funcsne_debug_fail_alloc(after)
        try:
            m = F.FuncSNE(X[:1000], 2, 16, 8, 8, 1.0, 8.0, seed=0)
        except F.FuncSNEError as e:
            assert e.code == -2, e  # FUNCSNE_E_OOM
            failed += 1
        else:
            m.close()
    F.funcsne_debug_fail_alloc(-1)
    assert failed >= 4
    m = F.FuncSNE(X[:1000], 2, 16, 8, 8, 1.0, 8.0, seed=0)
    m.step(3)
    st = m.export_state()
    for after in (0, 4, 9):
        F.funcsne_debug_fail_alloc(after)
        with pytest.raises(F.FuncSNEError) as ei:
            m.insert(X[1000:1200])
        assert ei.value.code == -2
        F.funcsne_debug_fail_alloc(-1)
        assert m.N == 1000 and m.stats()["N"] == 1000
        st1 = m.export_state()
        for k in ("Y", "hd_idx", "ld_idx", "beta", "P"):
            np.testing.assert_array_equal(st1[k], st[k])
    m.step(3)
    m.sync()
    assert m.insert(X[1000:1200]) == 1000 and m.N == 1200
    m.step(3)
    m.sync()
    assert np.isfinite(m.embedding()).all() and m.stats()["error_word"] == 0
    m.close()
