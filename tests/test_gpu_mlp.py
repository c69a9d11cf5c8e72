"""GPU parity of the placement MLP (forward, backward, Adam) against the FP64
oracle on identical bfloat16 operands, and its online training. What the
trained network gains over mean placement of inserted points is measured
in test_gpu_dynamic.py."""
import numpy as np
import pytest

import oracle as O
from paper_2509_07681_gb300 import funcsne as F
from paper_2509_07681_gb300 import synth

from gpu_util import lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    lib()


def _split_theta(th, D, H, d):
    o = [0, H * D, H * D + H, H * D + H + H * H, H * D + 2 * H + H * H, H * D + 2 * H + H * H + d * H]
    return o


# Element-wise comparison of a tensor-core result with the oracle's FP64
# result on the same bfloat16 operands, against the magnitude M of each
# element (oracle_mlp_grad_mag: the sum of the magnitudes of its terms,
# propagated through the layers). FP32 accumulation over K terms moves an
# element by at most about K 2^-24 M; the bound takes K = 1024, above every
# sum of these shapes (batch, input and hidden widths). An intermediate
# whose FP32 and FP64 values straddle a bfloat16 rounding boundary rounds one
# bfloat16 ulp apart on the two sides; it is one term among its element's
# many, so it stays inside the same bound unless the element has a handful
# of terms.
ELEM_TOL = 1024 * 2.0 ** -24


def _elem_err(gpu, ref, mag):
    gpu = np.asarray(gpu, dtype=np.float64).ravel()
    ref = np.asarray(ref, dtype=np.float64).ravel()
    mag = np.asarray(mag, dtype=np.float64).ravel()
    return float(np.max(np.abs(gpu - ref) / np.maximum(mag, 1e-300)))


@pytest.mark.parametrize("D,d,H,B", [(24, 4, 64, 512), (50, 3, 100, 300)])
def test_mlp_step_matches_oracle(D, d, H, B):
    """One training step against the oracle; the second shape leaves ragged
    tensor-core tiles (rows, columns and K values past the matrices) and rows
    that are not 16-byte multiples (single-value operand staging)."""
    X = synth.swissroll(n=3000, dim=D, n_clusters=8, seed=30)
    m = F.FuncSNE(X, d, 16, 8, 8, 1.0, 10.0, seed=3)
    m.set_option("mlp_batch", B)
    m.set_option("mlp_hidden", H)
    m.step(30)
    Y = m.embedding().astype(np.float64)
    for it in range(2):
        a = m.mlp_debug_step()
        assert a["step"] == it + 1
        # the batch: Philox counter (step, b, MLP, 0), word 0 mapped to [0, N)
        w0 = np.array([O.philox([it, b, 4, 0], [3, 0])[0] for b in range(B)], dtype=np.uint64)
        np.testing.assert_array_equal(a["batch_idx"], ((w0 * 3000) >> 32).astype(np.int32))
        idx = a["batch_idx"]
        # inputs: the oracle's standardisation of the batch rows, rounded to
        # bfloat16 in binary32 as on the device. The two sides' FP64 means
        # and stds differ only in summation order, which can move a binary32
        # mean or std by one ulp: at most one bfloat16 step, on rare elements
        mu, sd = O.mlp_stats(X)
        ref_x = O.mlp_inputs(X, idx, mu, sd)
        assert np.mean(a["xhat"] == ref_x) > 0.999
        assert np.max(np.abs(a["xhat"] - ref_x) / np.maximum(np.abs(ref_x), 1e-3)) <= 2 ** -7
        # targets: the oracle's y / RMS over the batch (FP64 against FP32)
        ref_t, s = O.mlp_targets(Y, idx)
        assert abs(a["scale"] - s) <= 1e-6 * s
        np.testing.assert_allclose(a["target"], ref_t, rtol=1e-6, atol=1e-7)
        # forward / backward on the same bfloat16 weights and FP32 biases
        o = _split_theta(None, D, H, d)
        th = a["weights_bf16"].astype(np.float64).copy()
        for lo, hi in [(o[1], o[2]), (o[3], o[4]), (o[5], len(th))]:
            th[lo:hi] = a["theta_before"][lo:hi]
        loss, g, out = O.mlp_grad(th, a["xhat"], a["target"], H, round_bf16=True)
        gm, om = O.mlp_grad_mag(th, a["xhat"], a["target"], H)
        assert abs(a["loss"] - loss) <= 1e-4 * loss
        # element by element: outputs and every gradient block (W1 b1 W2 b2 W3 b3)
        eo = _elem_err(a["output"], out, om)
        eg = [_elem_err(a["grad"][lo:hi], g[lo:hi], gm[lo:hi]) for lo, hi in zip(o, o[1:] + [len(th)])]
        print(f"MLP D={D} H={H} B={B} step {it}: max |gpu - oracle| / magnitude: output {eo:.2e}, gradient "
              f"blocks " + " ".join(f"{e:.2e}" for e in eg))
        assert eo < ELEM_TOL, eo
        for (lo, hi), e in zip(zip(o, o[1:] + [len(th)]), eg):
            assert e < ELEM_TOL, (lo, hi, e)
        # Adam from the exported moments' state: first steps from zero moments
        if it == 0:
            th0 = a["theta_before"].astype(np.float64)
            mm = np.zeros_like(th0)
            vv = np.zeros_like(th0)
            O.adam(th0, a["grad"].astype(np.float64), mm, vv, 1, lr=1e-3)
            np.testing.assert_allclose(a["theta_after"], th0, rtol=1e-5, atol=1e-6)
    m.close()


def test_mlp_training_reduces_loss_and_predicts():
    X = synth.swissroll(n=6000, dim=32, n_clusters=10, seed=31)
    m = F.FuncSNE(X, 4, 16, 8, 8, 1.0, 10.0, seed=4)
    m.set_option("mlp_batch", 1024)
    m.step(200)
    first = m.mlp_debug_step()["loss"]
    m.mlp_train(300)
    last = m.stats()["mlp_loss"]
    assert last < 0.5 * first
    pred = m.mlp_predict(X[:500])
    Y = m.embedding()[:500]
    # the learned map explains most of the embedding's variance
    r2 = 1 - np.sum((pred - Y) ** 2) / np.sum((Y - Y.mean(0)) ** 2)
    assert r2 > 0.5
    m.close()
