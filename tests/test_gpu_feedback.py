"""The feedback loop of Section 3 (Fig. 4): the HD neighbour search draws
candidates from the LD neighbour lists, so an embedding optimised by the
gradients makes the HD lists converge faster than an embedding held at its
random-projection start. Measured with the paper's quality measure, the
AUC of R_NX(K) of the estimated HD lists against exact neighbours
(K = 1 .. k_hd), on MNIST-shaped pixel rows (20,000 points, D = 784, d = 2
and d = 8, HD refinement every iteration, 1,000 sampled points)."""
import numpy as np
import pytest

from paper_2509_07681_gb300 import funcsne as F
from paper_2509_07681_gb300 import synth
from paper_2509_07681_gb300.quality import rnx_auc

from gpu_util import lib

pytestmark = pytest.mark.gpu

CHECKS = (50, 200, 400, 800)


def _curve(X, d, fixed, q, exact):
    m = F.FuncSNE(X, d, 32, 16, 16, 1.0, 30.0, seed=0, hd_mode=1)
    if fixed:
        m.set_option("lr", 1e-12)
    out, done = [], 0
    for c in CHECKS:
        m.step(c - done)
        done = c
        out.append(rnx_auc(m.knn(F.SPACE_HD, with_d2=False)[q], exact, len(X)))
    m.sync()
    m.close()
    return np.array(out)


@pytest.mark.parametrize("d", [2, 8])
def test_optimised_embedding_speeds_up_the_hd_search(d):
    lib()
    X = synth.pixels(n=20000, dim=784, seed=12)
    q = np.sort(np.random.default_rng(0).choice(len(X), 1000, replace=False)).astype(np.int32)
    with F.FuncSNE(X, d, 32, 16, 16, 1.0, 30.0, seed=0) as m:
        exact, _ = m.exact_knn(q, 32)
    opt = _curve(X, d, False, q, exact)
    fix = _curve(X, d, True, q, exact)
    print(f"d={d}: AUC of R_NX at {CHECKS} iterations: optimised " + " ".join(f"{v:.4f}" for v in opt)
          + ", fixed " + " ".join(f"{v:.4f}" for v in fix))
    # late in the run the optimised embedding proposes the better candidates
    assert opt[-1] > fix[-1]
