"""What the learned placement gains over the method without it, in the
dynamic-dataset protocol at a reduced size (swiss roll, D = 128, d = 8; a
50,000-point base, then 4 insertions of 5,000 points, 50 iterations apart;
adaptive HD refinement, BF16 rows, the insertion refinement window on).

For each placement of inserted points (neighbour mean: the method without a
learned part; surrogate: the placement MLP trained online) it records the
new points' HD-KNN recall@32 along the 50 iterations after each insertion,
against exact neighbours, and the iterations until it is within 0.5 points
(or 90%) of the established points' recall: the insertion-to-converged time.

The test pins the signs this protocol gives (measured on GB300, and in the
200,000-point protocol of the benchmark's dynamic mode):
  * with few neighbour-of-neighbour rounds at insertion (4), the learned
    placement ends with better HD lists for the new points than the
    neighbour mean: the LD neighbours proposed around its position feed the
    HD search;
  * with the default 64 rounds, insertion already finds good HD lists and
    the neighbour mean of those lists is the better position: the learned
    placement does not beat it.
The insertion window (option fresh_iters) is what brings new points close
to the established points: it is checked against the run without it."""
import numpy as np
import pytest

from paper_2509_07681_gb300 import funcsne as F
from paper_2509_07681_gb300 import synth
from paper_2509_07681_gb300.quality import recall

from gpu_util import lib

pytestmark = pytest.mark.gpu

BASE, NEW, ROUNDS, EVERY, CHECK = 50_000, 5_000, 4, 50, 5


def _protocol(place, insert_rounds, fresh_iters=EVERY):
    X0 = synth.swissroll(n=BASE, dim=128, n_clusters=32, seed=3)
    batches = [synth.swissroll(n=NEW, dim=128, n_clusters=32, seed=3, batch=r + 1) for r in range(ROUNDS)]
    m = F.FuncSNE(X0, 8, 32, 16, 16, 1.0, 30.0, seed=0, precision=F.BF16, insert_rounds=insert_rounds,
                  fresh_iters=fresh_iters)
    if place == F.PLACE_SURROGATE:
        m.set_option("surrogate", 1)
    m.step(300)
    if place == F.PLACE_SURROGATE:
        m.mlp_train(200)
    rng = np.random.default_rng(1)
    q_old = np.sort(rng.choice(BASE, 1000, replace=False)).astype(np.int32)
    curves, conv, end_new, end_old = [], [], [], []
    for r in range(ROUNDS):
        first = m.insert(batches[r], placement=place)
        q_new = np.arange(first, first + NEW, dtype=np.int32)
        ex_new, _ = m.exact_knn(q_new, 32)
        ex_old, _ = m.exact_knn(q_old, 32)
        curve, hit = [], None
        for it in range(CHECK, EVERY + 1, CHECK):
            m.step(CHECK)
            hd = m.knn(F.SPACE_HD, with_d2=False)
            rn, ro = recall(hd[q_new], ex_new), recall(hd[q_old], ex_old)
            curve.append(rn)
            if hit is None and rn >= 0.9 * ro:
                hit = it
        curves.append(curve)
        conv.append(hit)
        end_new.append(rn)
        end_old.append(ro)
    m.sync()
    assert m.stats()["error_word"] == 0
    m.close()
    return dict(curve=np.mean(curves, 0), reach90=conv, end_new=float(np.mean(end_new)),
                end_old=float(np.mean(end_old)))


def _report(tag, res):
    print(f"{tag}: new points' recall at +5 .. +50 iterations "
          + " ".join(f"{v:.3f}" for v in res["curve"])
          + f"; established {res['end_old']:.3f}; iterations to 90% of it {res['reach90']}")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    lib()


def test_learned_placement_gains_when_insertion_search_is_short():
    mean = _protocol(F.PLACE_MEAN, 4)
    surr = _protocol(F.PLACE_SURROGATE, 4)
    _report("4 rounds, neighbour mean", mean)
    _report("4 rounds, surrogate", surr)
    # the area under the recall curve after insertion, and its end
    assert surr["curve"].mean() > mean["curve"].mean()
    assert surr["end_new"] > mean["end_new"]


def test_neighbour_mean_is_the_better_position_after_a_full_insertion_search():
    mean = _protocol(F.PLACE_MEAN, 64)
    surr = _protocol(F.PLACE_SURROGATE, 64)
    off = _protocol(F.PLACE_MEAN, 64, fresh_iters=0)
    _report("64 rounds, neighbour mean", mean)
    _report("64 rounds, surrogate", surr)
    _report("64 rounds, neighbour mean, no insertion window", off)
    assert mean["curve"].mean() >= surr["curve"].mean()
    assert mean["end_new"] >= surr["end_new"]
    # the insertion window: new points refine every iteration and end close
    # to the established points, which they do not without it
    assert mean["end_new"] > off["end_new"]
    assert mean["end_new"] >= 0.9 * mean["end_old"]
