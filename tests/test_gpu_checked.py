"""The range-checked build (libfuncsne_checked.so, compiled with
-DFUNCSNE_CHECKED): the iteration kernels check every point index they read
from memory before addressing a row or a list with it, and report a bad one
through the device error word instead of trapping. The small parity cases
(one iteration against the oracle, insertion with its refinement window)
run under it in a child process that selects it with FUNCSNE_LIBRARY; a
check that fired would make funcsne_sync fail with FUNCSNE_E_RANGE."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_SCRIPT = r"""
import os, sys
root = os.environ["FUNCSNE_ROOT"]
sys.path[:0] = [root, os.path.join(root, "tests")]
from paper_2509_07681_gb300 import funcsne as F
from paper_2509_07681_gb300 import synth
lib = F.load()
assert os.path.basename(lib._name) == "libfuncsne_checked.so", lib._name
import test_gpu_parity as T
for case in ("ragged", "spectrum-shape", "k64-d32", "pixels-shape", "kld-gt-khd"):
    T.test_one_iteration_matches_oracle(case)
T.test_insertion_window_matches_oracle(0)
X = synth.spectrum(n=6000, dim=50, n_clusters=12, seed=21)
for prec in (F.FP32, F.BF16, F.FP8):
    m = F.FuncSNE(X[:5000], 16, 32, 32, 32, 1.0, 30.0, seed=0, precision=prec, fresh_iters=10)
    m.step(30)
    m.insert(X[5000:])
    m.step(30)
    m.sync()
    assert m.stats()["error_word"] == 0
    m.close()
print("CHECKED_OK")
"""


def test_parity_cases_under_the_range_checked_build():
    from paper_2509_07681_gb300.build import build
    path = build(checked=True)
    env = dict(os.environ, FUNCSNE_LIBRARY=path, FUNCSNE_ROOT=ROOT)
    r = subprocess.run([sys.executable, "-c", _SCRIPT], env=env, capture_output=True, text=True, timeout=1200,
                       cwd=ROOT)
    assert r.returncode == 0 and "CHECKED_OK" in r.stdout, (r.stdout[-2000:], r.stderr[-4000:])
