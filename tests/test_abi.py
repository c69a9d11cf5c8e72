"""Host-side checks of the C ABI (no GPU needed): the library builds for
sm_103a, loads, exports every entry point include/funcsne.h declares, and
rejects invalid arguments before touching the device."""
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2509_07681_gb300 import funcsne as F
from paper_2509_07681_gb300.build import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "funcsne.h")


@pytest.fixture(scope="module")
def lib():
    build()
    return F.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(funcsne_[a-z_]+)\s*\(", src)))


def test_header_lists_the_entry_points():
    names = declared_functions()
    assert {"funcsne_create", "funcsne_step", "funcsne_insert", "funcsne_get_embedding",
            "funcsne_destroy"} <= set(names)
    assert set(names) == set(F.ABI_FUNCTIONS), "binding and header disagree"


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", F.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s+(funcsne_\w+)", out))
    missing = set(declared_functions()) - exported
    assert not missing, f"not exported: {missing}"
    for name in declared_functions():
        assert hasattr(lib, name)


@pytest.mark.parametrize("kw,frag", [
    (dict(d=0), "d must be"),
    (dict(d=33), "d must be"),
    (dict(k_hd=1), "k_hd must be"),
    (dict(k_hd=65), "k_hd must be"),
    (dict(k_ld=0), "k_ld must be"),
    (dict(n_neg=0), "n_neg must be"),
    (dict(alpha=0.0), "alpha"),
    (dict(perplexity=1.0), "perplexity"),
    (dict(perplexity=40.0), "perplexity"),
    (dict(N=16), "N must exceed"),
])
def test_create_rejects_bad_arguments(lib, kw, frag):
    args = dict(N=100, D=5, d=2, k_hd=16, k_ld=8, n_neg=4, alpha=1.0, perplexity=5.0)
    args.update(kw)
    X = np.zeros((args["N"], args["D"]), dtype=np.float32)
    h = F._h()
    rc = lib.funcsne_create(X.ctypes.data, args["N"], args["D"], args["d"], args["k_hd"], args["k_ld"],
                            args["n_neg"], args["alpha"], args["perplexity"], 0, h)
    assert rc == -1
    assert frag in F.funcsne_last_error(None)
    assert not h.value


def test_null_handle_calls_fail_cleanly(lib):
    assert lib.funcsne_step(None, 1) == -1
    assert lib.funcsne_sync(None) == -1
    assert lib.funcsne_set_option(None, b"lr", 1.0) == -1
    ids = np.zeros(2, dtype=np.int64)
    rows = np.zeros((2, 5), dtype=np.float32)
    assert lib.funcsne_remove(None, ids.ctypes.data, 2) == -1
    assert lib.funcsne_update_points(None, ids.ctypes.data, 2, rows.ctypes.data) == -1
    assert lib.funcsne_get_data(None, rows.ctypes.data, 2) == -1
    assert lib.funcsne_get_embedding_async(None, rows.ctypes.data, 2) == -1
    assert lib.funcsne_wait_embedding(None) == -1
    assert lib.funcsne_debug_bounded_wait(None, 10) == -1
    lib.funcsne_destroy(None)


def test_noalloc_knn_rejects_huge_query_counts_before_touching_memory(lib):
    """n_q is bounded before any byte count is formed from it, so a count
    whose products would wrap around 64 bits is rejected (no device call,
    the 4-entry query buffer is never read past)."""
    X = np.zeros((64, 4), dtype=np.float32)
    q = np.zeros(4, dtype=np.int32)
    idx = np.zeros((4, 8), dtype=np.int32)
    for n_q in (2 ** 61, 2 ** 40, (4 << 20) // 4 + 1):
        rc = lib.funcsne_exact_knn_noalloc(X.ctypes.data, 64, 4, 4, q.ctypes.data, n_q, 8, idx.ctypes.data, None,
                                           None)
        assert rc == -1
        assert "static scratch" in F.funcsne_last_error(None)


def test_header_compiles_as_c_and_cxx():
    """The boundary is a plain C header: it compiles as C99 and as C++."""
    import shutil
    hdr = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "funcsne.h")
    for cc, lang, std in (("gcc", "c", "-std=c99"), ("g++", "c++", "-std=c++17")):
        if shutil.which(cc) is None:
            pytest.skip(f"{cc} not found")
        r = subprocess.run([cc, "-fsyntax-only", "-Wall", "-Werror", "-x", lang, std, hdr], capture_output=True,
                           text=True)
        assert r.returncode == 0, r.stderr
