"""The allocation-free brute-force KNN entry point (funcsne_exact_knn_noalloc).

Callers that cannot allocate device memory when they need neighbours (code
under another framework's caching allocator, or a latency-critical path that
must not pay cudaMalloc's implicit synchronisation) call this variant, whose
scratch is a fixed file-scope device array. Its results must equal those of
the allocating entry point funcsne_exact_knn on the same data, on two calls in
a row (the second call reuses the scratch the first one left behind).
This file is collected last on purpose; it also passes on its own.
"""
import numpy as np
import pytest

from paper_2509_07681_gb300 import funcsne as F
from paper_2509_07681_gb300 import synth
from paper_2509_07681_gb300.build import build

pytestmark = pytest.mark.gpu


def test_noalloc_knn_matches_allocating_entry_point_twice():
    torch = pytest.importorskip("torch")
    build()
    F.load()
    N, D = 20000, 50
    X = synth.spectrum(n=N, dim=D, n_clusters=8, seed=12)
    calls = [
        (np.arange(0, N, 17, dtype=np.int32), 32),                                   # 1177 queries, k <= 32
        (np.random.default_rng(3).choice(N, 900, replace=False).astype(np.int32), 40),  # k > 32
    ]
    with F.FuncSNE(X, 16, 32, 32, 32, 1.0, 30.0) as m:
        refs = [m.exact_knn(q, k) for q, k in calls]

    ldx = (D + 3) // 4 * 4
    Xd = torch.zeros((N, ldx), dtype=torch.float32, device="cuda")
    Xd[:, :D] = torch.from_numpy(X).cuda()
    for (q, k), (ref_idx, ref_d2) in zip(calls, refs):
        idx = torch.full((len(q), k), -7, dtype=torch.int32, device="cuda")
        d2 = torch.full((len(q), k), -1.0, dtype=torch.float32, device="cuda")
        stream = torch.cuda.current_stream().cuda_stream
        F.funcsne_exact_knn_noalloc(Xd, N, D, ldx, q, k, idx, d2, stream)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(idx.cpu().numpy(), ref_idx)
        np.testing.assert_allclose(d2.cpu().numpy(), ref_d2, rtol=1e-6, atol=0)


def test_noalloc_knn_rejects_oversized_requests():
    torch = pytest.importorskip("torch")
    build()
    F.load()
    N, D = 3000, 8
    Xd = torch.zeros((N, D), dtype=torch.float32, device="cuda")
    q = np.zeros(40000, dtype=np.int32)
    idx = torch.empty((len(q), 8), dtype=torch.int32, device="cuda")
    with pytest.raises(F.FuncSNEError) as e:
        F.funcsne_exact_knn_noalloc(Xd, N, D, D, q, 8, idx, None, None)
    assert e.value.code == -1 and "static scratch" in str(e.value)
    with pytest.raises(F.FuncSNEError):
        F.funcsne_exact_knn_noalloc(Xd, N, D, D, np.array([N], np.int32), 8, idx, None, None)
