"""ctypes wrapper of the FP64 CPU oracle (``funcsne_oracle.c``).

Test infrastructure only (see the package docstring). All state arrays are
numpy float64 / int32 arrays owned by :class:`OracleState`.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from .build import build_oracle

__all__ = ["lib", "set_threads", "threads", "philox", "OracleState", "bf16", "mlp_size", "mlp_init", "mlp_grad", "mlp_grad_mag", "mlp_stats", "mlp_inputs", "mlp_targets", "mlp_forward", "adam", "bisect", "entropy", "topk_merge", "ld_merge",
           "exact_z", "kl_divergence", "exact_grad", "bruteforce_knn", "query_knn",
           "ORACLE_BISECT_TOL", "ORACLE_BISECT_MAXIT", "STREAMS", "CAND_HD", "CAND_LD"]

ORACLE_BISECT_TOL = 1e-9
ORACLE_BISECT_MAXIT = 200
STREAMS = dict(COIN=0, REFINE=1, MLP=4, INSERT=5, INIT_HD=6, INIT_LD=7,
               INIT_Y=8, ZINIT=9)
CAND_HD = 32
CAND_LD = 32

_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build_oracle())
        _declare(_lib)
    return _lib


_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)
_lp = C.POINTER(C.c_int64)
_up = C.POINTER(C.c_uint32)
_bp = C.POINTER(C.c_uint8)


class _State(C.Structure):
    _fields_ = [("N", C.c_int64), ("D", C.c_int32), ("d", C.c_int32), ("k_hd", C.c_int32),
                ("k_ld", C.c_int32), ("n_neg", C.c_int32), ("alpha", C.c_double),
                ("perplexity", C.c_double), ("seed", C.c_uint64), ("lr", C.c_double),
                ("momentum", C.c_double), ("att_ratio", C.c_double), ("rep_ratio", C.c_double),
                ("exaggeration", C.c_double), ("exag_iters", C.c_int32), ("hd_mode", C.c_int32),
                ("neg_mode", C.c_int32), ("jump_iters", C.c_int32), ("jump_parts", C.c_int32),
                ("coin_floor", C.c_double), ("gamma_e", C.c_double), ("gamma_z", C.c_double),
                ("fresh_iters", C.c_int32), ("X", _dp), ("Y", _dp), ("V", _dp), ("hd_idx", _ip),
                ("hd_d2", _dp), ("ld_idx", _ip), ("beta", _dp), ("P", _dp), ("Zhat", C.c_double),
                ("E", C.c_double), ("t", C.c_uint32), ("fresh_lo", C.c_int64), ("fresh_until", C.c_uint32)]


def _declare(L):
    sp = C.POINTER(_State)
    L.oracle_set_threads.argtypes = [C.c_int]
    L.oracle_set_threads.restype = None
    L.oracle_threads.argtypes = []
    L.oracle_threads.restype = C.c_int
    L.oracle_philox4x32_10.argtypes = [_up, _up, _up]
    L.oracle_philox4x32_10.restype = None
    L.oracle_entropy.argtypes = [_dp, C.c_int, C.c_double, _dp]
    L.oracle_entropy.restype = C.c_double
    L.oracle_bisect.argtypes = [_dp, C.c_int, C.c_double, C.c_double, C.c_double, C.c_int, _dp, _dp]
    L.oracle_bisect.restype = C.c_int
    L.oracle_topk_merge.argtypes = [C.c_int64, C.c_int, _ip, _dp, C.c_int, _lp, _dp, _ip, _dp]
    L.oracle_topk_merge.restype = C.c_int
    L.oracle_ld_merge.argtypes = [C.c_int64, C.c_int, _ip, _dp, C.c_int, _lp, _dp]
    L.oracle_ld_merge.restype = C.c_int
    L.oracle_hd_candidates.argtypes = [sp, C.c_int64, _lp]
    L.oracle_hd_candidates.restype = None
    L.oracle_ld_candidates.argtypes = [sp, C.c_int64, _lp]
    L.oracle_ld_candidates.restype = None
    L.oracle_initial_list.argtypes = [C.c_uint64, C.c_int64, C.c_int64, C.c_int, C.c_uint32, _ip]
    L.oracle_initial_list.restype = None
    L.oracle_forces.argtypes = [sp, C.c_uint32, C.c_uint32, C.c_double, _dp, _dp, _dp]
    L.oracle_forces.restype = C.c_double
    L.oracle_init.argtypes = [sp, C.c_double, C.c_int]
    L.oracle_init.restype = None
    L.oracle_coin.argtypes = [sp]
    L.oracle_coin.restype = C.c_int
    L.oracle_step.argtypes = [sp, C.c_double, C.c_int, _dp, _dp, _bp, _lp, _dp]
    L.oracle_step.restype = None
    L.oracle_dense_p.argtypes = [sp, _dp]
    L.oracle_dense_p.restype = None
    L.oracle_exact_z.argtypes = [_dp, C.c_int64, C.c_int, C.c_double]
    L.oracle_exact_z.restype = C.c_double
    L.oracle_kl.argtypes = [_dp, _dp, C.c_int64, C.c_int, C.c_double]
    L.oracle_kl.restype = C.c_double
    L.oracle_exact_grad.argtypes = [_dp, _dp, C.c_int64, C.c_int, C.c_double, _dp]
    L.oracle_exact_grad.restype = None
    L.oracle_bruteforce_knn.argtypes = [_dp, C.c_int64, C.c_int, C.c_int, _ip, _dp]
    L.oracle_bruteforce_knn.restype = None
    L.oracle_query_knn.argtypes = [_dp, C.c_int64, C.c_int, _lp, C.c_int64, C.c_int, _ip, _dp]
    L.oracle_query_knn.restype = None
    L.oracle_insert.argtypes = [sp, C.c_int64, C.c_int, C.c_double, C.c_int]
    L.oracle_insert.restype = None
    L.oracle_scale.argtypes = [sp, C.c_double]
    L.oracle_scale.restype = None
    L.oracle_recalibrate.argtypes = [sp, C.c_double, C.c_int]
    L.oracle_recalibrate.restype = None
    L.oracle_remove.argtypes = [sp, _bp, C.c_double, C.c_int]
    L.oracle_remove.restype = C.c_int64
    L.oracle_forces_points.argtypes = [sp, C.c_uint32, C.c_uint32, C.c_double, _lp, C.c_int64, _dp, _dp]
    L.oracle_forces_points.restype = None
    L.oracle_bf16.argtypes = [C.c_double]
    L.oracle_bf16.restype = C.c_double
    L.oracle_mlp_init.argtypes = [C.c_int, C.c_int, C.c_int, C.c_uint64, _dp]
    L.oracle_mlp_init.restype = None
    L.oracle_mlp_grad.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, _dp, _dp, _dp, C.c_int, _dp, _dp]
    L.oracle_mlp_grad.restype = C.c_double
    L.oracle_mlp_grad_mag.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, _dp, _dp, _dp, _dp, _dp]
    L.oracle_mlp_grad_mag.restype = None
    L.oracle_mlp_stats.argtypes = [C.c_int64, C.c_int, _dp, _dp, _dp]
    L.oracle_mlp_stats.restype = None
    L.oracle_mlp_inputs.argtypes = [C.c_int, C.c_int, _dp, _lp, _dp, _dp, _dp]
    L.oracle_mlp_inputs.restype = None
    L.oracle_mlp_targets.argtypes = [C.c_int, C.c_int, _dp, _lp, _dp]
    L.oracle_mlp_targets.restype = C.c_double
    L.oracle_mlp_forward.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, _dp, _dp, C.c_int, _dp]
    L.oracle_mlp_forward.restype = None
    L.oracle_adam.argtypes = [C.c_int64, _dp, _dp, _dp, _dp, C.c_int, C.c_double, C.c_double, C.c_double,
                              C.c_double]
    L.oracle_adam.restype = None


def _p(a, t):
    return a.ctypes.data_as(t)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def set_threads(n):
    """Threads the oracle uses over points (its results do not depend on
    it); n <= 0 restores one per core."""
    lib().oracle_set_threads(int(n))


def threads():
    return int(lib().oracle_threads())


def philox(ctr, key):
    """Philox4x32-10 block: 4 counter words, 2 key words -> 4 output words."""
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    out = np.zeros(4, dtype=np.uint32)
    lib().oracle_philox4x32_10(_p(c, _up), _p(k, _up), _p(out, _up))
    return out


def entropy(d2, beta):
    d2 = _f64(d2)
    P = np.zeros_like(d2)
    h = lib().oracle_entropy(_p(d2, _dp), len(d2), float(beta), _p(P, _dp))
    return h, P


def bisect(d2, perplexity, beta0=0.0, tol=ORACLE_BISECT_TOL, maxit=ORACLE_BISECT_MAXIT):
    """Returns (beta, P, evaluations)."""
    d2 = _f64(d2)
    P = np.zeros_like(d2)
    b = C.c_double(0.0)
    it = lib().oracle_bisect(_p(d2, _dp), len(d2), float(perplexity), float(beta0), float(tol),
                             int(maxit), C.byref(b), _p(P, _dp))
    return b.value, P, it


def topk_merge(i, old_idx, old_d2, cand_idx, cand_d2):
    """Returns (new_idx, new_d2, changed)."""
    old_idx = np.ascontiguousarray(old_idx, dtype=np.int32)
    old_d2 = _f64(old_d2)
    cand_idx = np.ascontiguousarray(cand_idx, dtype=np.int64)
    cand_d2 = _f64(cand_d2)
    k = len(old_idx)
    ni = np.zeros(k, dtype=np.int32)
    nd = np.zeros(k, dtype=np.float64)
    ch = lib().oracle_topk_merge(int(i), k, _p(old_idx, _ip), _p(old_d2, _dp), len(cand_idx),
                                 _p(cand_idx, _lp), _p(cand_d2, _dp), _p(ni, _ip), _p(nd, _dp))
    return ni, nd, bool(ch)


def ld_merge(i, old_idx, old_d2, cand_idx, cand_d2):
    """The LD list's merge: old entries and new candidates ordered by
    (d2, idx), first k kept, also when nothing entered. Returns
    (new_idx, new_d2, changed)."""
    ni = np.array(old_idx, dtype=np.int32)
    nd = np.array(old_d2, dtype=np.float64)
    cand_idx = np.ascontiguousarray(cand_idx, dtype=np.int64)
    cand_d2 = _f64(cand_d2)
    ch = lib().oracle_ld_merge(int(i), len(ni), _p(ni, _ip), _p(nd, _dp), len(cand_idx), _p(cand_idx, _lp),
                               _p(cand_d2, _dp))
    return ni, nd, bool(ch)


def exact_z(Y, alpha):
    Y = _f64(Y)
    return lib().oracle_exact_z(_p(Y, _dp), Y.shape[0], Y.shape[1], float(alpha))


def kl_divergence(Pd, Y, alpha):
    Pd = _f64(Pd)
    Y = _f64(Y)
    return lib().oracle_kl(_p(Pd, _dp), _p(Y, _dp), Y.shape[0], Y.shape[1], float(alpha))


def exact_grad(Pd, Y, alpha):
    Pd = _f64(Pd)
    Y = _f64(Y)
    G = np.zeros_like(Y)
    lib().oracle_exact_grad(_p(Pd, _dp), _p(Y, _dp), Y.shape[0], Y.shape[1], float(alpha),
                            _p(G, _dp))
    return G


def bruteforce_knn(X, k):
    X = _f64(X)
    N = X.shape[0]
    idx = np.zeros((N, k), dtype=np.int32)
    d2 = np.zeros((N, k), dtype=np.float64)
    lib().oracle_bruteforce_knn(_p(X, _dp), N, X.shape[1], k, _p(idx, _ip), _p(d2, _dp))
    return idx, d2


def query_knn(X, queries, k):
    X = _f64(X)
    q = np.ascontiguousarray(queries, dtype=np.int64)
    idx = np.zeros((len(q), k), dtype=np.int32)
    d2 = np.zeros((len(q), k), dtype=np.float64)
    lib().oracle_query_knn(_p(X, _dp), X.shape[0], X.shape[1], _p(q, _lp), len(q), k,
                           _p(idx, _ip), _p(d2, _dp))
    return idx, d2


def bf16(x):
    """Round to bfloat16 (nearest even) through binary32, elementwise."""
    x = np.asarray(x, dtype=np.float64)
    f = x.astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    fin = (u & 0x7F800000) != 0x7F800000
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    out = np.where(fin, r.view(np.float32), f).astype(np.float64)
    return out


def mlp_size(D, H, d):
    return H * D + H + H * H + H + d * H + d


def mlp_init(D, H, d, seed):
    th = np.zeros(mlp_size(D, H, d))
    lib().oracle_mlp_init(D, H, d, seed, _p(th, _dp))
    return th


def mlp_grad(theta, X, T, H, round_bf16=True):
    """(loss, flat gradient, outputs) of one batch."""
    theta, X, T = _f64(theta), _f64(X), _f64(T)
    B, D = X.shape
    d = T.shape[1]
    g = np.zeros_like(theta)
    O = np.zeros((B, d))
    loss = lib().oracle_mlp_grad(B, D, H, d, _p(theta, _dp), _p(X, _dp), _p(T, _dp), int(round_bf16),
                                 _p(g, _dp), _p(O, _dp))
    return loss, g, O


def mlp_grad_mag(theta, X, T, H):
    """(gradient magnitudes, output magnitudes) of one batch: the sums of the
    magnitudes of the terms behind each gradient element and output of the
    rounded network (oracle_mlp_grad_mag)."""
    theta, X, T = _f64(theta), _f64(X), _f64(T)
    B, D = X.shape
    d = T.shape[1]
    g = np.zeros_like(theta)
    O = np.zeros((B, d))
    lib().oracle_mlp_grad_mag(B, D, H, d, _p(theta, _dp), _p(X, _dp), _p(T, _dp), _p(g, _dp), _p(O, _dp))
    return g, O


def mlp_stats(X):
    """Per-feature mean and population std (1 for constant features)."""
    X = _f64(X)
    N, D = X.shape
    mean, std = np.zeros(D), np.zeros(D)
    lib().oracle_mlp_stats(N, D, _p(X, _dp), _p(mean, _dp), _p(std, _dp))
    return mean, std


def mlp_inputs(X, idx, mean, std):
    """bfloat16 of (x - mean) / std for the rows idx, in binary32 arithmetic."""
    X = _f64(X)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    out = np.zeros((len(idx), X.shape[1]))
    lib().oracle_mlp_inputs(len(idx), X.shape[1], _p(X, _dp), _p(idx, _lp), _p(_f64(mean), _dp),
                            _p(_f64(std), _dp), _p(out, _dp))
    return out


def mlp_targets(Y, idx):
    """(y / s for the rows idx, s = RMS of those values)."""
    Y = _f64(Y)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    out = np.zeros((len(idx), Y.shape[1]))
    sc = lib().oracle_mlp_targets(len(idx), Y.shape[1], _p(Y, _dp), _p(idx, _lp), _p(out, _dp))
    return out, sc


def mlp_forward(theta, X, H, d, round_bf16=True):
    theta, X = _f64(theta), _f64(X)
    B, D = X.shape
    O = np.zeros((B, d))
    lib().oracle_mlp_forward(B, D, H, d, _p(theta, _dp), _p(X, _dp), int(round_bf16), _p(O, _dp))
    return O


def adam(theta, g, m, v, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """In-place Adam step on float64 arrays."""
    lib().oracle_adam(len(theta), _p(theta, _dp), _p(_f64(g), _dp), _p(m, _dp), _p(v, _dp), int(step),
                      float(lr), float(b1), float(b2), float(eps))


class OracleState:
    """The method's state held in FP64 numpy arrays, stepped by the C oracle."""

    def __init__(self, X, d, k_hd, k_ld, n_neg, alpha, perplexity, seed=0, lr=None,
                 momentum=0.8, att_ratio=1.0, rep_ratio=1.0, exaggeration=1.0, exag_iters=0,
                 hd_mode=0, neg_mode=0, jump_iters=0, jump_parts=2, coin_floor=0.05, gamma_e=0.1,
                 gamma_z=0.1, fresh_iters=0, init=True):
        self.X = _f64(X)
        N, D = self.X.shape
        self.N, self.D = N, D
        self.Y = np.zeros((N, d))
        self.V = np.zeros((N, d))
        self.hd_idx = np.zeros((N, k_hd), dtype=np.int32)
        self.hd_d2 = np.zeros((N, k_hd))
        self.ld_idx = np.zeros((N, k_ld), dtype=np.int32)
        self.beta = np.zeros(N)
        self.P = np.zeros((N, k_hd))
        if lr is None:
            lr = max(N / 12.0, 200.0)
        s = _State()
        s.N, s.D, s.d, s.k_hd, s.k_ld, s.n_neg = N, D, d, k_hd, k_ld, n_neg
        s.alpha, s.perplexity, s.seed = alpha, perplexity, seed
        s.lr, s.momentum, s.att_ratio, s.rep_ratio = lr, momentum, att_ratio, rep_ratio
        s.exaggeration, s.exag_iters, s.hd_mode, s.neg_mode = exaggeration, exag_iters, hd_mode, neg_mode
        s.jump_iters, s.jump_parts = jump_iters, jump_parts
        s.coin_floor, s.gamma_e, s.gamma_z = coin_floor, gamma_e, gamma_z
        s.fresh_iters, s.fresh_lo, s.fresh_until = fresh_iters, N, 0
        self._s = s
        self._bind()
        if init:
            lib().oracle_init(C.byref(s), ORACLE_BISECT_TOL, ORACLE_BISECT_MAXIT)

    def _bind(self):
        s = self._s
        s.X = _p(self.X, _dp)
        s.Y = _p(self.Y, _dp)
        s.V = _p(self.V, _dp)
        s.hd_idx = _p(self.hd_idx, _ip)
        s.hd_d2 = _p(self.hd_d2, _dp)
        s.ld_idx = _p(self.ld_idx, _ip)
        s.beta = _p(self.beta, _dp)
        s.P = _p(self.P, _dp)

    # scalar state and options
    def __getattr__(self, name):
        if name in ("Zhat", "E", "t", "lr", "momentum", "att_ratio", "rep_ratio", "exaggeration",
                    "exag_iters", "hd_mode", "neg_mode", "jump_iters", "jump_parts", "coin_floor", "gamma_e",
                    "gamma_z", "fresh_iters", "fresh_lo", "fresh_until", "alpha", "perplexity", "seed", "n_neg",
                    "k_hd", "k_ld", "d"):
            return getattr(self.__dict__["_s"], name)
        raise AttributeError(name)

    def set(self, **kw):
        for k, v in kw.items():
            setattr(self._s, k, v)

    def load(self, Y=None, V=None, hd_idx=None, ld_idx=None, beta=None, P=None, Zhat=None,
             E=None, t=None, d2=True, fresh_lo=None, fresh_until=None):
        """Overwrite parts of the state (for example with the GPU's exported state).
        HD distances are recomputed in FP64 from X (unless d2 is False: a
        state that will only give forces, which do not read them); the list
        order is kept."""
        if Y is not None:
            self.Y[...] = Y
        if V is not None:
            self.V[...] = V
        if hd_idx is not None:
            self.hd_idx[...] = hd_idx
        if ld_idx is not None:
            self.ld_idx[...] = ld_idx
        if beta is not None:
            self.beta[...] = beta
        if P is not None:
            self.P[...] = P
        if Zhat is not None:
            self._s.Zhat = Zhat
        if E is not None:
            self._s.E = E
        if t is not None:
            self._s.t = t
        if fresh_lo is not None:
            self._s.fresh_lo = fresh_lo
        if fresh_until is not None:
            self._s.fresh_until = fresh_until
        if not d2:
            return
        step = max(1, (1 << 24) // max(1, self.hd_idx.shape[1] * self.D))  # at most 128 MB a chunk
        for a in range(0, self.N, step):
            diff = self.X[a:a + step, None, :] - self.X[self.hd_idx[a:a + step]]
            self.hd_d2[a:a + step] = np.einsum("nkd,nkd->nk", diff, diff)

    def coin(self):
        return bool(lib().oracle_coin(C.byref(self._s)))

    def hd_candidates(self, i):
        out = np.zeros(CAND_HD, dtype=np.int64)
        lib().oracle_hd_candidates(C.byref(self._s), int(i), _p(out, _lp))
        return out

    def ld_candidates(self, i):
        out = np.zeros(CAND_LD, dtype=np.int64)
        lib().oracle_ld_candidates(C.byref(self._s), int(i), _p(out, _lp))
        return out

    def forces(self, zhat=None, t=None, stream=STREAMS["REFINE"]):
        """Returns (A, R, Z_t, z per point) for the current lists, P and Y."""
        A = np.zeros_like(self.Y)
        R = np.zeros_like(self.Y)
        z = np.zeros(self.N)
        zt = lib().oracle_forces(C.byref(self._s), self._s.t if t is None else t, stream,
                                 self._s.Zhat if zhat is None else zhat, _p(A, _dp), _p(R, _dp),
                                 _p(z, _dp))
        return A, R, zt, z

    def forces_points(self, pts, zhat=None, t=None, stream=STREAMS["REFINE"]):
        """(A, R) rows of the points pts only (for a sample of a large state)."""
        pts = np.ascontiguousarray(pts, dtype=np.int64)
        A = np.zeros((len(pts), self.d))
        R = np.zeros((len(pts), self.d))
        lib().oracle_forces_points(C.byref(self._s), self._s.t if t is None else t, stream,
                                   self._s.Zhat if zhat is None else zhat, _p(pts, _lp), len(pts),
                                   _p(A, _dp), _p(R, _dp))
        return A, R

    def step(self, tol=ORACLE_BISECT_TOL, maxit=ORACLE_BISECT_MAXIT):
        """One iteration. Returns dict(A, R, flags, coin, n_new, z)."""
        A = np.zeros_like(self.Y)
        R = np.zeros_like(self.Y)
        flags = np.zeros(self.N, dtype=np.uint8)
        info = np.zeros(2, dtype=np.int64)
        z = np.zeros(self.N)
        lib().oracle_step(C.byref(self._s), float(tol), int(maxit), _p(A, _dp), _p(R, _dp),
                          _p(flags, _bp), _p(info, _lp), _p(z, _dp))
        return dict(A=A, R=R, flags=flags, coin=bool(info[0]), n_new=int(info[1]), z=z)

    def insert(self, X_new, rounds=64, tol=ORACLE_BISECT_TOL, maxit=ORACLE_BISECT_MAXIT):
        """Append the rows of X_new (mean placement) after `rounds`
        neighbour-of-neighbour rounds. Returns the first new index."""
        X_new = _f64(X_new)
        n_old, n_new = self.N, X_new.shape[0]
        N = n_old + n_new

        def grow(a, fill=0):
            out = np.full((N,) + a.shape[1:], fill, dtype=a.dtype)
            out[:n_old] = a
            return out
        self.X = np.concatenate([self.X, X_new], axis=0)
        self.Y, self.V = grow(self.Y), grow(self.V)
        self.hd_idx, self.hd_d2, self.ld_idx = grow(self.hd_idx), grow(self.hd_d2), grow(self.ld_idx)
        self.beta, self.P = grow(self.beta), grow(self.P)
        self.N = N
        self._s.N = N
        self._bind()
        lib().oracle_insert(C.byref(self._s), n_old, int(rounds), float(tol), int(maxit))
        return n_old

    def scale(self, factor):
        """Scale Y and V by factor and re-estimate Zhat (the implosion)."""
        lib().oracle_scale(C.byref(self._s), float(factor))

    def set_perplexity(self, perplexity, tol=ORACLE_BISECT_TOL, maxit=ORACLE_BISECT_MAXIT):
        """Change the perplexity and recalibrate every point from its list."""
        self._s.perplexity = float(perplexity)
        lib().oracle_recalibrate(C.byref(self._s), float(tol), int(maxit))

    def update_rows(self, ids, X_rows, tol=ORACLE_BISECT_TOL, maxit=ORACLE_BISECT_MAXIT):
        """Replace rows of X (drift), then recalibrate every point."""
        self.X[np.asarray(ids, dtype=np.int64)] = _f64(X_rows)
        lib().oracle_recalibrate(C.byref(self._s), float(tol), int(maxit))

    def remove(self, ids, tol=ORACLE_BISECT_TOL, maxit=ORACLE_BISECT_MAXIT):
        """Remove the points `ids`; the kept points are renumbered in order.
        Returns the number of points left."""
        removed = np.zeros(self.N, dtype=np.uint8)
        removed[np.asarray(ids, dtype=np.int64)] = 1
        keep = removed == 0
        self.X = np.ascontiguousarray(self.X[keep])
        self._bind()
        n = lib().oracle_remove(C.byref(self._s), _p(removed, _bp), float(tol), int(maxit))
        for name in ("Y", "V", "hd_idx", "hd_d2", "ld_idx", "beta", "P"):
            setattr(self, name, np.ascontiguousarray(getattr(self, name)[:n]))
        self.N = int(n)
        self._s.N = int(n)
        self._bind()
        return int(n)

    def dense_p(self):
        Pd = np.zeros((self.N, self.N))
        lib().oracle_dense_p(C.byref(self._s), _p(Pd, _dp))
        return Pd

    def initial_list(self, i, k, stream):
        out = np.zeros(k, dtype=np.int32)
        lib().oracle_initial_list(self._s.seed, self.N, int(i), int(k), int(stream), _p(out, _ip))
        return out

    def copy(self):
        o = OracleState.__new__(OracleState)
        o.__dict__.update({k: (v.copy() if isinstance(v, np.ndarray) else v)
                           for k, v in self.__dict__.items() if k != "_s"})
        o._s = _State.from_buffer_copy(self._s)
        o._bind()
        return o
