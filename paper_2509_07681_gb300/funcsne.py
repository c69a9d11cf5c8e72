"""Thin Python binding of the C ABI in include/funcsne.h (argument marshalling
only: every step of the method runs in the CUDA kernels of libfuncsne.so).

The module-level functions carry the C names and signatures; ``FuncSNE`` is a
small convenience wrapper around a handle. Arrays may be numpy arrays (host
memory) or torch tensors (host or CUDA memory); the library detects which.
Loading fails loudly when the compiled library is missing: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

__all__ = ["load", "FuncSNEError", "FuncSNE", "FP32", "BF16", "FP8", "SPACE_HD", "SPACE_LD",
           "PLACE_MEAN", "PLACE_SURROGATE", "State", "Stats", "MlpDebug", "ABI_FUNCTIONS"]

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfuncsne.so")

FP32, BF16, FP8 = 0, 1, 2
SPACE_HD, SPACE_LD = 0, 1
PLACE_MEAN, PLACE_SURROGATE = 0, 1
ERRORS = {0: "OK", -1: "FUNCSNE_E_ARG", -2: "FUNCSNE_E_OOM", -3: "FUNCSNE_E_CUDA",
          -4: "FUNCSNE_E_NAN", -5: "FUNCSNE_E_RANGE", -6: "FUNCSNE_E_STATE"}


class FuncSNEError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class State(C.Structure):
    _fields_ = [("Y", C.c_void_p), ("V", C.c_void_p), ("hd_idx", C.c_void_p), ("hd_d2", C.c_void_p),
                ("ld_idx", C.c_void_p), ("beta", C.c_void_p), ("P", C.c_void_p), ("Zhat", C.c_double),
                ("E", C.c_double), ("t", C.c_uint32), ("fresh_lo", C.c_int64), ("fresh_until", C.c_uint32)]


class Stats(C.Structure):
    _fields_ = [("N", C.c_int64), ("t", C.c_uint32), ("E", C.c_double), ("Zhat", C.c_double),
                ("last_Z", C.c_double), ("last_n_new", C.c_int64), ("last_coin", C.c_int32),
                ("precision", C.c_int32), ("error_word", C.c_uint32), ("cand_scored", C.c_int64),
                ("cand_reranked", C.c_int64), ("mlp_steps", C.c_int64), ("mlp_loss", C.c_double),
                ("n_refined", C.c_int64)]


class MlpDebug(C.Structure):
    _fields_ = [("batch_idx", C.c_void_p), ("xhat", C.c_void_p), ("target", C.c_void_p), ("output", C.c_void_p),
                ("theta_before", C.c_void_p), ("weights_bf16", C.c_void_p), ("grad", C.c_void_p),
                ("theta_after", C.c_void_p), ("loss", C.c_double), ("scale", C.c_float), ("step", C.c_int32),
                ("n_params", C.c_int64)]


_h = C.c_void_p
_vp = C.c_void_p
ABI_FUNCTIONS = {
    "funcsne_create": (C.c_int, [_vp, C.c_int64, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                 C.c_float, C.c_float, C.c_uint64, C.POINTER(_h)]),
    "funcsne_set_option": (C.c_int, [_h, C.c_char_p, C.c_double]),
    "funcsne_get_option": (C.c_int, [_h, C.c_char_p, C.POINTER(C.c_double)]),
    "funcsne_set_stream": (C.c_int, [_h, _vp]),
    "funcsne_step": (C.c_int, [_h, C.c_int32]),
    "funcsne_sync": (C.c_int, [_h]),
    "funcsne_insert": (C.c_int, [_h, _vp, C.c_int64, C.c_int32, C.POINTER(C.c_int64)]),
    "funcsne_update_points": (C.c_int, [_h, _vp, C.c_int64, _vp]),
    "funcsne_remove": (C.c_int, [_h, _vp, C.c_int64]),
    "funcsne_get_embedding": (C.c_int, [_h, _vp, C.c_int64]),
    "funcsne_get_embedding_async": (C.c_int, [_h, _vp, C.c_int64]),
    "funcsne_debug_bounded_wait": (C.c_int, [_h, C.c_uint32]),
    "funcsne_debug_fail_alloc": (C.c_int, [C.c_int64]),
    "funcsne_debug_row_bounds": (C.c_int, [_h, _vp, C.c_int64]),
    "funcsne_wait_embedding": (C.c_int, [_h]),
    "funcsne_get_data": (C.c_int, [_h, _vp, C.c_int64]),
    "funcsne_scale_embedding": (C.c_int, [_h, C.c_float]),
    "funcsne_get_knn": (C.c_int, [_h, C.c_int32, _vp, _vp]),
    "funcsne_get_stats": (C.c_int, [_h, C.POINTER(Stats)]),
    "funcsne_export_state": (C.c_int, [_h, C.POINTER(State)]),
    "funcsne_import_state": (C.c_int, [_h, C.POINTER(State)]),
    "funcsne_debug_step": (C.c_int, [_h, _vp, _vp]),
    "funcsne_profile_step": (C.c_int, [_h, C.c_int32, C.POINTER(C.c_double)]),
    "funcsne_exact_knn": (C.c_int, [_h, _vp, C.c_int64, C.c_int32, _vp, _vp]),
    "funcsne_exact_knn_noalloc": (C.c_int, [_vp, C.c_int64, C.c_int32, C.c_int32, _vp, C.c_int64, C.c_int32,
                                            _vp, _vp, _vp]),
    "funcsne_mlp_train": (C.c_int, [_h, C.c_int32]),
    "funcsne_mlp_predict": (C.c_int, [_h, _vp, C.c_int64, _vp]),
    "funcsne_mlp_debug_step": (C.c_int, [_h, C.POINTER(MlpDebug)]),
    "funcsne_last_error": (C.c_char_p, [_h]),
    "funcsne_destroy": (None, [_h]),
}

_lib = None


def load(path: str | None = None):
    """Load libfuncsne.so (built by ``__graft_entry__.build()``), or the
    library that the environment variable FUNCSNE_LIBRARY names (for
    example the range-checked build, libfuncsne_checked.so)."""
    global _lib
    if _lib is not None:
        return _lib
    if path is None:
        path = os.environ.get("FUNCSNE_LIBRARY") or LIB_PATH
    if not os.path.exists(path):
        raise FuncSNEError(-6, f"{path} is missing: build it with paper_2509_07681_gb300.build.build()")
    lib = C.CDLL(path)
    for name, (res, args) in ABI_FUNCTIONS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(rc: int, h=None):
    if rc != 0:
        msg = load().funcsne_last_error(h)
        raise FuncSNEError(rc, msg.decode() if msg else "")


def _ptr(a):
    """(pointer, keep-alive) for a numpy array or torch tensor (C-contiguous)."""
    if a is None:
        return None, None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data, a
    try:
        import torch
    except ImportError:  # pragma: no cover
        torch = None
    if torch is not None and isinstance(a, torch.Tensor):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr(), a
    raise TypeError(f"unsupported array type {type(a)}")


# ---------------------------------------------------------------- C-named functions
def funcsne_create(X, d, k_hd, k_ld, n_neg, alpha, perplexity, seed=0):
    L = load()
    N, D = X.shape
    p, keep = _ptr(X)
    h = _h()
    rc = L.funcsne_create(p, N, D, d, k_hd, k_ld, n_neg, alpha, perplexity, seed, C.byref(h))
    _check(rc, None)
    return h


def funcsne_set_option(h, key, value):
    _check(load().funcsne_set_option(h, key.encode(), float(value)), h)


def funcsne_get_option(h, key):
    v = C.c_double()
    _check(load().funcsne_get_option(h, key.encode(), C.byref(v)), h)
    return v.value


def funcsne_set_stream(h, stream_ptr):
    _check(load().funcsne_set_stream(h, stream_ptr), h)


def funcsne_step(h, n_iters=1):
    _check(load().funcsne_step(h, int(n_iters)), h)


def funcsne_sync(h):
    _check(load().funcsne_sync(h), h)


def funcsne_insert(h, X_new, placement=PLACE_MEAN):
    p, keep = _ptr(X_new)
    first = C.c_int64()
    _check(load().funcsne_insert(h, p, X_new.shape[0], placement, C.byref(first)), h)
    return first.value


def funcsne_update_points(h, ids, X_rows):
    pi, keep_i = _ptr(ids)
    px, keep_x = _ptr(X_rows)
    _check(load().funcsne_update_points(h, pi, ids.shape[0], px), h)


def funcsne_remove(h, ids):
    pi, keep_i = _ptr(ids)
    _check(load().funcsne_remove(h, pi, ids.shape[0]), h)


def funcsne_scale_embedding(h, factor):
    _check(load().funcsne_scale_embedding(h, float(factor)), h)


def funcsne_get_embedding_async(h, out):
    p, keep = _ptr(out)
    _check(load().funcsne_get_embedding_async(h, p, out.shape[0]), h)
    return keep


def funcsne_wait_embedding(h):
    _check(load().funcsne_wait_embedding(h), h)


def funcsne_get_data(h, out):
    p, keep = _ptr(out)
    _check(load().funcsne_get_data(h, p, out.shape[0]), h)
    return out


def funcsne_get_embedding(h, out):
    p, keep = _ptr(out)
    _check(load().funcsne_get_embedding(h, p, out.shape[0]), h)
    return out


def funcsne_get_knn(h, space, idx, d2=None):
    pi, k1 = _ptr(idx)
    pd, k2 = _ptr(d2)
    _check(load().funcsne_get_knn(h, space, pi, pd), h)
    return idx, d2


def funcsne_get_stats(h):
    s = Stats()
    _check(load().funcsne_get_stats(h, C.byref(s)), h)
    return {f: getattr(s, f) for f, _ in Stats._fields_}


def funcsne_export_state(h, arrays):
    st = State()
    keep = []
    for f in ("Y", "V", "hd_idx", "hd_d2", "ld_idx", "beta", "P"):
        p, k = _ptr(arrays.get(f))
        setattr(st, f, p)
        keep.append(k)
    _check(load().funcsne_export_state(h, C.byref(st)), h)
    return dict(Zhat=st.Zhat, E=st.E, t=st.t, fresh_lo=st.fresh_lo, fresh_until=st.fresh_until)


def funcsne_import_state(h, arrays, Zhat, E, t, fresh_lo, fresh_until=0):
    """fresh_lo / fresh_until: the insertion window (fresh_lo = N: none)."""
    st = State()
    keep = []
    for f in ("Y", "V", "hd_idx", "hd_d2", "ld_idx", "beta", "P"):
        p, k = _ptr(arrays.get(f))
        setattr(st, f, p)
        keep.append(k)
    st.Zhat, st.E, st.t = float(Zhat), float(E), int(t)
    st.fresh_lo, st.fresh_until = int(fresh_lo), int(fresh_until)
    _check(load().funcsne_import_state(h, C.byref(st)), h)


def funcsne_debug_step(h, att, rep):
    pa, k1 = _ptr(att)
    pr, k2 = _ptr(rep)
    _check(load().funcsne_debug_step(h, pa, pr), h)
    return att, rep


PHASE_KERNELS = ("hd_refine", "ld_refine", "forces", "update")


def funcsne_profile_step(h, n_iters):
    """Summed milliseconds per kernel over n_iters iterations (dict)."""
    out = (C.c_double * 4)()
    _check(load().funcsne_profile_step(h, int(n_iters), out), h)
    return dict(zip(PHASE_KERNELS, list(out)))


def funcsne_exact_knn(h, queries, k, idx, d2=None):
    pq, k0 = _ptr(queries)
    pi, k1 = _ptr(idx)
    pd, k2 = _ptr(d2)
    _check(load().funcsne_exact_knn(h, pq, len(queries), k, pi, pd), h)
    return idx, d2


def funcsne_exact_knn_noalloc(X, N, D, ldx, queries, k, idx, d2=None, stream=None):
    """X, idx, d2: device arrays; queries: host int32 array. No device allocation."""
    px, k0 = _ptr(X)
    q = np.ascontiguousarray(queries, dtype=np.int32)
    pi, k1 = _ptr(idx)
    pd, k2 = _ptr(d2)
    _check(load().funcsne_exact_knn_noalloc(px, N, D, ldx, q.ctypes.data, len(q), k, pi, pd, stream), None)
    return idx, d2


def funcsne_mlp_train(h, n_steps):
    _check(load().funcsne_mlp_train(h, int(n_steps)), h)


def funcsne_mlp_predict(h, X, out):
    px, k0 = _ptr(X)
    po, k1 = _ptr(out)
    _check(load().funcsne_mlp_predict(h, px, X.shape[0], po), h)
    return out


def funcsne_mlp_debug_step(h, arrays):
    st = MlpDebug()
    keep = []
    for f in ("batch_idx", "xhat", "target", "output", "theta_before", "weights_bf16", "grad", "theta_after"):
        p, k = _ptr(arrays.get(f))
        setattr(st, f, p)
        keep.append(k)
    _check(load().funcsne_mlp_debug_step(h, C.byref(st)), h)
    return dict(loss=st.loss, scale=st.scale, step=st.step, n_params=st.n_params)


def funcsne_debug_row_bounds(h, out):
    """Each row's stored bound E_i >= ||x_i - x~_i|| of its BF16 / FP8 copy."""
    po, keep = _ptr(out)
    _check(load().funcsne_debug_row_bounds(h, po, int(out.shape[0])), h)
    return out


def funcsne_debug_fail_alloc(after):
    """After `after` more successful device allocations, fail the next one
    once (FUNCSNE_E_OOM); after < 0 switches this off. For tests."""
    _check(load().funcsne_debug_fail_alloc(int(after)))


def funcsne_last_error(h=None):
    m = load().funcsne_last_error(h)
    return m.decode() if m else ""


def funcsne_destroy(h):
    load().funcsne_destroy(h)


# ---------------------------------------------------------------- convenience wrapper
class FuncSNE:
    """One FUnc-SNE run on the current CUDA device.

    >>> m = FuncSNE(X, d=2, k_hd=32, k_ld=16, n_neg=16, alpha=1.0, perplexity=30.0)
    >>> m.step(500); Y = m.embedding()
    """

    def __init__(self, X, d, k_hd, k_ld, n_neg, alpha=1.0, perplexity=30.0, seed=0, **options):
        X = _as_f32(X)
        self.N, self.D = X.shape
        self.d, self.k_hd, self.k_ld, self.n_neg = d, k_hd, k_ld, n_neg
        self._alpha0, self._perplexity0, self._seed = alpha, perplexity, seed
        self.h = funcsne_create(X, d, k_hd, k_ld, n_neg, alpha, perplexity, seed)
        for k, v in options.items():
            self.set_option(k, v)

    def set_option(self, key, value):
        funcsne_set_option(self.h, key, value)

    def get_option(self, key):
        return funcsne_get_option(self.h, key)

    def set_stream(self, stream):
        """stream: a torch.cuda.Stream, a raw cudaStream_t integer, or None."""
        ptr = getattr(stream, "cuda_stream", stream)
        funcsne_set_stream(self.h, ptr)

    def step(self, n=1):
        funcsne_step(self.h, n)

    def sync(self):
        funcsne_sync(self.h)

    def profile_step(self, n=1):
        """Milliseconds per kernel (hd_refine, ld_refine, forces, update) over n iterations."""
        return funcsne_profile_step(self.h, n)

    def embedding(self, out=None):
        if out is None:
            out = np.empty((self.N, self.d), dtype=np.float32)
        return funcsne_get_embedding(self.h, out)

    def embedding_async(self, out):
        """Queue a read-out of the current embedding into `out` (N x d float32;
        pinned host memory or a CUDA tensor for the copy to overlap the next
        steps). `out` is valid after wait_embedding() or sync()."""
        self._pending_out = funcsne_get_embedding_async(self.h, out)
        return out

    def debug_bounded_wait(self, polls=1000):
        """A device wait that runs out; the next sync() raises FuncSNEError."""
        _check(load().funcsne_debug_bounded_wait(self.h, int(polls)), self.h)

    def wait_embedding(self):
        funcsne_wait_embedding(self.h)
        self._pending_out = None

    def knn(self, space=SPACE_HD, with_d2=True):
        k = self.k_hd if space == SPACE_HD else self.k_ld
        idx = np.empty((self.N, k), dtype=np.int32)
        d2 = np.empty((self.N, k), dtype=np.float32) if with_d2 else None
        funcsne_get_knn(self.h, space, idx, d2)
        return (idx, d2) if with_d2 else idx

    def stats(self):
        return funcsne_get_stats(self.h)

    def export_state(self):
        a = dict(Y=np.empty((self.N, self.d), np.float32), V=np.empty((self.N, self.d), np.float32),
                 hd_idx=np.empty((self.N, self.k_hd), np.int32),
                 hd_d2=np.empty((self.N, self.k_hd), np.float32),
                 ld_idx=np.empty((self.N, self.k_ld), np.int32), beta=np.empty(self.N, np.float32),
                 P=np.empty((self.N, self.k_hd), np.float32))
        a.update(funcsne_export_state(self.h, a))
        return a

    def import_state(self, st):
        arrays = {k: (_as_f32(v) if k in ("Y", "V", "beta", "P") else np.ascontiguousarray(v, np.int32))
                  for k, v in st.items() if k in ("Y", "V", "hd_idx", "ld_idx", "beta", "P") and v is not None}
        funcsne_import_state(self.h, arrays, st["Zhat"], st["E"], st["t"], st.get("fresh_lo", self.N),
                             st.get("fresh_until", 0))

    def debug_step(self):
        att = np.empty((self.N, self.d), np.float32)
        rep = np.empty((self.N, self.d), np.float32)
        funcsne_debug_step(self.h, att, rep)
        return att, rep

    def row_bounds(self):
        """Each row's stored bound E_i >= ||x_i - x~_i|| of its reduced-precision copy."""
        return funcsne_debug_row_bounds(self.h, np.empty(self.N, np.float32))

    def exact_knn(self, queries, k):
        q = np.ascontiguousarray(queries, dtype=np.int32)
        idx = np.empty((len(q), k), np.int32)
        d2 = np.empty((len(q), k), np.float32)
        funcsne_exact_knn(self.h, q, k, idx, d2)
        return idx, d2

    def mlp_train(self, n_steps=1):
        funcsne_mlp_train(self.h, n_steps)

    def mlp_predict(self, X):
        X = _as_f32(X)
        out = np.empty((X.shape[0], self.d), np.float32)
        return funcsne_mlp_predict(self.h, X, out)

    def mlp_debug_step(self):
        """One training step of the placement MLP; returns its inputs, outputs,
        gradient and parameters before / after (numpy arrays)."""
        B = int(self.get_option("mlp_batch"))
        H = int(self.get_option("mlp_hidden"))
        n = H * self.D + H + H * H + H + self.d * H + self.d
        a = dict(batch_idx=np.empty(B, np.int32), xhat=np.empty((B, self.D), np.float32),
                 target=np.empty((B, self.d), np.float32), output=np.empty((B, self.d), np.float32),
                 theta_before=np.empty(n, np.float32), weights_bf16=np.empty(n, np.float32),
                 grad=np.empty(n, np.float32), theta_after=np.empty(n, np.float32))
        a.update(funcsne_mlp_debug_step(self.h, a))
        return a

    def insert(self, X_new, placement=PLACE_MEAN):
        X_new = _as_f32(X_new)
        first = funcsne_insert(self.h, X_new, placement)
        self.N += X_new.shape[0]
        return first

    def anneal(self, alphas, iters_per_level):
        """Snapshots under growing tail weight (Section 4.2): for each alpha
        in `alphas` (usually decreasing, so the LD kernel tails get heavier
        and clusters fragment), set it, run `iters_per_level` iterations and
        keep a copy of the embedding. Returns the list of N x d snapshots;
        clustering them into a hierarchy is left to the caller."""
        snaps = []
        for a in alphas:
            self.set_option("alpha", float(a))
            self.step(int(iters_per_level))
            snaps.append(self.embedding())
        return snaps

    def scale_embedding(self, factor):
        """Scale Y and V by factor and re-estimate Zhat (the implosion)."""
        funcsne_scale_embedding(self.h, factor)

    def data(self, out=None):
        """The N x D HD rows the handle holds."""
        if out is None:
            out = np.empty((self.N, self.D), dtype=np.float32)
        return funcsne_get_data(self.h, out)

    CHECKPOINT_OPTIONS = ("lr", "momentum", "att_ratio", "rep_ratio", "exaggeration", "exag_iters", "hd_mode",
                          "precision", "alpha", "perplexity", "concurrent", "surrogate", "mlp_every", "mlp_lr",
                          "mlp_batch", "mlp_hidden", "forces_cw", "forces_pair", "ld_pair", "hd_lanes", "insert_rounds",
                          "jump_iters", "jump_parts", "coin_floor", "gamma_e", "gamma_z", "fresh_iters")

    def save(self, path):
        """Checkpoint: HD rows, the exported iteration state, the creation
        parameters, the seed and the options, in one .npz file. The placement
        MLP's parameters are not part of it (it retrains online)."""
        st = self.export_state()
        opts = {k: self.get_option(k) for k in self.CHECKPOINT_OPTIONS}
        np.savez(path, X=self.data(), **{k: v for k, v in st.items() if isinstance(v, np.ndarray)},
                 Zhat=st["Zhat"], E=st["E"], t=st["t"], fresh_lo=st["fresh_lo"], fresh_until=st["fresh_until"],
                 params=np.array([self.d, self.k_hd, self.k_ld, self.n_neg], dtype=np.int64),
                 alpha0=self._alpha0, perplexity0=self._perplexity0, seed=np.uint64(self._seed),
                 opt_keys=np.array(list(opts)), opt_vals=np.array(list(opts.values()), dtype=np.float64))

    @classmethod
    def load_checkpoint(cls, path):
        """Recreate a handle from save(): same rows, state, seed and options;
        the next iterations draw the same random numbers."""
        z = np.load(path)
        d, k_hd, k_ld, n_neg = (int(v) for v in z["params"])
        m = cls(z["X"], d, k_hd, k_ld, n_neg, float(z["alpha0"]), float(z["perplexity0"]), seed=int(z["seed"]))
        opts = dict(zip(z["opt_keys"].tolist(), z["opt_vals"].tolist()))
        for k in ("precision", "hd_lanes", "forces_cw", "forces_pair", "ld_pair", "concurrent", "mlp_batch", "mlp_hidden"):
            m.set_option(k, opts.pop(k))
        perp = opts.pop("perplexity")
        for k, v in opts.items():
            m.set_option(k, v)
        if perp != m.get_option("perplexity"):
            m.set_option("perplexity", perp)
        m.import_state({k: z[k] for k in ("Y", "V", "hd_idx", "ld_idx", "beta", "P")} |
                       {"Zhat": float(z["Zhat"]), "E": float(z["E"]), "t": int(z["t"]),
                        "fresh_lo": int(z["fresh_lo"]) if "fresh_lo" in z else m.N,
                        "fresh_until": int(z["fresh_until"]) if "fresh_until" in z else 0})
        return m

    def update_points(self, ids, X_rows):
        """Replace the HD rows of existing points (drift); every point is
        then recalibrated from its list."""
        ids = np.ascontiguousarray(ids, dtype=np.int64)
        funcsne_update_points(self.h, ids, _as_f32(X_rows))

    def remove(self, ids):
        """Remove points; the kept points are renumbered in order."""
        ids = np.ascontiguousarray(ids, dtype=np.int64)
        funcsne_remove(self.h, ids)
        self.N -= ids.shape[0]

    def close(self):
        if getattr(self, "h", None):
            funcsne_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def _as_f32(a):
    if isinstance(a, np.ndarray):
        return np.ascontiguousarray(a, dtype=np.float32)
    return a.contiguous()
