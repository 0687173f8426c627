"""ctypes binding of librecon (include/recon.h): the same entry points under
the same names, argument marshalling only.

Every computation runs in the CUDA library; this module converts NumPy arrays
and torch tensors to pointers and status codes to exceptions.  There is no
fallback: if ``librecon.so`` is missing or no GPU is usable, calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librecon.so")

RECON_OK, RECON_EINVAL, RECON_ENOMEM, RECON_ECUDA, RECON_ETIMEOUT, RECON_ESTATE, RECON_EUNSUPPORTED = range(7)
RECON_ISING, RECON_GAUSSIAN = 0, 1
RECON_X_INT8, RECON_X_FP32 = 0, 1
RECON_KNN_NNDESCENT, RECON_KNN_EXHAUSTIVE, RECON_KNN_AUTO, RECON_KNN_SCREEN = 0, 1, 2, 3
RECON_SEED_RANDOM, RECON_SEED_SCREEN, RECON_SEED_LEARNED = 0, 1, 2
RECON_DIST_GAIN, RECON_DIST_GRADIENT = 0, 1
STATUS_NAMES = ["RECON_OK", "RECON_EINVAL", "RECON_ENOMEM", "RECON_ECUDA", "RECON_ETIMEOUT", "RECON_ESTATE",
                "RECON_EUNSUPPORTED"]


class recon_options(C.Structure):
    _fields_ = [("lambda_", C.c_double), ("seed", C.c_uint64), ("eps_knn", C.c_double),
                ("max_knn_iters", C.c_int32), ("w_clamp", C.c_float), ("h_clamp", C.c_float),
                ("knn_mode", C.c_int32), ("seed_mode", C.c_int32), ("screen_c", C.c_int32),
                ("timing", C.c_int32), ("no_graphs", C.c_int32),
                ("learned_frac", C.c_float), ("distance", C.c_int32), ("screen_fp8", C.c_int32),
                ("screen_no_rank1", C.c_int32), ("shard_index", C.c_int32), ("shard_count", C.c_int32),
                ("screen_pair", C.c_int32)]


class recon_stats(C.Structure):
    _fields_ = [("pair_evals", C.c_int64), ("newton_passes", C.c_int64), ("knn_iters", C.c_int64),
                ("levels", C.c_int32), ("level_k", C.c_int32 * 16), ("level_size", C.c_int64 * 17),
                ("nnz", C.c_int64), ("samples", C.c_int64), ("kernel_launches", C.c_int64),
                ("score_launches", C.c_int64), ("score_pairs", C.c_int64), ("score_ms", C.c_double),
                ("screen_launches", C.c_int64), ("screen_ms", C.c_double), ("screen_flop", C.c_double),
                ("screen_survivors", C.c_int64), ("seeded_nodes", C.c_int64), ("tuned_threads", C.c_int64),
                ("dropped_offers", C.c_int64), ("screen_rank1", C.c_int64),
                ("device_bytes", C.c_int64), ("nnd_graph_loops", C.c_int64)]


class recon_peaks(C.Structure):
    _fields_ = [("sm_count", C.c_int32), ("sm_clock_mhz", C.c_double), ("l2_bytes", C.c_int64),
                ("fp32_tflops", C.c_double), ("fp64_tflops", C.c_double), ("mufu_rcp_gops", C.c_double),
                ("mufu_ex2_gops", C.c_double), ("mufu_lg2_gops", C.c_double), ("mufu_tanh_gops", C.c_double),
                ("l2_read_gbs", C.c_double), ("l2_buffer_bytes", C.c_double)]


class recon_train_opts(C.Structure):
    _fields_ = [("steps", C.c_int32), ("lr", C.c_float), ("seed", C.c_uint64), ("n_pairs", C.c_int64),
                ("pairs", C.c_void_p), ("targets", C.c_void_p), ("n_best", C.c_int64), ("n_random", C.c_int64),
                ("fixed_sketch", C.c_int32), ("reserved", C.c_int32 * 7)]


class ReconError(RuntimeError):
    def __init__(self, status: int, msg: str):
        self.status = status
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 7 else status}: {msg}")


_lib = None
_EXPORTS = {
    "recon_default_options": (None, [C.c_void_p]),
    "recon_init": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_int32, C.c_int32, C.c_int32,
                             C.c_void_p, C.c_void_p]),
    "recon_objective": (C.c_int, [C.c_void_p, C.c_void_p]),
    "recon_score": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_int32]),
    "recon_score_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
    "recon_select_best": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_void_p,
                                    C.c_void_p, C.c_int64, C.c_void_p, C.c_int32]),
    "recon_best_pairs": (C.c_int, [C.c_void_p, C.c_int32, C.c_double, C.c_void_p, C.c_void_p, C.c_int64,
                                   C.c_void_p, C.c_int32]),
    "recon_exhaustive_best": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p,
                                        C.c_int32]),
    "recon_cd_sweep": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.c_void_p]),
    "recon_field_sweep": (C.c_int, [C.c_void_p, C.c_void_p]),
    "recon_gcd_step": (C.c_int, [C.c_void_p, C.c_int32, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p]),
    "recon_get_model": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
    "recon_set_model": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]),
    "recon_get_stats": (C.c_int, [C.c_void_p, C.c_void_p]),
    "recon_save": (C.c_int, [C.c_void_p, C.c_char_p]),
    "recon_load": (C.c_int, [C.c_void_p, C.c_char_p, C.c_void_p]),
    "recon_set_list_lengths": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64]),
    "recon_row_best": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_float, C.c_void_p, C.c_void_p, C.c_int64,
                                 C.c_void_p]),
    "recon_knn_graph": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
    "recon_proposal_param_count": (C.c_int64, []),
    "recon_default_train_opts": (None, [C.c_void_p]),
    "recon_proposal_train": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "recon_proposal_weights": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64]),
    "recon_proposal_embed": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "recon_proposal_grad": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
    "recon_device_peaks": (C.c_int, [C.c_int32, C.c_void_p]),
    "recon_last_error": (C.c_char_p, [C.c_void_p]),
    "recon_destroy": (None, [C.c_void_p]),
}


def lib():
    """Loads librecon.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built (run __graft_entry__.build())")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _EXPORTS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(st: int, ctx=None):
    if st != RECON_OK:
        msg = lib().recon_last_error(ctx)
        raise ReconError(st, msg.decode() if msg else "")


# ------------------------------------------------------------------ marshalling

def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(x):
    """(pointer, is_device, keepalive) of a NumPy array or torch tensor."""
    if x is None:
        return None, 0, None
    if _is_torch(x):
        assert x.is_contiguous()
        return x.data_ptr(), int(x.is_cuda), x
    a = np.ascontiguousarray(x)
    return a.ctypes.data, 0, a


def _stream_handle(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def recon_default_options(**kw) -> recon_options:
    o = recon_options()
    lib().recon_default_options(C.byref(o))
    for k, v in kw.items():
        setattr(o, "lambda_" if k in ("lam", "lambda") else k, v)
    return o


def recon_init(X, model: int = RECON_ISING, options: recon_options | None = None, stream=None):
    """X: samples, sample-major (M x N): int8 spins (Ising) or float32 (Gaussian);
    a NumPy array or a (host or CUDA) torch tensor.  Returns a context handle."""
    if _is_torch(X):
        M, N = X.shape
        xt = RECON_X_INT8 if str(X.dtype) == "torch.int8" else RECON_X_FP32
    else:
        X = np.ascontiguousarray(X)
        M, N = X.shape
        xt = RECON_X_INT8 if X.dtype == np.int8 else RECON_X_FP32
    p, dev, keep = _ptr(X)
    ctx = C.c_void_p()
    opt = options if options is not None else recon_default_options()
    st = lib().recon_init(C.byref(ctx), p, M, N, xt, dev, model, C.byref(opt), _stream_handle(stream))
    _check(st, None)
    return ctx


def recon_objective(ctx) -> float:
    out = C.c_double()
    _check(lib().recon_objective(ctx, C.byref(out)), ctx)
    return out.value


def recon_score(ctx, pairs, d_out=None, w_out=None):
    """d(i,j) = -gain for each pair.  Host arrays in -> host arrays out; CUDA
    tensors in -> the given CUDA output tensors are filled."""
    if _is_torch(pairs) and pairs.is_cuda:
        P = pairs.shape[0]
        _check(lib().recon_score(ctx, pairs.data_ptr(), P, d_out.data_ptr(),
                                 w_out.data_ptr() if w_out is not None else None, 1), ctx)
        return d_out, w_out
    pairs = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
    P = len(pairs)
    d = np.empty(P, dtype=np.float32)
    w = np.empty(P, dtype=np.float32)
    _check(lib().recon_score(ctx, pairs.ctypes.data, P, d.ctypes.data, w.ctypes.data, 0), ctx)
    return d, w


def recon_score_noalloc(ctx, pairs):
    """recon_score for a host pair list without any device allocation (at most
    65536 pairs per call); returns host arrays (d, w)."""
    pairs = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
    P = len(pairs)
    d = np.empty(P, dtype=np.float32)
    w = np.empty(P, dtype=np.float32)
    _check(lib().recon_score_noalloc(ctx, pairs.ctypes.data, P, d.ctypes.data, w.ctypes.data), ctx)
    return d, w


def recon_best_pairs(ctx, k: int, kappa: float, N: int):
    m = int(np.floor(kappa * N + 0.5))
    cap = max(min(m, N * (N - 1) // 2), 1)
    pairs = np.empty((cap, 2), dtype=np.int32)
    d = np.empty(cap, dtype=np.float32)
    mo = C.c_int64()
    _check(lib().recon_best_pairs(ctx, k, float(kappa), pairs.ctypes.data, d.ctypes.data, cap, C.byref(mo), 0), ctx)
    return pairs[:mo.value], d[:mo.value]


def recon_select_best(ctx, pairs, d, m: int):
    """The m best of a scored pair list (host arrays), unique and ordered by
    (d, i, j): (pairs [n x 2], d [n])."""
    p = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
    dd = np.ascontiguousarray(np.asarray(d, dtype=np.float32).ravel())
    if len(dd) != len(p):
        raise ValueError("pairs and d differ in length")
    cap = min(int(m), len(p))
    out = np.empty((max(cap, 1), 2), dtype=np.int32)
    od = np.empty(max(cap, 1), dtype=np.float32)
    n = C.c_int64(0)
    _check(lib().recon_select_best(ctx, p.ctypes.data, dd.ctypes.data, len(p), int(m), out.ctypes.data, od.ctypes.data,
                                   cap, C.byref(n), 0), ctx)
    return out[:n.value], od[:n.value]


def recon_exhaustive_best(ctx, m: int, N: int):
    cap = max(min(m, N * (N - 1) // 2), 1)
    pairs = np.empty((cap, 2), dtype=np.int32)
    d = np.empty(cap, dtype=np.float32)
    mo = C.c_int64()
    _check(lib().recon_exhaustive_best(ctx, m, pairs.ctypes.data, d.ctypes.data, cap, C.byref(mo), 0), ctx)
    return pairs[:mo.value], d[:mo.value]


def recon_cd_sweep(ctx, pairs) -> float:
    p, dev, keep = _ptr(pairs if _is_torch(pairs) else np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
    P = pairs.shape[0] if _is_torch(pairs) else keep.shape[0]
    out = C.c_double()
    _check(lib().recon_cd_sweep(ctx, p, P, dev, C.byref(out)), ctx)
    return out.value


def recon_field_sweep(ctx) -> float:
    out = C.c_double()
    _check(lib().recon_field_sweep(ctx, C.byref(out)), ctx)
    return out.value


def recon_gcd_step(ctx, k: int, kappa: float):
    dl, ob, m = C.c_double(), C.c_double(), C.c_int64()
    _check(lib().recon_gcd_step(ctx, k, float(kappa), C.byref(dl), C.byref(ob), C.byref(m)), ctx)
    return dl.value, ob.value, m.value


def recon_get_model(ctx, N: int):
    nnz = C.c_int64()
    fields = np.empty(N, dtype=np.float32)
    st = lib().recon_get_model(ctx, None, None, 0, C.byref(nnz), fields.ctypes.data)
    if st not in (RECON_OK, RECON_EINVAL):
        _check(st, ctx)
    n = nnz.value
    ij = np.empty((max(n, 1), 2), dtype=np.int32)
    w = np.empty(max(n, 1), dtype=np.float32)
    _check(lib().recon_get_model(ctx, ij.ctypes.data, w.ctypes.data, n, C.byref(nnz), fields.ctypes.data), ctx)
    return ij[:n], w[:n], fields


def recon_set_model(ctx, ij, w, fields=None):
    ij = np.ascontiguousarray(np.asarray(ij, dtype=np.int32).reshape(-1, 2))
    w = np.ascontiguousarray(np.asarray(w, dtype=np.float32))
    f = None if fields is None else np.ascontiguousarray(np.asarray(fields, dtype=np.float32))
    _check(lib().recon_set_model(ctx, ij.ctypes.data, w.ctypes.data, len(w), None if f is None else f.ctypes.data),
           ctx)


def recon_get_stats(ctx) -> dict:
    s = recon_stats()
    _check(lib().recon_get_stats(ctx, C.byref(s)), ctx)
    return {"pair_evals": s.pair_evals, "newton_passes": s.newton_passes, "knn_iters": s.knn_iters,
            "levels": s.levels, "level_k": list(s.level_k[:max(s.levels, 0)]),
            "level_size": list(s.level_size[:max(s.levels, 0) + 1]), "nnz": s.nnz, "samples": s.samples,
            "kernel_launches": s.kernel_launches, "score_launches": s.score_launches,
            "score_pairs": s.score_pairs, "score_ms": s.score_ms, "screen_launches": s.screen_launches,
            "screen_ms": s.screen_ms, "screen_flop": s.screen_flop, "screen_survivors": s.screen_survivors,
            "seeded_nodes": s.seeded_nodes, "tuned_threads": s.tuned_threads,
            "dropped_offers": s.dropped_offers, "screen_rank1": s.screen_rank1, "device_bytes": s.device_bytes,
            "nnd_graph_loops": s.nnd_graph_loops}


def recon_set_list_lengths(ctx, k=None):
    """Per-node list lengths of the first FindBest level (None clears them)."""
    if k is None:
        _check(lib().recon_set_list_lengths(ctx, None, 0), ctx)
        return
    a = np.ascontiguousarray(np.asarray(k, dtype=np.int32))
    _check(lib().recon_set_list_lengths(ctx, a.ctypes.data, len(a)), ctx)


def recon_row_best(ctx, rows, d_cut: float, cap: int = None):
    """All pairs incident to `rows` with d < d_cut, exact, ascending (d, i, j):
    (pairs [n x 2], d [n], count found)."""
    r = np.ascontiguousarray(np.asarray(rows, dtype=np.int32).ravel())
    n = C.c_int64(0)
    if cap is None:
        _check(lib().recon_row_best(ctx, r.ctypes.data, len(r), C.c_float(d_cut), None, None, 0, C.byref(n)), ctx)
        cap = n.value
    p = np.empty((max(cap, 1), 2), dtype=np.int32)
    d = np.empty(max(cap, 1), dtype=np.float32)
    _check(lib().recon_row_best(ctx, r.ctypes.data, len(r), C.c_float(d_cut), p.ctypes.data, d.ctypes.data, cap,
                                C.byref(n)), ctx)
    k = min(n.value, cap)
    return p[:k], d[:k], n.value


def recon_knn_graph(ctx):
    """The first-level k-NN lists of the last FindBest search: (ids [N x k],
    d [N x k]), padding id -1 / d +inf; empty arrays when no lists were built."""
    k = C.c_int32(0)
    n = C.c_int64(0)
    _check(lib().recon_knn_graph(ctx, None, None, 0, C.byref(k), C.byref(n)), ctx)
    ids = np.empty((n.value, k.value), dtype=np.int32)
    d = np.empty((n.value, k.value), dtype=np.float32)
    if ids.size:
        _check(lib().recon_knn_graph(ctx, ids.ctypes.data, d.ctypes.data, ids.size, C.byref(k), C.byref(n)), ctx)
    return ids, d


def recon_proposal_param_count() -> int:
    return lib().recon_proposal_param_count()


def recon_proposal_train(ctx, steps: int = 300, lr: float = 3e-3, seed: int = 7, pairs=None, targets=None,
                         n_best: int = 0, n_random: int = 0, fixed_sketch: int = 0):
    """Trains the learned proposal; returns the loss before each step."""
    o = recon_train_opts()
    lib().recon_default_train_opts(C.byref(o))
    o.steps, o.lr, o.seed, o.n_best, o.n_random = steps, lr, seed, n_best, n_random
    o.fixed_sketch = fixed_sketch
    keep = []
    if pairs is not None:
        p = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
        keep.append(p)
        o.pairs, o.n_pairs = p.ctypes.data, len(p)
        if targets is not None:
            t = np.ascontiguousarray(np.asarray(targets, dtype=np.float32))
            keep.append(t)
            o.targets = t.ctypes.data
    loss = np.empty(max(steps, 1), dtype=np.float32)
    _check(lib().recon_proposal_train(ctx, C.byref(o), loss.ctypes.data), ctx)
    return loss[:steps]


def recon_proposal_weights(ctx, set_in=None):
    """Returns the parameters (W1 | b1 | W2 | b2, FP32); sets them first if given."""
    n = recon_proposal_param_count()
    out = np.empty(n, dtype=np.float32)
    si = None if set_in is None else np.ascontiguousarray(np.asarray(set_in, dtype=np.float32))
    _check(lib().recon_proposal_weights(ctx, out.ctypes.data, None if si is None else si.ctypes.data, n), ctx)
    return out


def recon_proposal_embed(ctx, N: int):
    sk = np.empty((N, 64), dtype=np.float32)
    em = np.empty((N, 32), dtype=np.float32)
    _check(lib().recon_proposal_embed(ctx, sk.ctypes.data, em.ctypes.data), ctx)
    return sk, em


def recon_proposal_grad(ctx, pairs, targets):
    p = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
    t = np.ascontiguousarray(np.asarray(targets, dtype=np.float32))
    g = np.empty(recon_proposal_param_count(), dtype=np.float32)
    loss = C.c_double()
    _check(lib().recon_proposal_grad(ctx, p.ctypes.data, t.ctypes.data, len(p), g.ctypes.data, C.byref(loss)), ctx)
    return g, loss.value


def recon_device_peaks(device: int = 0) -> dict:
    """The device's measured FP32/FP64 FMA, MUFU and L2-read ceilings (see recon_peaks)."""
    out = recon_peaks()
    _check(lib().recon_device_peaks(int(device), C.byref(out)))
    return {name: getattr(out, name) for name, _ in recon_peaks._fields_}


def recon_save(ctx, path: str):
    _check(lib().recon_save(ctx, path.encode()), ctx)


def recon_load(path: str, stream=None):
    ctx = C.c_void_p()
    _check(lib().recon_load(C.byref(ctx), path.encode(), _stream_handle(stream)), None)
    return ctx


def recon_last_error(ctx=None) -> str:
    m = lib().recon_last_error(ctx)
    return m.decode() if m else ""


def recon_destroy(ctx):
    if ctx:
        lib().recon_destroy(ctx)


class Recon:
    """Owning wrapper around a context."""

    def __init__(self, X, model: int = RECON_ISING, stream=None, **options):
        X_shape = tuple(X.shape)
        self.M, self.N = X_shape
        self.model = model
        self.ctx = recon_init(X, model, recon_default_options(**options), stream)

    def close(self):
        if self.ctx:
            recon_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def objective(self):
        return recon_objective(self.ctx)

    def score(self, pairs, d_out=None, w_out=None):
        return recon_score(self.ctx, pairs, d_out, w_out)

    def best_pairs(self, k: int, kappa: float):
        return recon_best_pairs(self.ctx, k, kappa, self.N)

    def row_best(self, rows, d_cut: float, cap: int = None):
        return recon_row_best(self.ctx, rows, d_cut, cap)

    def knn_graph(self):
        return recon_knn_graph(self.ctx)

    def exhaustive_best(self, m: int):
        return recon_exhaustive_best(self.ctx, m, self.N)

    def cd_sweep(self, pairs):
        return recon_cd_sweep(self.ctx, pairs)

    def field_sweep(self):
        return recon_field_sweep(self.ctx)

    def gcd_step(self, k: int, kappa: float):
        return recon_gcd_step(self.ctx, k, kappa)

    def get_model(self):
        return recon_get_model(self.ctx, self.N)

    def set_model(self, ij, w, fields=None):
        return recon_set_model(self.ctx, ij, w, fields)

    def stats(self):
        return recon_get_stats(self.ctx)

    def save(self, path):
        recon_save(self.ctx, path)
