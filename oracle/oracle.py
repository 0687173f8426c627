"""Python side of the FP64 CPU oracle (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg use this module.  It loads ``liboracle.so`` (built from
``recon_oracle.c`` with gcc) and composes its functions into the paper's
algorithms: coordinate descent (Algorithm 1), greedy coordinate descent
(Algorithm 2) with exhaustive or FindBest (Algorithm 3) selection, and the
recall measure of Sec. IV.  Nothing here imports the CUDA package, and the
CUDA package never imports this.

Every quantity is double precision.  X is node-major (N x M).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "recon_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None
_lock = threading.Lock()

_i8p = np.ctypeslib.ndpointer(np.int8, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")


class FindBestStats(C.Structure):
    _fields_ = [("levels", C.c_int), ("level_size", C.c_int64 * 64), ("level_D", C.c_int64 * 64),
                ("level_k", C.c_int * 64), ("knn_iters", C.c_int64)]


def build(force: bool = False) -> str:
    """Compile liboracle.so (plain C, -O2, OpenMP for timing runs only)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB_PATH)
            vp, d, i, i64 = C.c_void_p, C.c_double, C.c_int, C.c_int64
            L.orc_ising_phi.argtypes = [i, i, _i8p, _f64p, _f64p, _f64p]
            L.orc_ising_objective.argtypes = [i, i, _i8p, _f64p, _f64p, d]
            L.orc_ising_objective.restype = d
            L.orc_ising_pair_gain.argtypes = [i, _i8p, _i8p, _f64p, _f64p, d, d, d, C.POINTER(C.c_double)]
            L.orc_ising_pair_gain.restype = d
            L.orc_ising_score_pairs.argtypes = [i, i, _i8p, _f64p, _f64p, d, d, i64, _i32p, _f64p, _f64p, i]
            L.orc_ising_score_pairs_rows.argtypes = [i, _i8p, _f64p, d, d, i64, _i32p, vp, _f64p, _f64p, i]
            L.orc_ising_update_pairs.argtypes = [i, i, _i8p, _f64p, _f64p, d, d, i64, _i32p]
            L.orc_ising_update_pairs.restype = d
            L.orc_ising_field_sweep.argtypes = [i, i, _i8p, _f64p, _f64p, d]
            L.orc_ising_field_sweep.restype = d
            L.orc_gauss_mu.argtypes = [i, i, _f64p, _f64p, _f64p]
            L.orc_gauss_objective.argtypes = [i, i, _f64p, _f64p, _f64p, d]
            L.orc_gauss_objective.restype = d
            L.orc_gauss_pair_gain.argtypes = [i, _f64p, _f64p, _f64p, _f64p, d, d, d, d, d,
                                              C.POINTER(C.c_double)]
            L.orc_gauss_pair_gain.restype = d
            L.orc_gauss_score_pairs.argtypes = [i, i, _f64p, _f64p, _f64p, vp, d, d, i64, _i32p, vp, _f64p,
                                                _f64p, i]
            L.orc_gauss_update_pairs.argtypes = [i, i, _f64p, _f64p, _f64p, _f64p, d, d, i64, _i32p]
            L.orc_gauss_update_pairs.restype = d
            L.orc_gauss_diag_sweep.argtypes = [i, i, _f64p, _f64p, _f64p]
            L.orc_gauss_diag_sweep.restype = d
            L.orc_exhaustive_best.argtypes = [i, _f64p, i, _i32p, i64, _i32p]
            L.orc_exhaustive_best.restype = i64
            L.orc_exact_knn.argtypes = [i, _f64p, i, _i32p, i, _i32p]
            L.orc_nndescent.argtypes = [i, _f64p, i, _i32p, i, d, i, i, C.c_uint64, _i32p,
                                        C.POINTER(C.c_int64)]
            L.orc_nndescent.restype = i
            L.orc_findbest.argtypes = [i, _f64p, i, _i32p, i64, i, i, d, i, i, C.c_uint64, _i32p,
                                       C.POINTER(FindBestStats)]
            L.orc_findbest.restype = i64
            L.orc_nthreads.restype = i
            _lib = L
    return _lib


def nthreads() -> int:
    return lib().orc_nthreads()


def _pairs32(pairs) -> np.ndarray:
    p = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
    return p


def all_pairs(idx) -> np.ndarray:
    """Every unordered pair (a < b) of the given node ids, lexicographic."""
    idx = np.sort(np.asarray(idx, dtype=np.int64))
    a, b = np.triu_indices(len(idx), 1)
    return np.stack([idx[a], idx[b]], 1).astype(np.int32)


# ----------------------------------------------------------------------------
# Ising state (App. A)
# ----------------------------------------------------------------------------

class IsingOracle:
    """State (W, h) of the Ising pseudo-likelihood problem with its tracked
    fields phi (App. A).  W is dense; fine for the sizes the oracle serves."""

    def __init__(self, X: np.ndarray, lam: float, w_clamp: float = 5.0, h_clamp: float = 10.0,
                 dense: bool = True):
        self.X = np.ascontiguousarray(X, dtype=np.int8)
        self.N, self.M = self.X.shape
        self.lam, self.w_clamp, self.h_clamp = float(lam), float(w_clamp), float(h_clamp)
        self.h = np.zeros(self.N)
        self.W = np.zeros((self.N, self.N)) if dense else None
        self.phi = np.zeros((self.N, self.M))
        # W = 0 start (Sec. II); the fields are then fitted (App. A updates them alongside W)
        self.field_sweep()

    # -- state
    def set_state(self, W: np.ndarray, h: np.ndarray):
        self.W = np.ascontiguousarray(W, dtype=np.float64)
        self.h = np.ascontiguousarray(h, dtype=np.float64).copy()
        self.phi = np.empty((self.N, self.M))
        lib().orc_ising_phi(self.N, self.M, self.X, self.h, self.W, self.phi)

    def objective(self) -> float:
        return lib().orc_ising_objective(self.N, self.M, self.X, self.h, self.W, self.lam)

    def field_sweep(self) -> float:
        return lib().orc_ising_field_sweep(self.N, self.M, self.X, self.phi, self.h, self.h_clamp)

    # -- pair gains
    def score(self, pairs, nthreads: int = 0):
        """(gain, w*) per pair; d(i,j) = -gain."""
        p = _pairs32(pairs)
        g = np.empty(len(p))
        w = np.empty(len(p))
        if len(p):
            lib().orc_ising_score_pairs(self.N, self.M, self.X, self.phi, self.W, self.lam, self.w_clamp,
                                        len(p), p, g, w, nthreads)
        return g, w

    def update(self, pairs) -> float:
        """Sequential coordinate updates in the given order; returns sum |dW|."""
        p = _pairs32(pairs)
        if not len(p):
            return 0.0
        return lib().orc_ising_update_pairs(self.N, self.M, self.X, self.phi, self.W, self.lam,
                                            self.w_clamp, len(p), p)

    def dist_matrix(self, nthreads: int = 0) -> np.ndarray:
        """Dense d(i,j) = -gain(i,j) over all pairs (diagonal 0)."""
        p = all_pairs(np.arange(self.N))
        g, _ = self.score(p, nthreads)
        D = np.zeros((self.N, self.N))
        D[p[:, 0], p[:, 1]] = -g
        D[p[:, 1], p[:, 0]] = -g
        return D


def ising_grad_rows(X: np.ndarray, phi: np.ndarray, pairs, lam: float, wcur=None) -> np.ndarray:
    """|d log pi / d W_ij| of the Ising pseudo-likelihood at the current state
    (App. B, "Gradient as distance").  phi_i = h_i + sum_j W_ij x_j enters the
    terms of node i through x_j and those of node j through x_i, so the smooth
    derivative is D = sum_m [x_j (x_i - tanh phi_i) + x_i (x_j - tanh phi_j)];
    the Laplace prior adds -lam sign(W_ij) where W_ij != 0 and nothing at 0 (a
    central difference of lam |W| at W = 0 vanishes).  X node-major int8 (N x M),
    phi float64 (N x M), wcur the current couplings of the pairs (default 0)."""
    p = np.asarray(pairs, dtype=np.int64).reshape(-1, 2)
    x = np.asarray(X, dtype=np.float64)
    t = np.tanh(np.asarray(phi, dtype=np.float64))
    i, j = p[:, 0], p[:, 1]
    D = (x[j] * (x[i] - t[i]) + x[i] * (x[j] - t[j])).sum(axis=1)
    w = np.zeros(len(p)) if wcur is None else np.asarray(wcur, dtype=np.float64)
    return np.abs(D - lam * np.sign(w))


def gauss_grad_rows(X: np.ndarray, mu: np.ndarray, s2: np.ndarray, pairs, lam: float, wcur=None) -> np.ndarray:
    """|d log pi / d W_ij| of the Gaussian pseudo-likelihood: with the residual
    e_i = x_i + s2_i mu_i (mu_i = sum_j W_ij x_j), the terms of node i depend on
    W_ij through mu_i (derivative x_j) and those of node j through mu_j, so
    D = -sum_m (e_i x_j + e_j x_i); the prior adds -lam sign(W_ij) off zero."""
    p = np.asarray(pairs, dtype=np.int64).reshape(-1, 2)
    x = np.asarray(X, dtype=np.float64)
    e = x + np.asarray(s2, dtype=np.float64)[:, None] * np.asarray(mu, dtype=np.float64)
    i, j = p[:, 0], p[:, 1]
    D = -(e[i] * x[j] + e[j] * x[i]).sum(axis=1)
    w = np.zeros(len(p)) if wcur is None else np.asarray(wcur, dtype=np.float64)
    return np.abs(D - lam * np.sign(w))


def ising_score_rows(X: np.ndarray, phi: np.ndarray, pairs, lam: float, w_clamp: float = 10.0,
                     wcur=None, nthreads: int = 0):
    """Pair gains from explicit field rows (no dense W), for large N."""
    p = _pairs32(pairs)
    X = np.ascontiguousarray(X, dtype=np.int8)
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    g = np.empty(len(p))
    w = np.empty(len(p))
    wc = None if wcur is None else np.ascontiguousarray(wcur, dtype=np.float64)
    lib().orc_ising_score_pairs_rows(X.shape[1], X, phi, float(lam), float(w_clamp), len(p), p,
                                     None if wc is None else wc.ctypes.data, g, w, nthreads)
    return g, w


def ising_fields_at_zero(X: np.ndarray, h_clamp: float = 10.0) -> np.ndarray:
    """Field optimum at W = 0 by the oracle's bisection, without a dense W."""
    X = np.ascontiguousarray(X, dtype=np.int8)
    N, M = X.shape
    h = np.zeros(N)
    phi = np.zeros((N, M))
    lib().orc_ising_field_sweep(N, M, X, phi, h, h_clamp)
    return h


# ----------------------------------------------------------------------------
# Gaussian state (App. A)
# ----------------------------------------------------------------------------

class GaussOracle:
    """State (W off-diagonal, s2 = theta^2 = 1/W_ii) of the Gaussian
    pseudo-likelihood problem with its tracked neighbour sums mu (App. A)."""

    def __init__(self, X: np.ndarray, lam: float, w_clamp: float = 1e6):
        self.X = np.ascontiguousarray(X, dtype=np.float64)
        self.N, self.M = self.X.shape
        self.lam, self.w_clamp = float(lam), float(w_clamp)
        self.W = np.zeros((self.N, self.N))
        self.mu = np.zeros((self.N, self.M))
        self.s2 = np.ones(self.N)
        self.diag_sweep()

    def set_state(self, W: np.ndarray, s2: np.ndarray):
        self.W = np.ascontiguousarray(W, dtype=np.float64)
        self.s2 = np.ascontiguousarray(s2, dtype=np.float64).copy()
        self.mu = np.empty((self.N, self.M))
        lib().orc_gauss_mu(self.N, self.M, self.X, self.W, self.mu)

    def objective(self) -> float:
        return lib().orc_gauss_objective(self.N, self.M, self.X, self.s2, self.W, self.lam)

    def diag_sweep(self) -> float:
        return lib().orc_gauss_diag_sweep(self.N, self.M, self.X, self.mu, self.s2)

    field_sweep = diag_sweep

    def score(self, pairs, nthreads: int = 0):
        p = _pairs32(pairs)
        g = np.empty(len(p))
        w = np.empty(len(p))
        if len(p):
            lib().orc_gauss_score_pairs(self.N, self.M, self.X, self.mu, self.s2, self.W.ctypes.data,
                                        self.lam, self.w_clamp, len(p), p, None, g, w, nthreads)
        return g, w

    def update(self, pairs) -> float:
        p = _pairs32(pairs)
        if not len(p):
            return 0.0
        return lib().orc_gauss_update_pairs(self.N, self.M, self.X, self.mu, self.s2, self.W, self.lam,
                                            self.w_clamp, len(p), p)

    def dist_matrix(self, nthreads: int = 0) -> np.ndarray:
        p = all_pairs(np.arange(self.N))
        g, _ = self.score(p, nthreads)
        D = np.zeros((self.N, self.N))
        D[p[:, 0], p[:, 1]] = -g
        D[p[:, 1], p[:, 0]] = -g
        return D


def gauss_score_rows(X: np.ndarray, mu: np.ndarray, s2: np.ndarray, pairs, lam: float,
                     w_clamp: float = 1e6, wcur=None, nthreads: int = 0):
    p = _pairs32(pairs)
    X = np.ascontiguousarray(X, dtype=np.float64)
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    s2 = np.ascontiguousarray(s2, dtype=np.float64)
    g = np.empty(len(p))
    w = np.empty(len(p))
    wc = None if wcur is None else np.ascontiguousarray(wcur, dtype=np.float64)
    lib().orc_gauss_score_pairs(X.shape[0], X.shape[1], X, mu, s2, None, float(lam), float(w_clamp),
                                len(p), p, None if wc is None else wc.ctypes.data, g, w, nthreads)
    return g, w


def gauss_diag_at_zero(X: np.ndarray) -> np.ndarray:
    X = np.ascontiguousarray(X, dtype=np.float64)
    N, M = X.shape
    s2 = np.ones(N)
    lib().orc_gauss_diag_sweep(N, M, X, np.zeros((N, M)), s2)
    return s2


# ----------------------------------------------------------------------------
# searches over a dense distance matrix
# ----------------------------------------------------------------------------

def exhaustive_best(D: np.ndarray, m: int, S=None) -> np.ndarray:
    """m best pairs of S (Algorithm 3's exhaustive base case)."""
    N = D.shape[0]
    S = np.arange(N, dtype=np.int32) if S is None else np.ascontiguousarray(S, dtype=np.int32)
    out = np.empty((max(m, 1), 2), dtype=np.int32)
    r = lib().orc_exhaustive_best(N, np.ascontiguousarray(D), len(S), S, m, out)
    return out[:r]


def exact_knn(D: np.ndarray, k: int, S=None) -> np.ndarray:
    N = D.shape[0]
    S = np.arange(N, dtype=np.int32) if S is None else np.ascontiguousarray(S, dtype=np.int32)
    G = np.empty((len(S), k), dtype=np.int32)
    lib().orc_exact_knn(N, np.ascontiguousarray(D), len(S), S, k, G)
    return G


def nndescent(D: np.ndarray, k: int, eps: float = 1e-3, max_iters: int = 100, in_cap: int | None = None,
              seed: int = 1, S=None):
    """Algorithm 4 over S; returns (G, iterations, replacements)."""
    N = D.shape[0]
    S = np.arange(N, dtype=np.int32) if S is None else np.ascontiguousarray(S, dtype=np.int32)
    G = np.empty((len(S), k), dtype=np.int32)
    rep = C.c_int64(0)
    it = lib().orc_nndescent(N, np.ascontiguousarray(D), len(S), S, k, eps, max_iters,
                             k if in_cap is None else in_cap, seed, G, C.byref(rep))
    return G, it, rep.value


def findbest(D: np.ndarray, m: int, knn_exact: bool = True, k_min: int = 1, eps: float = 1e-3,
             max_iters: int = 100, in_cap: int | None = None, seed: int = 1, S=None):
    """Algorithm 3; returns (pairs (m x 2, ascending d), stats)."""
    N = D.shape[0]
    S = np.arange(N, dtype=np.int32) if S is None else np.ascontiguousarray(S, dtype=np.int32)
    out = np.empty((max(m, 1), 2), dtype=np.int32)
    st = FindBestStats()
    r = lib().orc_findbest(N, np.ascontiguousarray(D), len(S), S, m, 1 if knn_exact else 0, k_min, eps,
                           max_iters, in_cap if in_cap is not None else max(k_min, 1), seed, out,
                           C.byref(st))
    stats = {
        "levels": st.levels,
        "level_size": [st.level_size[t] for t in range(st.levels + 1)],
        "level_D": [st.level_D[t] for t in range(st.levels)],
        "level_k": [st.level_k[t] for t in range(st.levels)],
        "knn_iters": st.knn_iters,
    }
    return out[:r], stats


# ----------------------------------------------------------------------------
# Algorithms 1 and 2, and recall
# ----------------------------------------------------------------------------

def order_for_update(pairs: np.ndarray, gain: np.ndarray) -> np.ndarray:
    """The order in which a GCD iteration applies its selected pairs: by gain
    descending, ties by (i, j) ascending.  The paper applies them one at a time
    in unspecified order; the parallel form (App. B) updates pairs that share
    no node concurrently, which is equivalent to this sequential order when
    every pair waits for the earlier pairs that share a node with it."""
    pairs = _pairs32(pairs)
    o = np.lexsort((pairs[:, 1], pairs[:, 0], -np.asarray(gain)))
    return pairs[o]


def round_half_up(x: float) -> int:
    return int(np.floor(x + 0.5))


def gcd(state, kappa: float, eps: float, max_iters: int = 1000, search: str = "exhaustive",
        fb_kwargs=None, callback=None):
    """Algorithm 2 with a field sweep after each pair sweep (App. A).  Returns
    the list of per-iteration (objective, Delta)."""
    N = state.N
    m = round_half_up(kappa * N)
    hist = []
    for it in range(max_iters):
        D = state.dist_matrix()
        if search == "exhaustive":
            best = exhaustive_best(D, m)
        else:
            best, _ = findbest(D, m, **(fb_kwargs or {}))
        g = -D[best[:, 0], best[:, 1]]
        delta = state.update(order_for_update(best, g))
        delta += state.field_sweep()
        hist.append((state.objective(), delta))
        if callback:
            callback(it, state)
        if delta < eps:
            break
    return hist


def cd(state, eps: float, max_iters: int = 1000):
    """Algorithm 1: every pair i < j in lexicographic order, then a field
    sweep; stop when Delta < eps."""
    p = all_pairs(np.arange(state.N))
    hist = []
    for it in range(max_iters):
        delta = state.update(p) + state.field_sweep()
        hist.append((state.objective(), delta))
        if delta < eps:
            break
    return hist


def recall(found, exact_pairs, exact_gain, rel_floor: float = 1e-6, tol: float = 0.0,
           found_gain=None) -> float:
    """Fraction of the exact best pairs that were found (Sec. IV).  Exact pairs
    whose gain is not above rel_floor * max gain are ties at zero and are left
    out; a found pair whose gain equals the cut gain within tol also counts."""
    exact_pairs = _pairs32(exact_pairs)
    exact_gain = np.asarray(exact_gain, dtype=np.float64)
    if not len(exact_pairs):
        return 1.0
    gmax = exact_gain.max()
    keep = exact_gain > rel_floor * gmax
    ex = exact_pairs[keep]
    if not len(ex):
        return 1.0
    cut = exact_gain[keep].min()
    fset = {(int(a), int(b)) for a, b in _pairs32(found)}
    hits = sum((int(a), int(b)) in fset for a, b in ex)
    if tol > 0 and found_gain is not None:
        extra = sum(1 for (a, b), g in zip(_pairs32(found), found_gain)
                    if abs(g - cut) <= tol and (int(a), int(b)) not in {tuple(e) for e in ex.tolist()})
        hits = min(len(ex), hits + extra)
    return hits / len(ex)
