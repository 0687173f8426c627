"""Seeded synthetic inputs for the reconstruction workloads.

This module only *generates data*: planted graphs, their couplings and fields,
and samples drawn from the generative models of App. A (Ising spins by Gibbs
sampling, multivariate-Gaussian samples by an exact spectral sampler).  It holds
none of the reconstruction method's arithmetic (no objective, no pair gain, no
search) and is the one module that both the CUDA path's tests/benchmarks and
the CPU oracle take their inputs from.

Every random stream is keyed: ``seed`` names the workload and ``stream`` names
the derived quantity (graph, couplings, fields, samples, ...), so that each
quantity can be regenerated on its own.  Structure (graph, couplings, fields)
comes from NumPy's Philox generator, which gives identical values on every
platform; the bulk sample draws use torch generators on the requested device.

The paper's empirical datasets are not available; these workloads stand in for
them at the sizes the benchmark configurations name.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# stream ids
GRAPH, COUPLINGS, FIELDS, SAMPLES, SUBSAMPLE, PAIRS, STATE = range(7)


def rng(seed: int, stream: int) -> np.random.Generator:
    """Philox generator keyed by (seed, stream)."""
    return np.random.Generator(np.random.Philox(key=np.array([seed, stream], dtype=np.uint64)))


# ----------------------------------------------------------------------------
# planted graphs (edge lists with a < b)
# ----------------------------------------------------------------------------

def erdos_renyi(N: int, mean_deg: float, g: np.random.Generator) -> np.ndarray:
    """G(N, p) with p = mean_deg/(N-1).  For large N the edge count is drawn
    from its binomial law and the edges are drawn uniformly without
    replacement (rejection of loops and repeats)."""
    p = mean_deg / (N - 1)
    npairs = N * (N - 1) // 2
    if N <= 4000:
        iu = np.triu_indices(N, 1)
        keep = g.random(len(iu[0])) < p
        return np.stack([iu[0][keep], iu[1][keep]], 1).astype(np.int64)
    E = int(g.binomial(npairs, p))
    got = np.empty((0,), dtype=np.int64)
    while len(got) < E:
        need = (E - len(got)) * 11 // 10 + 16
        a = g.integers(0, N, need)
        b = g.integers(0, N, need)
        ok = a != b
        lo, hi = np.minimum(a, b)[ok], np.maximum(a, b)[ok]
        key = lo.astype(np.int64) * N + hi
        got = np.unique(np.concatenate([got, key]))
    got = got[g.permutation(len(got))[:E]]
    got.sort()
    return np.stack([got // N, got % N], 1)


def random_regular(N: int, d: int, g: np.random.Generator, max_tries: int = 100000) -> np.ndarray:
    """Random d-regular simple graph by the configuration model, rejecting
    pairings with loops or repeated edges."""
    assert (N * d) % 2 == 0
    stubs = np.repeat(np.arange(N), d)
    for _ in range(max_tries):
        perm = g.permutation(stubs)
        a, b = perm[0::2], perm[1::2]
        if np.any(a == b):
            continue
        lo, hi = np.minimum(a, b), np.maximum(a, b)
        key = lo.astype(np.int64) * N + hi
        if len(np.unique(key)) != len(key):
            continue
        o = np.argsort(key)
        return np.stack([lo[o], hi[o]], 1).astype(np.int64)
    raise RuntimeError("configuration model failed to produce a simple graph")


def torus(L1: int, L2: int) -> np.ndarray:
    """2-D periodic lattice, node (r, c) -> r*L2 + c, 4 neighbours."""
    r, c = np.meshgrid(np.arange(L1), np.arange(L2), indexing="ij")
    v = (r * L2 + c).ravel()
    right = (r * L2 + (c + 1) % L2).ravel()
    down = (((r + 1) % L1) * L2 + c).ravel()
    e = np.concatenate([np.stack([v, right], 1), np.stack([v, down], 1)])
    e = np.stack([e.min(1), e.max(1)], 1)
    key = np.unique(e[:, 0] * (L1 * L2) + e[:, 1])
    return np.stack([key // (L1 * L2), key % (L1 * L2)], 1).astype(np.int64)


def greedy_coloring(N: int, edges: np.ndarray) -> np.ndarray:
    """Proper vertex colouring, greedy in node order (for chromatic Gibbs)."""
    deg = np.bincount(edges.ravel(), minlength=N)
    off = np.concatenate([[0], np.cumsum(deg)])
    nbr = np.empty(off[-1], dtype=np.int64)
    pos = off[:-1].copy()
    for a, b in ((edges[:, 0], edges[:, 1]), (edges[:, 1], edges[:, 0])):
        order = np.argsort(a, kind="stable")
        a_s, b_s = a[order], b[order]
        cnt = np.bincount(a_s, minlength=N)
        starts = np.concatenate([[0], np.cumsum(cnt)])[:-1]
        idx = np.arange(len(a_s)) - np.repeat(starts, cnt)
        nbr[pos[a_s] + idx] = b_s
        pos += cnt
    color = np.full(N, -1, dtype=np.int64)
    off_l, nbr_l = off.tolist(), nbr.tolist()
    col_l = color.tolist()
    for v in range(N):
        used = {col_l[u] for u in nbr_l[off_l[v]:off_l[v + 1]] if col_l[u] >= 0}
        c = 0
        while c in used:
            c += 1
        col_l[v] = c
    return np.asarray(col_l, dtype=np.int64)


# ----------------------------------------------------------------------------
# samplers
# ----------------------------------------------------------------------------

def gibbs_ising(N: int, edges: np.ndarray, w: np.ndarray, h: np.ndarray, M: int, sweeps: int,
                seed: int, device: str = "cpu") -> np.ndarray:
    """M independent Ising samples (App. A model), each from its own uniform
    random +-1 start followed by `sweeps` Gibbs sweeps.  A sweep visits every
    node once; nodes of one colour class of a proper colouring are conditionally
    independent and are drawn together (a systematic, chromatic scan).  Spin i
    is set to +1 with probability 1/(1 + exp(-2 f_i)), f_i = h_i + sum_j w_ij x_j.
    Returns int8, node-major (N x M)."""
    import torch

    color = greedy_coloring(N, edges)
    ncol = int(color.max()) + 1 if N else 0
    dev = torch.device(device)
    gen = torch.Generator(device=dev)
    gen.manual_seed(int(rng(seed, SAMPLES).integers(0, 2**62)))
    X = (torch.randint(0, 2, (N, M), generator=gen, device=dev, dtype=torch.int8) * 2 - 1).float()
    a = np.concatenate([edges[:, 0], edges[:, 1]])
    b = np.concatenate([edges[:, 1], edges[:, 0]])
    ww = np.concatenate([w, w])
    classes = []
    for c in range(ncol):
        nodes = np.nonzero(color == c)[0]
        local = np.full(N, -1, dtype=np.int64)
        local[nodes] = np.arange(len(nodes))
        sel = color[a] == c
        classes.append((torch.as_tensor(nodes, device=dev),
                        torch.as_tensor(local[a[sel]], device=dev),
                        torch.as_tensor(b[sel], device=dev),
                        torch.as_tensor(ww[sel], dtype=torch.float32, device=dev).unsqueeze(1),
                        torch.as_tensor(h[nodes], dtype=torch.float32, device=dev).unsqueeze(1)))
    for _ in range(sweeps):
        for nodes, tgt, src, wc, hc in classes:
            f = hc.expand(len(nodes), M).clone()
            if len(tgt):
                f.index_add_(0, tgt, wc * X[src])
            u = torch.rand((len(nodes), M), generator=gen, device=dev)
            X[nodes] = torch.where(u * (1.0 + torch.exp(-2.0 * f)) < 1.0, 1.0, -1.0)
    return X.to(torch.int8).cpu().numpy()


def gaussian_torus_samples(L1: int, L2: int, off: float, diag: float, M: int, seed: int) -> np.ndarray:
    """Exact samples of N(0, Q^-1) for the periodic-lattice precision matrix
    Q = diag*I + off*A (A the 4-neighbour torus adjacency), which is
    block-circulant: x = F^-1[ F[z] / sqrt(eig) ] with z white noise and
    eig(a,b) = diag + 2 off cos(2 pi a/L1) + 2 off cos(2 pi b/L2).
    Returns float64, node-major (N x M), node (r,c) -> r*L2 + c."""
    g = rng(seed, SAMPLES)
    a = np.arange(L1)[:, None]
    b = np.arange(L2)[None, :]
    eig = diag + 2 * off * np.cos(2 * np.pi * a / L1) + 2 * off * np.cos(2 * np.pi * b / L2)
    assert eig.min() > 0
    z = g.standard_normal((M, L1, L2))
    x = np.fft.ifft2(np.fft.fft2(z) / np.sqrt(eig)[None]).real
    return np.ascontiguousarray(x.reshape(M, L1 * L2).T)


def gaussian_dense_samples(Q: np.ndarray, M: int, seed: int) -> np.ndarray:
    """Samples of N(0, Q^-1) through the Cholesky factor Q = L L^T:
    x = L^-T z.  Node-major (N x M), float64."""
    g = rng(seed, SAMPLES)
    L = np.linalg.cholesky(Q)
    z = g.standard_normal((Q.shape[0], M))
    import scipy.linalg

    return scipy.linalg.solve_triangular(L.T, z, lower=False)


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------

def gaussian_er_precision(N: int, deg: float, mean: float, std: float, eps: float, seed: int):
    """The paper's synthetic Gaussian model (its runtime and convergence
    studies): off-diagonal precision entries on an Erdos-Renyi graph of mean
    degree `deg`, each ~ N(mean, std^2), and W_ii = sum_j |W_ij| / (1 - eps)^2,
    so W is diagonally dominant and positive definite.  A node without edges
    would get W_ii = 0 (an improper variable); it takes the median diagonal of
    the others, so that its variance is of the same order as theirs.
    Returns (edges [E x 2], off-diagonal values [E], diagonal [N])."""
    edges = erdos_renyi(N, deg, rng(seed, GRAPH))
    w = rng(seed, COUPLINGS).normal(mean, std, len(edges))
    rowsum = np.bincount(edges[:, 0], np.abs(w), minlength=N) + np.bincount(edges[:, 1], np.abs(w), minlength=N)
    diag = rowsum / (1.0 - eps) ** 2
    diag[rowsum == 0] = np.median(diag[rowsum > 0]) if (rowsum > 0).any() else 1.0
    return edges, w, diag


def gaussian_precision_samples(N: int, edges: np.ndarray, w: np.ndarray, diag: np.ndarray, M: int, seed: int,
                               device: str = "cpu", tol: float = 1e-10, max_iter: int = 20000) -> np.ndarray:
    """M exact samples of N(0, W^-1) for a sparse diagonally dominant W.
    W = B^T B with one row sqrt|w_ij| (e_i + sign(w_ij) e_j) per edge and one row
    sqrt(r_i) e_i per node (r_i = W_ii - sum_j |W_ij| >= 0), so b = B^T z with z
    white noise is N(0, W), and x = W^-1 b is N(0, W^-1).  The M systems W x = b
    are solved together by conjugate gradients in float64 (torch, on `device`)
    to a relative residual of `tol`.  Returns float64, node-major (N x M)."""
    import torch

    dev = torch.device(device)
    E = len(edges)
    i = torch.as_tensor(edges[:, 0], device=dev)
    j = torch.as_tensor(edges[:, 1], device=dev)
    wt = torch.as_tensor(w, dtype=torch.float64, device=dev)
    dg = torch.as_tensor(diag, dtype=torch.float64, device=dev)
    absw = wt.abs()
    r = dg - (torch.zeros(N, dtype=torch.float64, device=dev).index_add_(0, i, absw).index_add_(0, j, absw))
    r = r.clamp_min(0.0)
    gen = torch.Generator(device=dev)
    gen.manual_seed(int(rng(seed, SAMPLES).integers(0, 2**62)))
    ze = torch.randn((E, M), generator=gen, dtype=torch.float64, device=dev)
    zn = torch.randn((N, M), generator=gen, dtype=torch.float64, device=dev)
    se = absw.sqrt().unsqueeze(1) * ze
    b = r.sqrt().unsqueeze(1) * zn
    b.index_add_(0, i, se)
    b.index_add_(0, j, torch.sign(wt).unsqueeze(1) * se)
    rows = torch.cat([i, j, torch.arange(N, device=dev)])
    cols = torch.cat([j, i, torch.arange(N, device=dev)])
    vals = torch.cat([wt, wt, dg])
    Wm = torch.sparse_coo_tensor(torch.stack([rows, cols]), vals, (N, N), check_invariants=True).coalesce()
    x = torch.zeros_like(b)
    res = b.clone()
    p = res.clone()
    rr = (res * res).sum(0)
    b2 = rr.clone()
    for _ in range(max_iter):
        if bool((rr <= tol * tol * b2).all()):
            break
        Ap = torch.sparse.mm(Wm, p)
        alpha = rr / (p * Ap).sum(0)
        x += alpha * p
        res -= alpha * Ap
        rr_new = (res * res).sum(0)
        p = res + (rr_new / rr) * p
        rr = rr_new
    return x.cpu().numpy()


@dataclass
class Workload:
    name: str
    model: str               # "ising" | "gaussian"
    N: int
    M: int
    X: np.ndarray             # node-major, int8 (ising) or float64 (gaussian)
    edges: np.ndarray         # planted graph (a < b)
    w: np.ndarray             # planted off-diagonal couplings
    h: np.ndarray             # planted fields (ising) / diagonal (gaussian)
    k: int = 16
    kappa: float = 1.0
    extra: dict = field(default_factory=dict)
    lam: float = 0.0          # the penalty this workload is run with

    def __post_init__(self):
        if not self.lam:
            self.lam = default_lambda(self.N, self.M)

    def samples_major(self) -> np.ndarray:
        """The samples as the public API takes them: sample-major M x N."""
        return np.ascontiguousarray(self.X.T)


def ising_workload(name: str, N: int, M: int, graph: str, deg: float, coupling: str, coup_scale: float,
                   field_scale: float, sweeps: int, seed: int, k: int, kappa: float,
                   device: str = "cpu") -> Workload:
    gg = rng(seed, GRAPH)
    if graph == "er":
        edges = erdos_renyi(N, deg, gg)
    elif graph == "regular":
        edges = random_regular(N, int(deg), gg)
    else:
        raise ValueError(graph)
    gc = rng(seed, COUPLINGS)
    if coupling == "normal":
        w = gc.normal(0.0, coup_scale, len(edges))
    else:  # "pm": random sign, fixed magnitude
        w = coup_scale * (2.0 * (gc.random(len(edges)) < 0.5) - 1.0)
    h = rng(seed, FIELDS).normal(0.0, field_scale, N) if field_scale > 0 else np.zeros(N)
    X = gibbs_ising(N, edges, w, h, M, sweeps, seed, device=device)
    return Workload(name, "ising", N, M, X, edges, w, h, k=k, kappa=kappa)


def config(name: str, device: str = "cpu", sweeps: int | None = None, M: int | None = None,
           N: int | None = None) -> Workload:
    """The benchmark workloads, by name:

    ising_n100_m200   : N=100, M=200, Erdos-Renyi mean degree 3, w ~ N(0, 0.5^2),
                        h ~ N(0, 0.1^2), 1000 Gibbs sweeps; k=10, kappa=1.
    ising_n2000_m1000 : N=2000, M=1000, random 4-regular, w = +-0.3, h = 0; k=16, kappa=2.
    ising_n1e5_m500   : N=100000, M=500, Erdos-Renyi mean degree 5, w ~ N(0, 0.3^2), h = 0.
    gauss_n20000_m2000: N=20000 (100 x 200 torus), M=2000, off-diagonal -0.2,
                        diagonal 1.0 + sum|off| = 1.8; per-node k drawn from 8..64.
    ising_n1e6_m200   : N=1000000, M=200, Erdos-Renyi mean degree 5, w ~ N(0, 0.3^2), h = 0;
                        k=16, kappa=1.
    Penalty: lambda = c sqrt(2 M ln N) with c = 1, except c = 2 for the two large
    Ising workloads: there c = 1 would leave about 1% of all N^2/2 pairs (pure
    sampling noise, |g| above lambda) with a nonzero optimum, while c = 2 keeps
    that number O(N) (the union bound over the pairs), the sparsity the penalty is
    there for.
    Optional overrides shrink a workload for tests (N, M, sweeps)."""
    if name == "ising_n100_m200":
        return ising_workload(name, N or 100, M or 200, "er", 3, "normal", 0.5, 0.1,
                              sweeps or 1000, 1000, 10, 1.0, device)
    if name == "ising_n2000_m1000":
        return ising_workload(name, N or 2000, M or 1000, "regular", 4, "pm", 0.3, 0.0,
                              sweeps or 1000, 2000, 16, 2.0, device)
    if name == "ising_n1e5_m500":
        wl = ising_workload(name, N or 100000, M or 500, "er", 5, "normal", 0.3, 0.0,
                            sweeps or 1000, 3000, 16, 1.0, device)
        wl.lam = default_lambda(wl.N, wl.M, 2.0)
        return wl
    if name == "ising_n1e6_m200":
        wl = ising_workload(name, N or 1000000, M or 200, "er", 5, "normal", 0.3, 0.0,
                            sweeps or 1000, 5000, 16, 1.0, device)
        wl.lam = default_lambda(wl.N, wl.M, 2.0)
        return wl
    if name == "gauss_n20000_m2000":
        L1, L2 = (100, 200) if N is None else (int(math.isqrt(N // 2)), N // int(math.isqrt(N // 2)))
        MM = M or 2000
        X = gaussian_torus_samples(L1, L2, -0.2, 1.8, MM, 4000)
        edges = torus(L1, L2)
        kk = rng(4000, STATE).integers(8, 65, L1 * L2)
        return Workload(name, "gaussian", L1 * L2, MM, X, edges, np.full(len(edges), -0.2),
                        np.full(L1 * L2, 1.8), k=16, kappa=1.0, extra={"k_per_node": kk})
    raise ValueError(name)


def default_lambda(N: int, M: int, c: float = 1.0) -> float:
    """Penalty lambda = c*sqrt(2 M ln N), the usual l1-logistic scaling for a
    log-likelihood summed over M samples (the paper leaves lambda to the user)."""
    return c * math.sqrt(2.0 * M * math.log(N))


def random_pairs(N: int, P: int, seed: int, stream: int = PAIRS) -> np.ndarray:
    """P uniformly random unordered pairs (a < b), int32 (P x 2)."""
    g = rng(seed, stream)
    a = g.integers(0, N, 2 * P + 16)
    b = g.integers(0, N, 2 * P + 16)
    ok = a != b
    a, b = a[ok][:P], b[ok][:P]
    return np.stack([np.minimum(a, b), np.maximum(a, b)], 1).astype(np.int32)
