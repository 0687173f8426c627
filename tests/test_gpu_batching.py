"""The batching workload: the multivariate-Gaussian model on a 100 x 200
periodic lattice (N=20,000, M=2,000 samples), NNDescent lists of uneven length
k_i drawn from 8..64 per node, scored by the segmented scorer (one block per
node's candidate list, block width picked by the autotuner).  Checked against
the FP64 oracle on sampled pairs and against the exact best pairs of the
tensor-core screen."""
import math

import numpy as np
import pytest

from paper_2401_01404_gb300 import inputs

pytestmark = pytest.mark.gpu

REL, FLOOR = 1e-5, 1e-5


@pytest.fixture(scope="module")
def R():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__

    __graft_entry__.build()
    from paper_2401_01404_gb300 import recon

    return recon


@pytest.fixture(scope="module")
def c4():
    return inputs.config("gauss_n20000_m2000")


def test_uneven_lists_on_the_lattice(R, oracle, c4):
    wl = c4
    Xs = np.ascontiguousarray(wl.X.T.astype(np.float32))
    lam = wl.lam
    nnd = R.Recon(Xs, R.RECON_GAUSSIAN, lam=lam, timing=1)
    kk = wl.extra["k_per_node"]
    assert kk.min() >= 8 and kk.max() <= 64
    R.recon_set_list_lengths(nnd.ctx, kk)
    p, d = nnd.best_pairs(8, 1.0)
    st = nnd.stats()
    assert st["level_k"][0] == int(kk.max())
    assert st["tuned_threads"] in (64, 128, 256, 512)
    assert len(p) == wl.N and np.all(p[:, 0] < p[:, 1]) and np.all(np.diff(d) >= 0)
    # exact best pairs through the screen
    scr = R.Recon(Xs, R.RECON_GAUSSIAN, lam=lam, knn_mode=R.RECON_KNN_SCREEN)
    pe, de = scr.best_pairs(8, 1.0)
    # NNDescent never reports a pair better than the exact best
    assert d.min() >= de.min() - 1e-5 * abs(de.min())
    ge = -de.astype(np.float64)
    truth = {tuple(x) for x, g in zip(pe.tolist(), ge) if g > 1e-6 * ge.max()}
    rec = len(truth & {tuple(x) for x in p.tolist()}) / max(len(truth), 1)
    print("uneven-list NNDescent recall on the lattice:", rec)
    # On a lattice only the 4 lattice neighbours carry gain, so a node's first true
    # neighbour is found by chance (probability ~ k^2 / N per iteration): the FP64
    # sequential NNDescent of the oracle falls, at k = 36, from 0.99 (N = 1,200)
    # to 0.71 (N = 4,800) and 0.43 (N = 10,000); at k = 16 from 0.64 to 0.14.
    # Here N = 20,000 with k_i in 8..64: a low recall is the method's, and the
    # exact screen is the path for lattices.
    assert rec > 0.1, rec
    # the lattice edges lead the exact list
    edges = {tuple(e) for e in wl.edges.tolist()}
    assert np.mean([tuple(x) in edges for x in pe[:len(truth)].tolist()]) > 0.95
    # sampled pairs against the oracle (Gaussian gains at the W = 0 start)
    pairs = np.concatenate([inputs.random_pairs(wl.N, 3000, 13), pe[:2000]])
    dg, _ = nnd.score(pairs)
    X64 = Xs.T.astype(np.float64)
    s2 = oracle.gauss_diag_at_zero(X64)
    g_ref, _ = oracle.gauss_score_rows(X64, np.zeros_like(X64), s2, pairs, lam)
    tol = REL * np.abs(g_ref) + FLOOR * g_ref.max()
    assert np.all(np.abs(-dg.astype(np.float64) - g_ref) <= tol)


def test_small_torus_recall_matches_the_oracle(R, oracle):
    """On a 30 x 40 torus (N = 1,200) with lists of k = 36 the oracle's sequential
    NNDescent finds 0.99 of the exact best N pairs; the batch form must too."""
    L1, L2, M = 30, 40, 2000
    X = inputs.gaussian_torus_samples(L1, L2, -0.2, 1.8, M, 4000)
    N = L1 * L2
    lam = inputs.default_lambda(N, M)
    Xs = np.ascontiguousarray(X.T.astype(np.float32))
    scr = R.Recon(Xs, R.RECON_GAUSSIAN, lam=lam, knn_mode=R.RECON_KNN_SCREEN)
    pe, de = scr.best_pairs(36, 1.0)
    ge = -de.astype(np.float64)
    truth = {tuple(x) for x, g in zip(pe.tolist(), ge) if g > 1e-6 * ge.max()}
    recs = []
    for seed in (3, 4):
        c = R.Recon(Xs, R.RECON_GAUSSIAN, lam=lam, seed=seed, max_knn_iters=30)
        p, _ = c.best_pairs(36, 1.0)
        recs.append(len(truth & {tuple(x) for x in p.tolist()}) / len(truth))
    assert min(recs) > 0.95, recs


def test_uneven_lists_ising(R):
    """Per-node lengths on the Ising model: recall against the exact best pairs
    rises with the lengths."""
    N, M = 1500, 600
    wl = inputs.ising_workload("t", N, M, "regular", 4, "pm", 0.3, 0.0, 200, 2200, 16, 2.0, device="cuda")
    lam = inputs.default_lambda(N, M)
    Xs = wl.samples_major()
    scr = R.Recon(Xs, R.RECON_ISING, lam=lam, knn_mode=R.RECON_KNN_SCREEN)
    pe, de = scr.best_pairs(16, 2.0)
    ge = -de.astype(np.float64)
    truth = {tuple(x) for x, g in zip(pe.tolist(), ge) if g > 1e-6 * ge.max()}
    recs = []
    for lo, hi in ((8, 16), (32, 64)):
        c = R.Recon(Xs, R.RECON_ISING, lam=lam, seed=3)
        R.recon_set_list_lengths(c.ctx, inputs.rng(5, inputs.STATE).integers(lo, hi + 1, N))
        p, _ = c.best_pairs(8, 2.0)
        recs.append(len(truth & {tuple(x) for x in p.tolist()}) / len(truth))
    assert recs[1] > recs[0] and recs[1] > 0.97, recs


def _check_lists(R, ctx, klen=None):
    """The first-level lists: ids distinct, in range and not the node itself,
    ascending in d, each d the pair's score, padding past k_i."""
    ids, d = ctx.knn_graph()
    n, K = ids.shape
    assert n > 0 and K > 0
    klen = np.full(n, K) if klen is None else np.asarray(klen)
    pad = np.arange(K)[None, :] >= klen[:, None]
    assert np.all(ids[pad] == -1) and np.all(np.isinf(d[pad]))
    live = ~pad
    rows = np.broadcast_to(np.arange(n)[:, None], ids.shape)
    assert np.all((ids[live] >= 0) & (ids[live] < n) & (ids[live] != rows[live]))
    for r in range(n):
        row = ids[r, :klen[r]]
        assert len(set(row.tolist())) == len(row), r
    dl = np.where(live, d, np.inf)
    assert np.all(dl[:, 1:] >= dl[:, :-1]), np.argwhere(dl[:, 1:] < dl[:, :-1])[:5]
    pairs = np.stack([np.minimum(rows[live], ids[live]), np.maximum(rows[live], ids[live])], 1).astype(np.int32)
    ds, _ = ctx.score(pairs)
    assert np.allclose(ds, d[live], rtol=1e-5, atol=1e-5 * np.abs(ds).max())


def test_knn_graph_invariants(R):
    L1, L2, M = 30, 40, 2000
    X = inputs.gaussian_torus_samples(L1, L2, -0.2, 1.8, M, 4000)
    N = L1 * L2
    Xs = np.ascontiguousarray(X.T.astype(np.float32))
    g = R.Recon(Xs, R.RECON_GAUSSIAN, lam=inputs.default_lambda(N, M), seed=3)
    for k, iters in ((36, 1), (36, 3), (16, 5)):
        g2 = R.Recon(Xs, R.RECON_GAUSSIAN, lam=inputs.default_lambda(N, M), seed=3, max_knn_iters=iters, eps_knn=0.0)
        g2.best_pairs(k, 1.0)
        _check_lists(R, g2)
    wl = inputs.ising_workload("t", 900, 400, "regular", 4, "pm", 0.3, 0.0, 100, 2300, 16, 2.0, device="cuda")
    c = R.Recon(wl.samples_major(), R.RECON_ISING, lam=inputs.default_lambda(900, 400), seed=5)
    kk = inputs.rng(6, inputs.STATE).integers(8, 41, 900)
    R.recon_set_list_lengths(c.ctx, kk)
    c.best_pairs(8, 2.0)
    _check_lists(R, c, np.maximum(kk, -(-4 * 1800 // 900)))
    # a search that goes on to a second level keeps the first level's lists: 20
    # near-copies of one spin row form a clique whose members' lists hold only
    # clique partners, all among the best 2m edges (saturated, Algorithm 3)
    X = np.array(wl.X, copy=True)
    flip = np.random.default_rng(8).random((19, X.shape[1])) < 0.05
    X[1:20] = np.where(flip, -X[0], X[0])
    c2 = R.Recon(np.ascontiguousarray(X.T), R.RECON_ISING, lam=inputs.default_lambda(900, 400), seed=5)
    c2.best_pairs(8, 2.0)
    st = c2.stats()
    assert st["level_size"][1] >= 20, st["level_size"][:3]
    ids, _ = c2.knn_graph()
    assert ids.shape == (900, 8)
    _check_lists(R, c2)
    # the screen builds no lists
    s = R.Recon(Xs, R.RECON_GAUSSIAN, lam=1.0, knn_mode=R.RECON_KNN_SCREEN)
    s.best_pairs(8, 1.0)
    ids, d = s.knn_graph()
    assert ids.size == 0
