"""Parity of the CUDA Ising path against the FP64 oracle, through the C ABI.

Tolerances (written here, applied element by element): pair gains within
1e-5 relative to the oracle plus an absolute floor of 1e-5 x the largest gain
of the batch (gains at the L1 threshold have no meaningful relative error);
objectives within 1e-6 relative; integer outputs (pair sets) exactly, or by
recall where ties at zero gain make several answers correct."""
import math

import numpy as np
import pytest

from paper_2401_01404_gb300 import inputs

pytestmark = pytest.mark.gpu

REL, FLOOR, OBJ_REL = 1e-5, 1e-5, 1e-6


@pytest.fixture(scope="module")
def R():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__

    __graft_entry__.build()
    from paper_2401_01404_gb300 import recon

    return recon


def _wl(N, M, seed=1000, sweeps=200, h_scale=0.1):
    g = inputs.rng(seed, inputs.GRAPH)
    edges = inputs.erdos_renyi(N, 3, g)
    w = inputs.rng(seed, inputs.COUPLINGS).normal(0, 0.5, len(edges))
    h = inputs.rng(seed, inputs.FIELDS).normal(0, h_scale, N)
    X = inputs.gibbs_ising(N, edges, w, h, M, sweeps, seed)
    return X


def assert_gains(g_gpu, g_ref):
    g_gpu = np.asarray(g_gpu, dtype=np.float64)
    tol = REL * np.abs(g_ref) + FLOOR * max(float(np.max(g_ref)), 1e-30)
    bad = np.abs(g_gpu - g_ref) > tol
    assert not bad.any(), (int(bad.sum()), float(np.max(np.abs(g_gpu - g_ref) - tol)), g_gpu[bad][:5], g_ref[bad][:5])


def _ctx(R, X, lam, **kw):
    return R.Recon(np.ascontiguousarray(X.T), R.RECON_ISING, lam=lam, **kw)


@pytest.mark.parametrize("N,M", [(100, 200), (37, 75), (64, 1000), (2, 1), (5, 33), (40, 1024), (33, 993)])
def test_start_state_matches_oracle(R, oracle, N, M):
    X = _wl(N, M, seed=11 + N + M)
    lam = inputs.default_lambda(max(N, 3), M)
    ctx = _ctx(R, X, lam)
    o = oracle.IsingOracle(X, lam)
    assert ctx.objective() == pytest.approx(o.objective(), rel=OBJ_REL)
    _, _, h = ctx.get_model()
    assert np.allclose(h, o.h, rtol=1e-5, atol=1e-5)
    pairs = oracle.all_pairs(np.arange(N))
    d, w = ctx.score(pairs)
    g_ref, w_ref = o.score(pairs)
    assert_gains(-d, g_ref)
    assert np.allclose(w, w_ref, rtol=1e-3, atol=1e-4)


@pytest.mark.parametrize("c", [0.0, 0.5, 1.0, 2.0])
def test_gains_across_penalties(R, oracle, c):
    N, M = 60, 300
    X = _wl(N, M, seed=5)
    lam = inputs.default_lambda(N, M, c)
    ctx = _ctx(R, X, lam)
    o = oracle.IsingOracle(X, lam, w_clamp=5.0)
    pairs = oracle.all_pairs(np.arange(N))
    assert_gains(-ctx.score(pairs)[0], o.score(pairs)[0])


def _random_state(N, seed, density=0.15, scale=0.4):
    g = np.random.default_rng(seed)
    iu = np.triu_indices(N, 1)
    keep = g.random(len(iu[0])) < density
    ij = np.stack([iu[0][keep], iu[1][keep]], 1).astype(np.int32)
    w = g.normal(0, scale, len(ij)).astype(np.float32)
    h = g.normal(0, 0.3, N).astype(np.float32)
    W = np.zeros((N, N))
    W[ij[:, 0], ij[:, 1]] = w
    W[ij[:, 1], ij[:, 0]] = w
    return ij, w, h, W


@pytest.mark.parametrize("N,M", [(50, 200), (45, 999), (30, 37)])
def test_gains_with_couplings_set(R, oracle, N, M):
    """Pairs already in W are scored too (their update may change or remove
    them)."""
    X = _wl(N, M, seed=7)
    lam = inputs.default_lambda(N, M, 0.7)
    ij, w, h, W = _random_state(N, 8)
    ctx = _ctx(R, X, lam)
    ctx.set_model(ij, w, h)
    o = oracle.IsingOracle(X, lam, w_clamp=5.0)
    o.set_state(W.astype(np.float32).astype(np.float64), h.astype(np.float64))
    assert ctx.objective() == pytest.approx(o.objective(), rel=OBJ_REL)
    pairs = oracle.all_pairs(np.arange(N))
    d, wst = ctx.score(pairs)
    g_ref, w_ref = o.score(pairs)
    assert_gains(-d, g_ref)
    big = g_ref > 1e-3 * g_ref.max()
    assert np.allclose(wst[big], w_ref[big], rtol=2e-3, atol=2e-4)


def test_cd_sweep_equals_sequential_updates(R, oracle):
    """Pairs that share nodes are applied in the given order; the matching
    batches give the same state as the sequential loop of Algorithm 2."""
    N, M = 40, 400
    X = _wl(N, M, seed=21)
    lam = inputs.default_lambda(N, M, 0.5)
    ctx = _ctx(R, X, lam)
    o = oracle.IsingOracle(X, lam, w_clamp=5.0)
    g = np.random.default_rng(22)
    pairs = oracle.all_pairs(np.arange(N))
    order = g.permutation(len(pairs))[:300]
    plist = np.concatenate([pairs[order], pairs[order[:20]]])  # repeats are applied twice
    d_gpu = ctx.cd_sweep(plist)
    d_ref = o.update(plist)
    assert d_gpu == pytest.approx(d_ref, rel=1e-4, abs=1e-6)
    assert ctx.objective() == pytest.approx(o.objective(), rel=OBJ_REL)
    ij, w, _ = ctx.get_model()
    Wg = np.zeros((N, N))
    Wg[ij[:, 0], ij[:, 1]] = w
    assert np.allclose(Wg, np.triu(o.W, 1), atol=2e-4)
    # the field sweep afterwards
    assert ctx.field_sweep() == pytest.approx(o.field_sweep(), rel=1e-3, abs=1e-5)
    _, _, h = ctx.get_model()
    assert np.allclose(h, o.h, atol=2e-5)
    assert ctx.objective() == pytest.approx(o.objective(), rel=OBJ_REL)


def test_gcd_reaches_the_oracle_optimum(R, oracle):
    """Algorithm 2 to convergence on both sides: the objective is convex, so
    both reach the same optimum."""
    N, M = 30, 400
    X = _wl(N, M, seed=31)
    lam = inputs.default_lambda(N, M, 0.5)
    ctx = _ctx(R, X, lam, knn_mode=R.RECON_KNN_EXHAUSTIVE)
    for _ in range(300):
        delta, obj, m = ctx.gcd_step(4, 1.0)
        if delta < 1e-6:
            break
    o = oracle.IsingOracle(X, lam, w_clamp=5.0)
    oracle.gcd(o, kappa=1.0, eps=1e-9, max_iters=3000)
    assert ctx.objective() == pytest.approx(o.objective(), rel=OBJ_REL)
    ij, w, _ = ctx.get_model()
    Wg = np.zeros((N, N))
    Wg[ij[:, 0], ij[:, 1]] = w
    assert np.allclose(Wg, np.triu(o.W, 1), atol=2e-3)


def _exact_top(o, m, N):
    from oracle import oracle as orc

    pairs = orc.all_pairs(np.arange(N))
    g, _ = o.score(pairs)
    order = np.lexsort((pairs[:, 1], pairs[:, 0], -g))
    return pairs[order[:m]], g[order[:m]], pairs, g


@pytest.mark.parametrize("N,M,m", [(100, 200, 100), (64, 500, 300), (90, 128, 20),
                                   # 32-word rows: the segmented scorer's widest instantiation,
                                   # including a ragged last word (993, 600) and a full one (1024)
                                   (160, 600, 150), (150, 1000, 120), (130, 1024, 100), (140, 993, 200)])
def test_exhaustive_best_matches_oracle(R, oracle, N, M, m):
    X = _wl(N, M, seed=41 + m)
    lam = inputs.default_lambda(N, M, 0.5)
    ctx = _ctx(R, X, lam)
    o = oracle.IsingOracle(X, lam, w_clamp=5.0)
    top, gtop, allp, allg = _exact_top(o, m, N)
    p, d = ctx.exhaustive_best(m)
    assert len(p) == m
    assert np.all(p[:, 0] < p[:, 1])
    assert np.all(np.diff(d) >= 0)  # ascending d
    # positive-gain pairs are unique up to float ties at the cut
    gd = dict(zip(map(tuple, allp.tolist()), allg))
    g_found = np.array([gd[tuple(x)] for x in p.tolist()])
    # the gains the segmented all-pairs scorer reported, element by element
    assert_gains(-d, g_found)
    cut = gtop.min()
    strict = {tuple(x) for x, gg in zip(top.tolist(), gtop) if gg > cut * (1 + 1e-4) + 1e-9}
    assert strict <= {tuple(x) for x in p.tolist()}
    assert np.all(g_found >= cut - (REL * cut + FLOOR * allg.max()))


@pytest.mark.parametrize("N,M,kappa", [(100, 200, 1.0), (120, 300, 2.0), (80, 150, 0.5)])
def test_findbest_with_exact_knn_is_exhaustive(R, oracle, N, M, kappa):
    """Lenhof-Smid: FindBest over the exact KNN returns the m best pairs."""
    X = _wl(N, M, seed=51 + N)
    lam = inputs.default_lambda(N, M, 0.3)
    ctx = _ctx(R, X, lam, knn_mode=R.RECON_KNN_EXHAUSTIVE)
    m = int(math.floor(kappa * N + 0.5))
    p1, d1 = ctx.best_pairs(4, kappa)
    p2, d2 = ctx.exhaustive_best(m)
    assert np.allclose(np.sort(d1), np.sort(d2), rtol=0, atol=0)
    pos = d2 < 0
    assert {tuple(x) for x in p2[pos].tolist()} == {tuple(x) for x in p1[d1 < 0].tolist()}
    st = ctx.stats()
    sizes = st["level_size"]
    for t in range(len(sizes) - 1):
        assert sizes[t + 1] <= sizes[t] // 2


def test_findbest_nndescent_recall(R, oracle):
    N, M = 400, 300
    X = _wl(N, M, seed=61)
    lam = inputs.default_lambda(N, M, 0.5)
    ctx = _ctx(R, X, lam, knn_mode=R.RECON_KNN_NNDESCENT)
    o = oracle.IsingOracle(X, lam, w_clamp=5.0)
    m = N
    top, gtop, allp, allg = _exact_top(o, m, N)
    p, d = ctx.best_pairs(10, 1.0)
    assert len(p) == m and np.all(np.diff(d) >= 0)
    rec = oracle.recall(p, top, gtop)
    assert rec >= 0.9, rec
    st = ctx.stats()
    assert st["knn_iters"] >= 1 and st["level_k"][0] >= 10


def test_knn_lists_at_full_size_match_oracle(R, oracle):
    """N=2000, M=1000 (32-word rows): every entry of the first level's k-NN
    lists, whose d the segmented scorer computed inside the NNDescent search
    (launch configuration of the benchmark), against the FP64 oracle at the
    W = 0 start, pair by pair; the lists are ascending, distinct and self-free."""
    wl = inputs.config("ising_n2000_m1000", device="cuda")
    lam = inputs.default_lambda(wl.N, wl.M)
    ctx = R.Recon(wl.samples_major(), R.RECON_ISING, lam=lam, knn_mode=R.RECON_KNN_NNDESCENT)
    ctx.best_pairs(16, 2.0)
    ids, d = ctx.knn_graph()
    assert ids.shape == (wl.N, 16)
    assert np.all(ids >= 0) and np.all(ids != np.arange(wl.N)[:, None])
    assert all(len(set(r)) == len(r) for r in ids.tolist())
    assert np.all(np.diff(d, axis=1) >= 0)
    pairs = np.stack([np.repeat(np.arange(wl.N), 16), ids.ravel()], 1).astype(np.int32)
    h = oracle.ising_fields_at_zero(wl.X)
    phi = np.repeat(h[:, None], wl.M, 1)
    g_ref, _ = oracle.ising_score_rows(wl.X, phi, pairs, lam)
    assert_gains(-d.ravel(), g_ref)
    assert (g_ref > 0).sum() >= wl.N  # the lists hold the planted neighbours, not only zero gains
    st = ctx.stats()
    assert st["knn_iters"] >= 2


def test_invalid_inputs_are_rejected(R):
    X = np.ones((10, 4), dtype=np.int8)
    X[3, 2] = 0
    with pytest.raises(R.ReconError) as e:
        R.Recon(X, R.RECON_ISING, lam=1.0)
    assert e.value.status == R.RECON_EINVAL
    X[3, 2] = -1
    ctx = R.Recon(X, R.RECON_ISING, lam=1.0)
    for bad in ([[0, 4]], [[1, 1]], [[-1, 2]]):
        with pytest.raises(R.ReconError) as e:
            ctx.score(bad)
        assert e.value.status == R.RECON_EINVAL
    d, w = ctx.score(np.zeros((0, 2), dtype=np.int32))
    assert len(d) == 0
    with pytest.raises(R.ReconError) as e:
        R.Recon(np.ones((1025, 3), dtype=np.int8), R.RECON_ISING, lam=1.0)
    assert e.value.status == R.RECON_EUNSUPPORTED


def test_constant_columns_and_tiny_sizes(R, oracle):
    """Degenerate data: a constant spin column (its field goes to the clamp)."""
    N, M = 8, 50
    X = _wl(N, M, seed=71)
    X[2, :] = 1
    X[5, :] = -1
    lam = 2.0
    ctx = _ctx(R, X, lam)
    o = oracle.IsingOracle(X, lam, w_clamp=5.0)
    _, _, h = ctx.get_model()
    assert h[2] == pytest.approx(10.0) and h[5] == pytest.approx(-10.0)
    assert ctx.objective() == pytest.approx(o.objective(), rel=OBJ_REL)
    pairs = oracle.all_pairs(np.arange(N))
    assert_gains(-ctx.score(pairs)[0], o.score(pairs)[0])


def test_checkpoint_roundtrip(R, tmp_path):
    N, M = 50, 100
    X = _wl(N, M, seed=81)
    ctx = _ctx(R, X, 3.0, knn_mode=R.RECON_KNN_EXHAUSTIVE)
    ctx.gcd_step(4, 1.0)
    path = str(tmp_path / "ck.bin")
    ctx.save(path)
    c2 = R.recon_load(path)
    a = ctx.gcd_step(4, 1.0)
    b = R.recon_gcd_step(c2, 4, 1.0)
    # the resumed run continues bit for bit
    assert a == b
    ij1, w1, h1 = ctx.get_model()
    ij2, w2, h2 = R.recon_get_model(c2, N)
    assert np.array_equal(ij1, ij2) and np.array_equal(w1, w2) and np.array_equal(h1, h2)
    R.recon_destroy(c2)


def test_full_size_sampled_pairs(R, oracle):
    """N=2000, M=1000 (random 4-regular, couplings +-0.3): 3000 uniformly random
    pairs and the 1000 best pairs, scored by the CUDA path in the launch the
    search uses, against the oracle one pair at a time."""
    wl = inputs.config("ising_n2000_m1000", device="cuda")
    lam = inputs.default_lambda(wl.N, wl.M)
    ctx = R.Recon(wl.samples_major(), R.RECON_ISING, lam=lam)
    h = oracle.ising_fields_at_zero(wl.X)
    phi = np.repeat(h[:, None], wl.M, 1)
    rp = inputs.random_pairs(wl.N, 3000, 9)
    top, _ = ctx.exhaustive_best(1000)
    pairs = np.concatenate([rp, top])
    d, _ = ctx.score(pairs)
    g_ref, _ = oracle.ising_score_rows(wl.X, phi, pairs, lam)
    assert_gains(-d, g_ref)
    planted = {tuple(e) for e in wl.edges.tolist()}
    assert np.mean([tuple(p) in planted for p in top[:500].tolist()]) > 0.9
