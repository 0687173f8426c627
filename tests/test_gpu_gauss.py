"""Parity of the CUDA Gaussian (covariance-selection) path against the FP64
oracle, through the C ABI.  Same tolerances as the Ising tests: pair gains
within 1e-5 relative plus 1e-5 x the batch's largest gain, objectives within
1e-6 relative."""
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


def assert_gains(g_gpu, g_ref):
    g_gpu = np.asarray(g_gpu, dtype=np.float64)
    tol = REL * np.abs(g_ref) + FLOOR * max(float(np.max(g_ref)), 1e-30)
    bad = np.abs(g_gpu - g_ref) > tol
    assert not bad.any(), (int(bad.sum()), g_gpu[bad][:5], g_ref[bad][:5])


def _torus(L1, L2, M, seed=4000):
    X = inputs.gaussian_torus_samples(L1, L2, -0.2, 1.8, M, seed)
    return X.astype(np.float32).astype(np.float64)  # the library takes float samples


def _ctx(R, X, lam, **kw):
    return R.Recon(np.ascontiguousarray(X.T.astype(np.float32)), R.RECON_GAUSSIAN, lam=lam, **kw)


@pytest.mark.parametrize("L1,L2,M", [(6, 7, 100), (10, 10, 2000), (5, 9, 37), (1, 2, 1)])
def test_gauss_start_state(R, oracle, L1, L2, M):
    if L1 * L2 < 2:
        pytest.skip()
    X = _torus(L1, L2, M) if L1 > 1 else np.random.default_rng(1).normal(0, 1, (2, M))
    lam = 0.1 * np.sqrt(M)
    ctx = _ctx(R, X, lam)
    o = oracle.GaussOracle(X, lam)
    assert ctx.objective() == pytest.approx(o.objective(), rel=OBJ_REL)
    _, _, s2 = ctx.get_model()
    assert np.allclose(s2, o.s2, rtol=1e-5)
    N = X.shape[0]
    pairs = oracle.all_pairs(np.arange(N))
    d, w = ctx.score(pairs)
    g_ref, w_ref = o.score(pairs)
    assert_gains(-d, g_ref)
    big = g_ref > 1e-3 * max(g_ref.max(), 1e-30)
    assert np.allclose(w[big], w_ref[big], rtol=1e-4, atol=1e-6)


def test_gauss_updates_and_diagonal(R, oracle):
    L1, L2, M = 8, 8, 400
    X = _torus(L1, L2, M)
    N = L1 * L2
    lam = 0.2 * np.sqrt(M)
    ctx = _ctx(R, X, lam)
    o = oracle.GaussOracle(X, lam)
    pairs = oracle.all_pairs(np.arange(N))
    g = np.random.default_rng(3)
    plist = pairs[g.permutation(len(pairs))[:600]]
    d_gpu = ctx.cd_sweep(plist)
    d_ref = o.update(plist)
    assert d_gpu == pytest.approx(d_ref, rel=1e-4)
    assert ctx.objective() == pytest.approx(o.objective(), rel=OBJ_REL)
    assert ctx.field_sweep() == pytest.approx(o.diag_sweep(), rel=1e-3, abs=1e-6)
    _, _, s2 = ctx.get_model()
    assert np.allclose(s2, o.s2, rtol=2e-5)
    assert ctx.objective() == pytest.approx(o.objective(), rel=OBJ_REL)
    assert_gains(-ctx.score(pairs)[0], o.score(pairs)[0])


def test_gauss_gcd_recovers_the_lattice(R):
    """Greedy coordinate descent on the periodic lattice recovers its 4-neighbour
    couplings (negative off-diagonal precision entries)."""
    L1, L2, M = 10, 12, 2000
    X = _torus(L1, L2, M)
    N = L1 * L2
    ctx = _ctx(R, X, 0.05 * np.sqrt(M), knn_mode=R.RECON_KNN_EXHAUSTIVE)
    for _ in range(60):
        delta, obj, m = ctx.gcd_step(8, 2.0)
        if delta < 1e-4:
            break
    ij, w, s2 = ctx.get_model()
    edges = {tuple(e) for e in inputs.torus(L1, L2).tolist()}
    top = ij[np.argsort(w)[:len(edges)]]  # most negative couplings
    prec = np.mean([tuple(p) in edges for p in top.tolist()])
    assert prec > 0.95
    assert np.all(w[np.argsort(w)[:len(edges)]] < 0)


def test_gauss_findbest_exact_knn(R):
    L1, L2, M = 9, 11, 300
    X = _torus(L1, L2, M)
    ctx = _ctx(R, X, 0.05 * np.sqrt(M), knn_mode=R.RECON_KNN_EXHAUSTIVE)
    N = L1 * L2
    p1, d1 = ctx.best_pairs(4, 1.0)
    p2, d2 = ctx.exhaustive_best(N)
    assert np.array_equal(np.sort(d1), np.sort(d2))


def test_gaussian_checkpoint_roundtrip(R, tmp_path):
    """A checkpoint of the Gaussian model (samples rebuilt from the device
    layout) loads into a context that continues exactly as the saved one."""
    X = inputs.gaussian_torus_samples(6, 7, -0.2, 1.8, 150, 4000).astype(np.float32)
    N = X.shape[0]
    ctx = R.Recon(np.ascontiguousarray(X.T), R.RECON_GAUSSIAN, lam=0.5, knn_mode=R.RECON_KNN_EXHAUSTIVE)
    ctx.gcd_step(4, 1.0)
    path = str(tmp_path / "g.bin")
    ctx.save(path)
    c2 = R.recon_load(path)
    a = ctx.gcd_step(4, 1.0)
    b = R.recon_gcd_step(c2, 4, 1.0)
    assert a == b
    ij1, w1, s1 = ctx.get_model()
    ij2, w2, s2 = R.recon_get_model(c2, N)
    assert np.array_equal(ij1, ij2) and np.array_equal(w1, w2) and np.array_equal(s1, s2)
    R.recon_destroy(c2)
