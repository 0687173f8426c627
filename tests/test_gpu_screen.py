"""The tensor-core gradient screen (RECON_KNN_SCREEN): its best pairs must be
the exact best pairs — the screen only discards pairs whose gain is provably
zero, and the survivors are scored exactly.  Checked against the oracle and
against the CUDA-core exhaustive search, element by element, on sizes with
ragged tiles (N not a multiple of 128, M not a multiple of 64).  Three forms:
the general one with bf16 operands, the same with FP8 (E4M3) operands (a wider
margin keeps it exact), and the rank-one form of the empty network (E4M3 spin
product, exact; the library's default whenever no coupling is stored)."""
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


def _wl(N, M, seed):
    edges = inputs.erdos_renyi(N, 3, inputs.rng(seed, inputs.GRAPH))
    w = inputs.rng(seed, inputs.COUPLINGS).normal(0, 0.5, len(edges))
    h = inputs.rng(seed, inputs.FIELDS).normal(0, 0.1, N)
    return inputs.gibbs_ising(N, edges, w, h, M, 150, seed)


# screen forms: options of each (the general forms are forced off the rank-one path)
FORMS = {"bf16": dict(screen_fp8=0, screen_no_rank1=1), "fp8": dict(screen_fp8=1, screen_no_rank1=1),
         "rank1": dict(screen_fp8=0, screen_no_rank1=0)}


def _grad_at_zero(X, oracle):
    """F'(0) of every pair at the W = 0 start: sum_m [x_j (x_i - t_i) + x_i (x_j - t_j)]
    with t_i = tanh(h_i) and h the oracle's fitted fields."""
    t = np.tanh(oracle.ising_fields_at_zero(X))
    Xf = X.astype(np.float64)
    s = Xf.sum(1)
    return 2.0 * Xf @ Xf.T - np.outer(s, t) - np.outer(t, s)


def _close(g_gpu, g_ref):
    tol = REL * np.abs(g_ref) + FLOOR * max(float(np.max(g_ref)), 1e-30)
    return np.abs(np.asarray(g_gpu, dtype=np.float64) - g_ref) <= tol


@pytest.mark.parametrize("form", ["bf16", "fp8", "rank1"])
@pytest.mark.parametrize("N,M,c", [(100, 200, 1.0), (300, 130, 0.5), (257, 1000, 1.0), (129, 37, 0.7),
                                   (200, 256, 1.0), (140, 1024, 1.0)])
def test_screen_keeps_every_pair_with_a_gain(R, oracle, N, M, c, form):
    X = _wl(N, M, 100 + N)
    lam = inputs.default_lambda(N, M, c)
    o = oracle.IsingOracle(X, lam)
    allp = oracle.all_pairs(np.arange(N))
    g_ref, _ = o.score(allp)
    npos = int((g_ref > 1e-6 * g_ref.max()).sum())
    scr = R.Recon(np.ascontiguousarray(X.T), R.RECON_ISING, lam=lam, knn_mode=R.RECON_KNN_SCREEN, timing=1,
                  **FORMS[form])
    kappa = (len(allp) + 0.4) / N  # ask for every pair: the screen returns exactly its survivors
    p, d = scr.best_pairs(4, kappa)
    found = {tuple(x) for x in p.tolist()}
    pos = {tuple(x) for x, g in zip(allp.tolist(), g_ref) if g > 1e-6 * g_ref.max()}
    assert pos <= found, len(pos - found)
    st = scr.stats()
    assert st["screen_launches"] == 1 and st["screen_survivors"] == len(p)
    assert st["screen_rank1"] == (1 if form == "rank1" else 0)
    if form != "fp8":
        assert len(p) < len(allp) or npos > len(allp) // 2  # the screen discarded pairs
    if form == "rank1":
        # the rank-one form is exact up to its small margin (Mp / 2048): its survivors
        # are the pairs with |F'(0)| above lambda minus that margin, and no others
        G = _grad_at_zero(X, oracle)[allp[:, 0], allp[:, 1]]
        mp = 32 * ((M + 31) // 32)
        must = int((np.abs(G) > lam + 1e-3).sum())
        may = int((np.abs(G) > lam - mp / 2048.0 - 1e-3).sum())
        assert must <= len(p) <= may, (must, len(p), may)
    gd = dict(zip(map(tuple, allp.tolist()), g_ref))
    assert _close(-d, np.array([gd[x] for x in map(tuple, p.tolist())])).all()


@pytest.mark.parametrize("form", ["bf16", "fp8", "rank1"])
@pytest.mark.parametrize("N,M,kappa", [(200, 300, 1.0), (500, 500, 2.0), (1100, 250, 1.0)])
def test_screen_best_equals_exhaustive(R, N, M, kappa, form):
    X = _wl(N, M, 200 + N)
    lam = inputs.default_lambda(N, M)
    Xs = np.ascontiguousarray(X.T)
    scr = R.Recon(Xs, R.RECON_ISING, lam=lam, knn_mode=R.RECON_KNN_SCREEN, **FORMS[form])
    ex = R.Recon(Xs, R.RECON_ISING, lam=lam)
    m = int(math.floor(kappa * N + 0.5))
    p1, d1 = scr.best_pairs(8, kappa)
    p2, d2 = ex.exhaustive_best(m)
    pos2 = d2 < -1e-6 * max(-d2.min(), 1e-30)
    # every positive-gain pair of the exact answer, except float ties at the cut
    cut = d2[pos2].max() if pos2.any() else 0.0
    strict = {tuple(x) for x, dv in zip(p2.tolist(), d2) if dv < cut - 1e-4 * abs(cut)}
    assert strict <= {tuple(x) for x in p1.tolist()}
    n = min(len(d1), len(d2))
    assert np.allclose(d1[:n], d2[:n], rtol=1e-5, atol=1e-5 * abs(d2.min()))


@pytest.mark.parametrize("form", ["bf16", "fp8", "rank1"])
def test_screen_with_couplings_and_in_gcd(R, oracle, form):
    """After GCD steps W is nonzero: stored couplings are rescored too, and a
    screen-driven GCD reaches the oracle's optimum (the rank-one form runs at
    the first step only, the general bf16 form after it)."""
    N, M = 60, 300
    X = _wl(N, M, 301)
    lam = inputs.default_lambda(N, M, 0.5)
    scr = R.Recon(np.ascontiguousarray(X.T), R.RECON_ISING, lam=lam, knn_mode=R.RECON_KNN_SCREEN,
                  **FORMS[form])
    for _ in range(400):
        delta, obj, m = scr.gcd_step(4, 1.0)
        if delta < 1e-6:
            break
    o = oracle.IsingOracle(X, lam)
    oracle.gcd(o, kappa=1.0, eps=1e-9, max_iters=3000)
    assert scr.objective() == pytest.approx(o.objective(), rel=1e-6)
    assert scr.stats()["screen_rank1"] == (1 if form == "rank1" else 0)


def test_screen_gaussian(R, oracle):
    L1, L2, M = 9, 13, 300
    X = inputs.gaussian_torus_samples(L1, L2, -0.2, 1.8, M, 4000).astype(np.float32).astype(np.float64)
    N = L1 * L2
    lam = 0.05 * math.sqrt(M)
    o = oracle.GaussOracle(X, lam)
    allp = oracle.all_pairs(np.arange(N))
    g_ref, _ = o.score(allp)
    scr = R.Recon(np.ascontiguousarray(X.T.astype(np.float32)), R.RECON_GAUSSIAN, lam=lam,
                  knn_mode=R.RECON_KNN_SCREEN)
    p, d = scr.best_pairs(4, (len(allp) + 0.4) / N)
    found = {tuple(x) for x in p.tolist()}
    pos = {tuple(x) for x, g in zip(allp.tolist(), g_ref) if g > 1e-6 * g_ref.max()}
    assert pos <= found


def test_screen_forms_agree_on_a_larger_lattice(R):
    """Several hundred tiles, M = 200 (K = 448: the fp8 rows end in a half
    k-block; the rank-one rows in 224 of 256 entries): every form gives the same
    positive-gain best pairs, the fp8 margin only adds survivors, and the
    rank-one form keeps the fewest."""
    N, M = 6000, 200
    edges = inputs.erdos_renyi(N, 3, inputs.rng(7, inputs.GRAPH))
    w = inputs.rng(7, inputs.COUPLINGS).normal(0, 0.5, len(edges))
    X = inputs.gibbs_ising(N, edges, w, np.zeros(N), M, 100, 7)
    Xs = np.ascontiguousarray(X.T)
    lam = inputs.default_lambda(N, M)
    out = {}
    for form in FORMS:
        c = R.Recon(Xs, R.RECON_ISING, lam=lam, knn_mode=R.RECON_KNN_SCREEN, **FORMS[form])
        p, d = c.best_pairs(16, 1.0)
        out[form] = (p, d, c.stats()["screen_survivors"])
        c.close()
    s_b, s_f, s_r = out["bf16"][2], out["fp8"][2], out["rank1"][2]
    assert s_f >= s_b >= s_r
    p0, d0, _ = out["bf16"]
    pos0 = {tuple(x) for x, dv in zip(p0.tolist(), d0) if dv < 0}
    for form in ("fp8", "rank1"):
        p1, d1, _ = out[form]
        assert np.array_equal(d0, d1)
        assert pos0 == {tuple(x) for x, dv in zip(p1.tolist(), d1) if dv < 0}


@pytest.mark.parametrize("form", ["bf16", "fp8", "rank1"])
@pytest.mark.parametrize("N,M", [(129, 37), (300, 130), (700, 1000), (2600, 200)])
def test_pair_form_equals_single_cta_form(R, N, M, form):
    """The CTA-pair screen (one M = 256 MMA per super-tile over a cluster of two
    CTAs) keeps exactly the single-CTA screen's survivors, with the same exact
    gains: ragged last super-tiles (N not a multiple of 256), a single
    super-tile, K from one to 32 k-blocks."""
    X = _wl(N, M, 500 + N)
    lam = inputs.default_lambda(N, M, 0.7)
    Xs = np.ascontiguousarray(X.T)
    out = []
    for pair in (1, 0):
        c = R.Recon(Xs, R.RECON_ISING, lam=lam, knn_mode=R.RECON_KNN_SCREEN, screen_pair=pair,
                    timing=1, **FORMS[form])
        kappa = (N * (N - 1) / 2 + 0.4) / N  # every survivor comes back
        p, d = c.best_pairs(4, kappa)
        st = c.stats()
        assert st["screen_survivors"] == len(p) and st["screen_launches"] == 1
        order = np.lexsort((p[:, 1], p[:, 0]))
        out.append((p[order], d[order]))
        c.close()
    assert len(out[0][0]) > 0
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])


def test_fp8_screen_is_refused_for_the_gaussian_model(R):
    X = np.ones((20, 6), dtype=np.float32)
    with pytest.raises(R.ReconError) as e:
        R.Recon(X, R.RECON_GAUSSIAN, lam=1.0, knn_mode=R.RECON_KNN_SCREEN, screen_fp8=1)
    assert e.value.status == R.RECON_EUNSUPPORTED


@pytest.mark.parametrize("form", ["bf16", "fp8"])
def test_screen_after_gcd_steps_equals_exhaustive(R, form):
    """With couplings set (residuals vary per sample, so every rounding error
    differs), the screen's best pairs still equal the exhaustive search's."""
    N, M = 700, 400
    X = _wl(N, M, 77)
    Xs = np.ascontiguousarray(X.T)
    lam = inputs.default_lambda(N, M)
    scr = R.Recon(Xs, R.RECON_ISING, lam=lam, knn_mode=R.RECON_KNN_SCREEN, **FORMS[form])
    for _ in range(3):
        scr.gcd_step(8, 1.0)
    ij, w, h = scr.get_model()
    assert len(ij) > 0
    ex = R.Recon(Xs, R.RECON_ISING, lam=lam)
    ex.set_model(ij, w, h)
    p1, d1 = scr.best_pairs(8, 1.0)
    p2, d2 = ex.exhaustive_best(N)
    pos2 = d2 < -1e-6 * max(-d2.min(), 1e-30)
    cut = d2[pos2].max() if pos2.any() else 0.0
    strict = {tuple(x) for x, dv in zip(p2.tolist(), d2) if dv < cut - 1e-4 * abs(cut)}
    assert strict <= {tuple(x) for x in p1.tolist()}
    n = min(len(d1), len(d2))
    assert np.allclose(d1[:n], d2[:n], rtol=1e-5, atol=1e-5 * abs(d2.min()))
