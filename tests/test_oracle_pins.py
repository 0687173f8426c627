"""Pins of the FP64 oracle against facts that do not come from the oracle:
closed forms, brute force, identities of App. A, and the invariants and the
correctness theorem of Algorithm 3 (Sec. III).  No GPU."""
import math

import numpy as np
import pytest

from paper_2401_01404_gb300 import inputs


def _rand_spins(N, M, seed, bias=0.0):
    g = np.random.default_rng(seed)
    return np.where(g.random((N, M)) < 0.5 + bias, 1, -1).astype(np.int8)


def _rand_W(N, seed, p=0.3, scale=0.4, diag=0.0):
    g = np.random.default_rng(seed)
    A = np.triu((g.random((N, N)) < p) * g.normal(0, scale, (N, N)), 1)
    W = A + A.T
    np.fill_diagonal(W, diag)
    return W


def _pl_numpy(X, h, W, lam):
    """Pseudo-likelihood through the conditionals P(x_i|rest) = sigmoid(2 x_i f_i)
    (App. A) with f = h + W_offdiag X, written independently of the oracle."""
    Wo = W - np.diag(np.diag(W))
    f = h[:, None] + Wo @ X.astype(np.float64)
    z = 2.0 * X * f
    ll = -np.logaddexp(0.0, -z).sum()
    return ll - lam * np.abs(np.triu(Wo, 1)).sum()


# ---------------------------------------------------------------- objective


def test_objective_empty_state_is_minus_NM_ln2(oracle):
    X = _rand_spins(7, 33, 1)
    o = oracle.IsingOracle(X, lam=3.0)
    o.set_state(np.zeros((7, 7)), np.zeros(7))
    assert o.objective() == pytest.approx(-7 * 33 * math.log(2.0), rel=1e-15)


def test_objective_matches_conditional_form(oracle):
    N, M, lam = 9, 40, 1.7
    X = _rand_spins(N, M, 2)
    W = _rand_W(N, 3, diag=5.0)  # a nonzero diagonal must be ignored
    h = np.random.default_rng(4).normal(0, 0.3, N)
    o = oracle.IsingOracle(X, lam=lam)
    o.set_state(W, h)
    assert o.objective() == pytest.approx(_pl_numpy(X, h, W, lam), rel=1e-12)


def test_fields_at_zero_coupling_are_atanh_of_mean(oracle):
    X = _rand_spins(6, 50, 5, bias=0.2)
    X[0, :] = 1  # constant column: the optimum is beyond the clamp
    o = oracle.IsingOracle(X, lam=1.0, h_clamp=10.0)
    xbar = X.mean(1)
    expect = np.where(np.abs(xbar) < 1, np.arctanh(np.clip(xbar, -0.999999, 0.999999)), 10.0 * np.sign(xbar))
    assert np.allclose(o.h, expect, rtol=1e-10, atol=1e-10)


# ---------------------------------------------------------------- pair gain


def test_gain_at_zero_field_closed_form(oracle):
    """h = 0, W = 0: F(w) = 2wS - 2M log cosh w with S = sum x_i x_j, so
    tanh w* = r - sign(r) lambda/(2M), r = S/M, and the gain is
    2 S w* - 2 M log cosh w* - lambda |w*|."""
    M = 64
    X = _rand_spins(2, M, 6, bias=0.0)
    X[1, :40] = X[0, :40]  # correlated pair
    S = float((X[0].astype(int) * X[1]).sum())
    for lam in (0.0, 3.0, 20.0):
        o = oracle.IsingOracle(X, lam=lam)
        o.set_state(np.zeros((2, 2)), np.zeros(2))
        g, w = o.score([[0, 1]])
        r = S / M
        if abs(2 * S) <= lam:
            assert w[0] == 0.0 and g[0] == 0.0
            continue
        ws = math.atanh(r - math.copysign(lam / (2 * M), r))
        gain = 2 * S * ws - 2 * M * math.log(math.cosh(ws)) - lam * abs(ws)
        assert w[0] == pytest.approx(ws, rel=1e-11)
        assert g[0] == pytest.approx(gain, rel=1e-11)


def test_gain_zero_iff_gradient_below_lambda(oracle):
    """w* = 0 exactly when |sum_m [x_j(x_i - t_i) + x_i(x_j - t_j)]| <= lambda."""
    N, M = 12, 80
    X = _rand_spins(N, M, 7)
    W = _rand_W(N, 8, p=0.2)
    h = np.random.default_rng(9).normal(0, 0.2, N)
    lam = 12.0
    o = oracle.IsingOracle(X, lam=lam)
    Wz = W.copy()
    Wz[0, :] = Wz[:, 0] = 0.0  # pairs (0, j) sit at W = 0
    o.set_state(Wz, h)
    f = h[:, None] + (Wz - np.diag(np.diag(Wz))) @ X
    t = np.tanh(f)
    pairs = np.array([[0, j] for j in range(1, N)], dtype=np.int32)
    g, w = o.score(pairs)
    seen_zero = seen_nonzero = 0
    for (i, j), gi, wi in zip(pairs, g, w):
        d0 = np.sum(X[j] * (X[i] - t[i]) + X[i] * (X[j] - t[j]))
        if abs(d0) <= lam:
            assert wi == 0.0 and gi == 0.0
            seen_zero += 1
        else:
            assert np.sign(wi) == np.sign(d0) and gi > 0
            seen_nonzero += 1
    assert seen_zero and seen_nonzero


def test_gain_equals_objective_difference(oracle):
    """Applying the update raises pi by exactly the reported gain."""
    N, M, lam = 10, 60, 4.0
    X = _rand_spins(N, M, 10)
    W = _rand_W(N, 11, p=0.4)
    h = np.random.default_rng(12).normal(0, 0.2, N)
    o = oracle.IsingOracle(X, lam=lam)
    o.set_state(W, h)
    base = o.objective()
    pairs = np.array([[a, b] for a in range(N) for b in range(a + 1, N)], dtype=np.int32)
    g, w = o.score(pairs)
    for (i, j), gi, wi in list(zip(pairs, g, w))[::3]:
        W2 = W.copy()
        W2[i, j] = W2[j, i] = wi
        expect = _pl_numpy(X, h, W2, lam) - _pl_numpy(X, h, W, lam)
        assert gi == pytest.approx(expect, rel=1e-9, abs=1e-9 * abs(base))
        assert gi >= -1e-9


def test_gain_is_grid_maximum(oracle):
    """Brute force over a fine grid of w agrees with the bisection maximiser."""
    N, M, lam = 5, 24, 2.5
    X = _rand_spins(N, M, 13)
    W = _rand_W(N, 14, p=0.5)
    h = np.random.default_rng(15).normal(0, 0.3, N)
    o = oracle.IsingOracle(X, lam=lam)
    o.set_state(W, h)
    grid = np.linspace(-4, 4, 16001)
    for i, j in [(0, 1), (1, 3), (2, 4), (0, 4)]:
        g, w = o.score([[i, j]])
        base = _pl_numpy(X, h, W, lam)
        vals = []
        for wv in grid:
            W2 = W.copy()
            W2[i, j] = W2[j, i] = wv
            vals.append(_pl_numpy(X, h, W2, lam) - base)
        vals = np.array(vals)
        assert g[0] >= vals.max() - 1e-9
        assert g[0] - vals.max() < 1e-4 * max(1.0, abs(g[0]))
        assert abs(w[0] - grid[vals.argmax()]) <= 2 * (grid[1] - grid[0]) + 1e-9 or g[0] < 1e-6


def test_gain_is_symmetric(oracle):
    N, M = 8, 50
    X = _rand_spins(N, M, 16)
    o = oracle.IsingOracle(X, lam=2.0)
    o.set_state(_rand_W(N, 17), np.random.default_rng(18).normal(0, .2, N))
    p = np.array([[a, b] for a in range(N) for b in range(a + 1, N)], dtype=np.int32)
    g1, w1 = o.score(p)
    g2, w2 = o.score(p[:, ::-1].copy())
    assert np.allclose(g1, g2, rtol=1e-12, atol=1e-12) and np.allclose(w1, w2, rtol=1e-12, atol=1e-12)


def test_gcd_recovers_planted_edges(oracle):
    """With many samples, GCD's reconstruction puts its largest couplings on
    the planted edges (the statistical content of the objective)."""
    N, M = 24, 3000
    edges = inputs.erdos_renyi(N, 3, inputs.rng(77, inputs.GRAPH))
    w = 0.4 * np.where(inputs.rng(77, inputs.COUPLINGS).random(len(edges)) < 0.5, -1.0, 1.0)
    X = inputs.gibbs_ising(N, edges, w, np.zeros(N), M, 300, 77)
    o = oracle.IsingOracle(X, lam=inputs.default_lambda(N, M))
    oracle.gcd(o, kappa=2.0, eps=1e-3, max_iters=200)
    iu = np.triu_indices(N, 1)
    top = np.argsort(-np.abs(o.W[iu]))[:len(edges)]
    planted = {tuple(e) for e in edges.tolist()}
    prec = np.mean([(int(iu[0][q]), int(iu[1][q])) in planted for q in top])
    assert prec >= 0.95
    # the signs of the recovered couplings are the planted signs
    for (a, b), wv in zip(edges, w):
        if (a, b) in {(int(iu[0][q]), int(iu[1][q])) for q in top}:
            assert np.sign(o.W[a, b]) == np.sign(wv)


# ---------------------------------------------------------------- coordinate descent


def test_single_updates_never_decrease_objective(oracle):
    N, M = 10, 60
    X = _rand_spins(N, M, 19)
    o = oracle.IsingOracle(X, lam=3.0)
    prev = o.objective()
    rng = np.random.default_rng(20)
    for _ in range(60):
        a, b = sorted(rng.choice(N, 2, replace=False))
        o.update([[a, b]])
        cur = o.objective()
        assert cur >= prev - 1e-9 * abs(prev)
        prev = cur
    o.field_sweep()
    assert o.objective() >= prev - 1e-9 * abs(prev)


def _small_problem():
    wl = inputs.config("ising_n100_m200", N=14, M=300, sweeps=200)
    return wl.X, inputs.default_lambda(wl.N, wl.M, 0.5)


def test_gcd_and_cd_reach_the_same_optimum(oracle):
    """The objective is convex: CD and GCD (kappa > 0) converge to the same
    optimum (Sec. III)."""
    X, lam = _small_problem()
    a = oracle.IsingOracle(X, lam=lam)
    b = oracle.IsingOracle(X, lam=lam)
    ha = oracle.cd(a, eps=1e-10, max_iters=400)
    hb = oracle.gcd(b, kappa=1.0, eps=1e-10, max_iters=4000)
    assert ha[-1][1] < 1e-10 and hb[-1][1] < 1e-10
    assert a.objective() == pytest.approx(b.objective(), rel=1e-8)
    assert np.allclose(a.W, b.W, atol=1e-5)


def test_gcd_with_all_pairs_selects_what_cd_updates(oracle):
    """With kappa N >= N(N-1)/2, GCD's selection is every pair."""
    X, lam = _small_problem()
    o = oracle.IsingOracle(X, lam=lam)
    N = o.N
    m = oracle.round_half_up(N * (N - 1) / 2 / N * N)
    best = oracle.exhaustive_best(o.dist_matrix(), m)
    assert len(best) == N * (N - 1) // 2
    assert {tuple(p) for p in best.tolist()} == {tuple(p) for p in oracle.all_pairs(np.arange(N)).tolist()}


# ---------------------------------------------------------------- Gaussian


def _fd_slopes(o, set_state, W, pairs, eps=1e-5):
    """Central differences of the oracle's objective along each W_ij (= W_ji)."""
    out = []
    for i, j in pairs.tolist():
        vals = []
        for sgn in (1.0, -1.0):
            W2 = W.copy()
            W2[i, j] += sgn * eps
            W2[j, i] += sgn * eps
            set_state(W2)
            vals.append(o.objective())
        out.append((vals[0] - vals[1]) / (2 * eps))
    set_state(W)
    return np.array(out)


def test_ising_gradient_distance_is_the_objective_slope(oracle):
    """The gradient distance (App. B) equals the slope of log pi along W_ij, at
    zero and at nonzero couplings (where the prior adds -lam sign W_ij)."""
    N, M, lam = 9, 40, 3.0
    X = _rand_spins(N, M, 31)
    W = _rand_W(N, 32, p=0.4, scale=0.3)
    h = np.random.default_rng(33).normal(0, 0.2, N)
    o = oracle.IsingOracle(X, lam=lam)
    o.set_state(W, h)
    pairs = oracle.all_pairs(np.arange(N))
    wc = W[pairs[:, 0], pairs[:, 1]]
    assert (wc != 0).sum() >= 5 and (wc == 0).sum() >= 5
    g = oracle.ising_grad_rows(X, o.phi, pairs, lam, wcur=wc)
    fd = _fd_slopes(o, lambda W2: o.set_state(W2, h), W, pairs)
    assert np.allclose(g, np.abs(fd), rtol=1e-6, atol=1e-6)


def test_gauss_gradient_distance_is_the_objective_slope(oracle):
    N, M, lam = 8, 35, 0.9
    g0 = np.random.default_rng(41)
    X = g0.normal(0, 1, (N, M))
    W = _rand_W(N, 42, p=0.4, scale=0.2, diag=9.0)
    s2 = g0.uniform(0.4, 1.3, N)
    o = oracle.GaussOracle(X, lam=lam)
    o.set_state(W, s2)
    pairs = oracle.all_pairs(np.arange(N))
    wc = W[pairs[:, 0], pairs[:, 1]]
    assert (wc != 0).sum() >= 5 and (wc == 0).sum() >= 5
    g = oracle.gauss_grad_rows(X, o.mu, s2, pairs, lam, wcur=wc)
    fd = _fd_slopes(o, lambda W2: o.set_state(W2, s2), W, pairs)
    assert np.allclose(g, np.abs(fd), rtol=1e-6, atol=1e-6)


def test_gauss_objective_matches_normal_logpdf(oracle):
    from scipy.stats import norm

    N, M, lam = 7, 30, 0.8
    g = np.random.default_rng(21)
    X = g.normal(0, 1, (N, M))
    W = _rand_W(N, 22, diag=9.0)
    s2 = g.uniform(0.3, 1.5, N)
    o = oracle.GaussOracle(X, lam=lam)
    o.set_state(W, s2)
    Wo = W - np.diag(np.diag(W))
    mu = Wo @ X
    ll = norm.logpdf(X, loc=-s2[:, None] * mu, scale=np.sqrt(s2)[:, None]).sum()
    assert o.objective() == pytest.approx(ll - lam * np.abs(np.triu(Wo, 1)).sum(), rel=1e-12)


def test_gauss_gain_matches_soft_threshold_closed_form(oracle):
    """The Gaussian 1-D problem is quadratic: with a = -sum(e_i x_j + e_j x_i),
    b = s2_i sum x_j^2 + s2_j sum x_i^2 and z = W + a/b, the maximiser is the
    soft threshold sign(z) max(|z| - lambda/b, 0)."""
    N, M = 9, 40
    g = np.random.default_rng(23)
    X = g.normal(0, 1, (N, M))
    W = _rand_W(N, 24, p=0.4, scale=0.3)
    s2 = g.uniform(0.3, 1.5, N)
    for lam in (0.0, 5.0, 25.0):
        o = oracle.GaussOracle(X, lam=lam)
        o.set_state(W, s2)
        p = oracle.all_pairs(np.arange(N))
        gain, wst = o.score(p)
        mu = (W - np.diag(np.diag(W))) @ X
        e = X + s2[:, None] * mu
        for (i, j), gg, ww in zip(p, gain, wst):
            a = -np.sum(e[i] * X[j] + e[j] * X[i])
            b = s2[i] * np.sum(X[j] ** 2) + s2[j] * np.sum(X[i] ** 2)
            z = W[i, j] + a / b
            w_cf = np.sign(z) * max(abs(z) - lam / b, 0.0)
            dlt = w_cf - W[i, j]
            g_cf = a * dlt - b * dlt * dlt / 2 - lam * abs(w_cf) + lam * abs(W[i, j])
            assert ww == pytest.approx(w_cf, rel=1e-10, abs=1e-12)
            assert gg == pytest.approx(g_cf, rel=1e-9, abs=1e-9)


def test_gauss_diagonal_closed_form(oracle):
    """theta_i^2 = u* = (-M + sqrt(M^2 + 4AC))/(2C), A = sum x^2, C = sum mu^2;
    at W = 0 it is the sample second moment."""
    N, M = 6, 50
    g = np.random.default_rng(25)
    X = g.normal(0, 1.3, (N, M))
    o = oracle.GaussOracle(X, lam=1.0)
    assert np.allclose(o.s2, (X ** 2).mean(1), rtol=1e-12)
    W = _rand_W(N, 26, p=0.6, scale=0.5)
    o.set_state(W, np.ones(N))
    o.diag_sweep()
    mu = (W - np.diag(np.diag(W))) @ X
    A, Cc = (X ** 2).sum(1), (mu ** 2).sum(1)
    u = (-M + np.sqrt(M * M + 4 * A * Cc)) / (2 * Cc)
    assert np.allclose(o.s2, u, rtol=1e-11)


def _gauss_problem(N=13, M=80, seed=51):
    """Samples of a sparse Gaussian precision model (dense Cholesky sampler)."""
    W = _rand_W(N, seed, p=0.3, scale=0.3)
    np.fill_diagonal(W, np.abs(W).sum(1) + 1.0)
    X = inputs.gaussian_dense_samples(W, M, seed + 1)
    return X, 2.0 * math.sqrt(M)


def test_gauss_update_reports_the_objective_increase(oracle):
    """One coupling update (App. A's tracked sums mu_i += dW x_j, mu_j += dW x_i)
    raises the objective by exactly the gain the score reports, measured against
    an objective whose neighbour sums are rebuilt from W from scratch; the
    tracked sums equal W x afterwards."""
    X, lam = _gauss_problem()
    N = X.shape[0]
    o = oracle.GaussOracle(X, lam=0.25 * lam)
    rng = np.random.default_rng(52)
    moved = 0
    for _ in range(40):
        a, b = sorted(rng.choice(N, 2, replace=False))
        gain, wst = o.score([[a, b]])
        before = o.objective()
        o.update([[a, b]])
        assert o.W[a, b] == pytest.approx(wst[0], rel=1e-9, abs=1e-12) and o.W[b, a] == o.W[a, b]
        mu_tracked = o.mu.copy()
        o.set_state(o.W, o.s2)  # mu rebuilt from W
        assert np.allclose(mu_tracked, o.mu, rtol=1e-10, atol=1e-10)
        after = o.objective()
        assert after - before == pytest.approx(gain[0], rel=1e-8, abs=1e-9 * abs(before))
        assert after >= before - 1e-9 * abs(before)
        moved += abs(wst[0]) > 0
        if _ % 7 == 6:
            o.diag_sweep()
    assert moved >= 10
    Wo = o.W - np.diag(np.diag(o.W))
    assert np.allclose(o.mu, Wo @ X, rtol=1e-10, atol=1e-10)


def test_gauss_single_updates_never_decrease_objective(oracle):
    X, lam = _gauss_problem(seed=53)
    o = oracle.GaussOracle(X, lam=lam)
    prev = o.objective()
    rng = np.random.default_rng(54)
    for _ in range(60):
        a, b = sorted(rng.choice(o.N, 2, replace=False))
        o.update([[a, b]])
        cur = o.objective()
        assert cur >= prev - 1e-12 * abs(prev)
        prev = cur
    o.diag_sweep()
    assert o.objective() >= prev - 1e-12 * abs(prev)


def test_gauss_gcd_and_cd_reach_the_same_optimum(oracle):
    """The Gaussian pseudo-likelihood with the Laplace prior is convex in W for
    fixed diagonal and the joint sweep converges: CD (Algorithm 1) and GCD
    (Algorithm 2, kappa = 1) end at the same optimum."""
    X, lam = _gauss_problem(N=14, M=120, seed=55)
    a = oracle.GaussOracle(X, lam=lam)
    b = oracle.GaussOracle(X, lam=lam)
    ha = oracle.cd(a, eps=1e-11, max_iters=3000)
    hb = oracle.gcd(b, kappa=1.0, eps=1e-11, max_iters=20000)
    assert ha[-1][1] < 1e-11 and hb[-1][1] < 1e-11
    assert a.objective() == pytest.approx(b.objective(), rel=1e-8)
    assert np.allclose(a.W, b.W, atol=1e-5)
    assert np.allclose(a.s2, b.s2, rtol=1e-5)
    # at the optimum every single-coupling gain is zero
    g, _ = a.score(oracle.all_pairs(np.arange(a.N)))
    assert g.max() <= 1e-8 * abs(a.objective())


# ---------------------------------------------------------------- searches


def _rand_D(N, seed):
    g = np.random.default_rng(seed)
    A = g.random((N, N))
    D = np.triu(A, 1)
    return D + D.T


def _geo_D(N, seed, dim=3):
    """Distances of random points in a cube: the kind of structure the
    neighbour-of-neighbour search exploits."""
    x = np.random.default_rng(seed).random((N, dim))
    return np.sqrt(((x[:, None, :] - x[None, :, :]) ** 2).sum(-1))


@pytest.mark.parametrize("N,m", [(20, 10), (40, 25), (60, 30), (60, 90), (33, 200)])
def test_findbest_with_exact_knn_is_exact(oracle, N, m):
    """Lenhof-Smid: with an exact KNN, Algorithm 3 returns the m closest pairs;
    m <= |D| <= 2m at each level and |S_{t+1}| <= |S_t|/2 (Sec. III)."""
    D = _rand_D(N, N * 1000 + m)
    got, st = oracle.findbest(D, m, knn_exact=True)
    ref = oracle.exhaustive_best(D, m)
    assert {tuple(p) for p in got.tolist()} == {tuple(p) for p in ref.tolist()}
    for t, nD in enumerate(st["level_D"]):
        assert m <= nD <= 2 * m
    sizes = st["level_size"]
    for t in range(len(sizes) - 1):
        assert sizes[t + 1] <= sizes[t] // 2


def test_findbest_regular_best_graph_needs_one_level(oracle):
    """If the m best pairs form a 2*kappa-regular graph, S' is empty after the
    first KNN level (Sec. III, d-regular case)."""
    N, kappa = 50, 2
    m = kappa * N
    D = 10.0 + _rand_D(N, 99)
    g = np.random.default_rng(98)
    vals = g.random(m)
    q = 0
    for i in range(N):
        for s in (1, 2):  # circulant C_N(1,2): 4-regular, m = 2N edges
            j = (i + s) % N
            D[i, j] = D[j, i] = vals[q]
            q += 1
    got, st = oracle.findbest(D, m, knn_exact=True)
    assert st["levels"] == 1 and st["level_size"][1] == 0
    assert {tuple(p) for p in got.tolist()} == {tuple(p) for p in oracle.exhaustive_best(D, m).tolist()}


def test_nndescent_recall_and_iterations(oracle):
    """NNDescent (Algorithm 4) on a random instance: near-exact k-NN within a
    few multiples of log_{2k} N iterations."""
    N, k = 300, 8
    D = _geo_D(N, 5)
    G, iters, _ = oracle.nndescent(D, k, eps=1e-3, max_iters=60, seed=3)
    ex = oracle.exact_knn(D, k)
    rec = np.mean([len(set(G[i]) & set(ex[i])) / k for i in range(N)])
    assert rec > 0.9
    assert iters <= 3 * (2 * math.ceil(math.log(N) / math.log(2 * k)) + 2)
    # every list holds k distinct ids that differ from the node
    for i in range(N):
        assert len(set(G[i])) == k and i not in set(G[i])


def test_nndescent_with_full_lists_is_exact(oracle):
    N = 12
    D = _rand_D(N, 6)
    G, _, _ = oracle.nndescent(D, N - 1, seed=4)
    ex = oracle.exact_knn(D, N - 1)
    assert all(set(G[i]) == set(ex[i]) for i in range(N))


def test_findbest_with_nndescent_recall(oracle):
    N, m = 200, 200
    D = _geo_D(N, 7)
    got, st = oracle.findbest(D, m, knn_exact=False, k_min=6, seed=11)
    ref = oracle.exhaustive_best(D, m)
    gain_ref = -D[ref[:, 0], ref[:, 1]]
    assert oracle.recall(got, ref, gain_ref - gain_ref.min() + 1) > 0.9


def test_recall_counts_only_nonzero_exact_gains(oracle):
    ex = np.array([[0, 1], [0, 2], [1, 2], [2, 3]])
    gain = np.array([5.0, 3.0, 0.0, 0.0])
    assert oracle.recall([[0, 1], [0, 2]], ex, gain) == 1.0
    assert oracle.recall([[0, 1], [2, 3]], ex, gain) == 0.5
