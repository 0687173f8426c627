"""Row-exhaustive scoring (recon_row_best), the ground truth of the subsample
protocol: every pair incident to a set of rows with d below a cut, scored
against all N columns.  Checked against the FP64 oracle scoring the same rows,
for both models, with the cut inside the distribution (pairs within the
tolerance of the cut may fall either side)."""
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


def _row_pairs(N, rows):
    rows = np.unique(rows)
    out = set()
    for i in rows.tolist():
        for j in range(N):
            if j != i:
                out.add((min(i, j), max(i, j)))
    return np.array(sorted(out), dtype=np.int32)


def _check(ctx, pairs_all, g_ref, rows, rank):
    order = np.sort(-g_ref)
    cut = float(order[rank])  # d of the rank-th best pair incident to the rows
    p, d, n = ctx.row_best(rows, cut)
    assert n == len(p) and np.all(p[:, 0] < p[:, 1])
    # ascending (d, i, j), unique
    key = np.lexsort((p[:, 1], p[:, 0], d))
    assert np.array_equal(key, np.arange(len(p)))
    assert len({tuple(x) for x in p.tolist()}) == len(p)
    tol = REL * np.abs(g_ref) + FLOOR * np.abs(g_ref).max()
    ref = {tuple(x): g for x, g in zip(pairs_all.tolist(), g_ref)}
    for x, dv in zip(p.tolist(), d):
        g = ref[tuple(x)]
        assert abs(-float(dv) - g) <= REL * abs(g) + FLOOR * np.abs(g_ref).max()
    sure = {tuple(x) for x, g, t in zip(pairs_all.tolist(), g_ref, tol) if -g < cut - t}
    got = {tuple(x) for x in p.tolist()}
    assert sure <= got
    maybe = {tuple(x) for x, g, t in zip(pairs_all.tolist(), g_ref, tol) if -g < cut + t}
    assert got <= maybe
    return p, d


def test_row_best_ising(R, oracle):
    N, M = 700, 300
    edges = inputs.erdos_renyi(N, 3, inputs.rng(21, inputs.GRAPH))
    w = inputs.rng(21, inputs.COUPLINGS).normal(0, 0.5, len(edges))
    X = inputs.gibbs_ising(N, edges, w, np.zeros(N), M, 200, 21)
    lam = inputs.default_lambda(N, M, 0.3)
    ctx = R.Recon(np.ascontiguousarray(X.T), R.RECON_ISING, lam=lam)
    g = np.random.default_rng(4)
    rows = np.concatenate([g.choice(N, 40, replace=False), [5, 5, 6]])
    pairs_all = _row_pairs(N, rows)
    h = oracle.ising_fields_at_zero(X)
    phi = np.repeat(h[:, None], M, 1)
    g_ref, _ = oracle.ising_score_rows(X, phi, pairs_all, lam, w_clamp=5.0)
    _check(ctx, pairs_all, g_ref, rows, 150)
    # a cut below every score gives nothing; no rows give nothing
    assert ctx.row_best(rows, -1e30)[2] == 0
    assert ctx.row_best(np.zeros(0, np.int32), 0.0)[2] == 0
    # after a GCD step the rows agree with recon_score at the new state
    ctx.gcd_step(8, 1.0)
    p, d, n = ctx.row_best(rows, 0.0)
    ds, _ = ctx.score(p)  # the generic scorer (another summation order)
    assert np.all(np.abs(ds - d) <= REL * np.abs(ds) + FLOOR * np.abs(ds).max())
    with pytest.raises(R.ReconError) as e:
        ctx.row_best([N], 0.0)
    assert e.value.status == R.RECON_EINVAL


def test_row_best_gauss(R, oracle):
    L1, L2, M = 20, 25, 400
    X = inputs.gaussian_torus_samples(L1, L2, -0.2, 1.8, M, 77)
    N = L1 * L2
    lam = inputs.default_lambda(N, M)
    ctx = R.Recon(np.ascontiguousarray(X.T.astype(np.float32)), R.RECON_GAUSSIAN, lam=lam)
    rows = np.random.default_rng(9).choice(N, 30, replace=False)
    pairs_all = _row_pairs(N, rows)
    X64 = X.astype(np.float32).astype(np.float64)
    s2 = oracle.gauss_diag_at_zero(X64)
    g_ref, _ = oracle.gauss_score_rows(X64, np.zeros_like(X64), s2, pairs_all, lam)
    _check(ctx, pairs_all, g_ref, rows, 60)
