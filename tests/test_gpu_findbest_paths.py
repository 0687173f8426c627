"""FindBest's one-CTA paths for small levels -- the D+ selection as a radix
select of the 2m best directed edges (Algorithm 3 needs them as a set), and the
final list as a shared-memory sort by (d, i, j) -- against the general radix
sorts that they replace (RECON_FINDBEST_SORTS=1 switches them off).  Same
k-NN lists, so the same best pairs bit for bit, on the empty network and after
GCD steps, with one and with several FindBest levels."""
import os

import numpy as np
import pytest

from paper_2401_01404_gb300 import inputs

pytestmark = pytest.mark.gpu


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


def _ctx(R, Xs, lam, sorts):
    if sorts:
        os.environ["RECON_FINDBEST_SORTS"] = "1"
    try:
        return R.Recon(Xs, R.RECON_ISING, lam=lam)
    finally:
        os.environ.pop("RECON_FINDBEST_SORTS", None)


def _expected_one_level(ids, d, m):
    """Algorithm 3's first level from its k-NN lists, on the host: D+ = the 2m
    best directed edges (by d), D = their pairs, and the m best pairs of D in
    (d, i, j) order.  Also the d of the 2m-th edge: the device breaks ties
    between edges of equal d (by a hash of the pair), so a pair whose d equals
    that cut may or may not be in D."""
    x = np.repeat(np.arange(ids.shape[0]), ids.shape[1])
    y, dv = ids.ravel(), d.ravel().astype(np.float64)
    keep = y >= 0
    x, y, dv = x[keep], y[keep], dv[keep]
    o = np.argsort(dv, kind="stable")
    n2m = min(2 * m, len(o))
    cut = dv[o[n2m - 1]]
    best = {}
    for e in o[:n2m]:
        a, b = (x[e], y[e]) if x[e] < y[e] else (y[e], x[e])
        best.setdefault((int(a), int(b)), dv[e])
    items = sorted(best.items(), key=lambda t: (t[1], t[0][0], t[0][1]))[:m]
    return items, cut


# (N, M, k, kappa): 2000 x 16 = 32000 list entries and 8000 selected (the
# benchmark's shape); 700 nodes with kappa = 1; 300 nodes with kappa = 3
# (several levels, the last one exhaustive); 5000 nodes, where the lists (80000
# entries) and the result (10000 pairs) exceed the one-CTA paths' limits and
# both contexts sort
@pytest.mark.parametrize("N,M,k,kappa", [(2000, 400, 16, 2.0), (700, 300, 8, 1.0), (300, 200, 4, 3.0),
                                         (5000, 200, 16, 1.0)])
def test_small_paths_equal_general_sorts(R, N, M, k, kappa):
    X = _wl(N, M, 900 + N)
    Xs = np.ascontiguousarray(X.T)
    lam = inputs.default_lambda(N, M)
    m = int(np.floor(kappa * N + 0.5))
    for sorts in (False, True):
        c = _ctx(R, Xs, lam, sorts)
        for step in range(3):
            p, dd = c.best_pairs(k, kappa)
            assert len(p) > 0
            # (d, i, j) order, i < j, one entry per pair
            assert np.all(np.diff(dd) >= 0)
            assert np.all(p[:, 0] < p[:, 1])
            assert len({tuple(x) for x in p.tolist()}) == len(p)
            st = c.stats()
            if st["levels"] == 1 and st["level_size"][1] < 2:
                # one level: the result is the first level's D, recomputed from its lists
                ids, dl = c.knn_graph()
                items, cut = _expected_one_level(ids, dl, m)
                got = {tuple(x): v for x, v in zip(p.tolist(), dd.tolist())}
                want = {pq: v for pq, v in items}
                sure = {pq for pq, v in want.items() if v < cut}
                assert sure <= set(got), (sorts, step, len(sure - set(got)))
                for pq, v in got.items():
                    assert pq in want or v >= cut, (sorts, step, pq)
                assert len(p) == min(m, len(want)) or dd[-1] >= cut
            c.gcd_step(k, kappa)
        c.close()


def test_device_loop_matches_host_loop(R):
    """NNDescent's iterations as one conditional graph (the stopping test on the
    device; the default) against the host loop (one launch and one host test per
    iteration; what options.timing uses): the same kind of result, within the
    search's own run-to-run spread, and no more iterations than the cap."""
    N, M, k, kappa = 2000, 400, 16, 2.0
    X = _wl(N, M, 4242)
    Xs = np.ascontiguousarray(X.T)
    lam = inputs.default_lambda(N, M)
    m = int(np.floor(kappa * N + 0.5))
    ex = R.Recon(Xs, R.RECON_ISING, lam=lam)
    pe, de = ex.exhaustive_best(m)
    truth = {tuple(x) for x, v in zip(pe.tolist(), de) if v < 0}
    ex.close()
    rec, iters = {}, {}
    for timing in (0, 1):
        c = R.Recon(Xs, R.RECON_ISING, lam=lam, timing=timing)
        p, d = c.best_pairs(k, kappa)
        st = c.stats()
        assert st["nnd_graph_loops"] == (1 if timing == 0 else 0)
        iters[timing] = st["knn_iters"]
        rec[timing] = len(truth & {tuple(x) for x in p.tolist()}) / max(len(truth), 1)
        # a second search reuses the instantiated loop
        c.best_pairs(k, kappa)
        assert c.stats()["nnd_graph_loops"] == (2 if timing == 0 else 0)
        c.close()
    max_iters = 2 * int(np.ceil(np.log(N) / np.log(2 * k))) + 2
    assert 1 <= iters[0] <= max_iters and 1 <= iters[1] <= max_iters
    assert abs(iters[0] - iters[1]) <= 2
    assert rec[0] > 0.8 and abs(rec[0] - rec[1]) < 0.03, rec


@pytest.mark.parametrize("N,M", [(2000, 400), (1500, 1000), (800, 37)])
def test_pair_scores_do_not_depend_on_the_block(R, N, M):
    """The segmented scorer solves every pair in one orientation (the
    lower-numbered node first), so a pair found from both ends of the k-NN graph
    carries the same d in both lists, bit for bit, also after GCD steps (W != 0:
    Newton passes); otherwise two FindBest levels could report one pair twice
    with d values that differ in the last bit."""
    X = _wl(N, M, 321 + N)
    Xs = np.ascontiguousarray(X.T)
    c = R.Recon(Xs, R.RECON_ISING, lam=inputs.default_lambda(N, M))
    both_total = 0
    for step in range(3):
        c.best_pairs(16, 1.0)
        ids, d = c.knn_graph()
        seen = {}
        for x in range(ids.shape[0]):
            for y, dv in zip(ids[x].tolist(), d[x].tolist()):
                if y >= 0:
                    seen[(x, y)] = dv
        both = [(a, b) for (a, b) in seen if a < b and (b, a) in seen]
        both_total += len(both)
        bad = [(a, b, seen[(a, b)], seen[(b, a)]) for a, b in both if seen[(a, b)] != seen[(b, a)]]
        assert not bad, (step, len(bad), bad[:3])
        c.gcd_step(16, 1.0)
    assert both_total > 100
    c.close()
