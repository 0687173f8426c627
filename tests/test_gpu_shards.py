"""A split best-pairs search on one GPU: the shards of the exact screen
(recon_options.shard_index / shard_count), run one after another, merged by
recon_select_best, give exactly the unsharded answer -- at the empty network
(rank-one form) and with couplings stored (general form).  The shards are
independent launches with nothing waiting on another, as they would be on
separate GPUs.  And recon_select_best against a plain sort on the host."""
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
    edges = inputs.erdos_renyi(N, 4, inputs.rng(seed, inputs.GRAPH))
    w = inputs.rng(seed, inputs.COUPLINGS).normal(0, 0.4, len(edges))
    return np.ascontiguousarray(inputs.gibbs_ising(N, edges, w, np.zeros(N), M, 100, seed).T)


def _split(R, Xs, lam, k, kappa, S, model=None, form=None):
    from paper_2401_01404_gb300 import shards

    N = Xs.shape[1]
    lists, flop = [], 0.0
    for s in range(S):
        c = R.Recon(Xs, R.RECON_ISING, lam=lam, knn_mode=R.RECON_KNN_SCREEN, timing=1, **(form or {}),
                    **shards.shard_options(s, S))
        if model is not None:
            c.set_model(*model)
        lists.append(c.best_pairs(k, kappa))
        flop += c.stats()["screen_flop"]
        c.close()
    P = np.concatenate([p for p, _ in lists])
    D = np.concatenate([d for _, d in lists])
    sel = R.Recon(Xs, R.RECON_ISING, lam=lam)
    out = R.recon_select_best(sel.ctx, P, D, shards.best_m(N, kappa))
    sel.close()
    return out, flop


@pytest.mark.parametrize("S", [2, 3])
@pytest.mark.parametrize("N,M,kappa", [(3000, 200, 1.0), (1100, 333, 2.0)])
def test_shards_merge_to_the_whole_at_the_empty_network(R, N, M, kappa, S):
    Xs = _wl(N, M, 40 + N)
    lam = inputs.default_lambda(N, M)
    whole = R.Recon(Xs, R.RECON_ISING, lam=lam, knn_mode=R.RECON_KNN_SCREEN, timing=1)
    p0, d0 = whole.best_pairs(16, kappa)
    st = whole.stats()
    assert st["screen_rank1"] == 1
    (p1, d1), flop = _split(R, Xs, lam, 16, kappa, S)
    assert np.array_equal(p0, p1) and np.array_equal(d0, d1)
    # the shards together do the whole screen's work once
    assert flop == pytest.approx(st["screen_flop"], rel=1e-12)


@pytest.mark.parametrize("form", [dict(screen_fp8=0), dict(screen_fp8=1)])
def test_shards_merge_to_the_whole_with_couplings(R, form):
    N, M = 1500, 250
    Xs = _wl(N, M, 77)
    lam = inputs.default_lambda(N, M)
    base = R.Recon(Xs, R.RECON_ISING, lam=lam, knn_mode=R.RECON_KNN_SCREEN, **form)
    base.gcd_step(8, 1.0)
    model = base.get_model()
    assert len(model[0]) > 0
    # the whole search at the same state, set the same way as the shards' (fields rebuilt from W)
    ref = R.Recon(Xs, R.RECON_ISING, lam=lam, knn_mode=R.RECON_KNN_SCREEN, timing=1, **form)
    ref.set_model(*model)
    p0, d0 = ref.best_pairs(8, 1.0)
    assert ref.stats()["screen_rank1"] == 0
    (p1, d1), _ = _split(R, Xs, lam, 8, 1.0, 2, model=model, form=form)
    assert np.array_equal(p0, p1) and np.array_equal(d0, d1)


def test_select_best_orders_and_deduplicates(R):
    N = 500
    Xs = _wl(N, 60, 5)
    c = R.Recon(Xs, R.RECON_ISING, lam=1.0)
    g = np.random.default_rng(3)
    pairs = inputs.random_pairs(N, 4000, 11)
    pairs = pairs[np.unique(pairs[:, 0].astype(np.int64) * N + pairs[:, 1], return_index=True)[1]]
    # many ties in d (no -0.0, which orders before +0.0)
    d = (-np.round(g.exponential(1.0, len(pairs)), 2)).astype(np.float32) + np.float32(0.0)
    d[g.random(len(d)) < 0.3] = 0.0
    # every pair twice (one copy reversed), as two shards could report it
    P = np.concatenate([pairs, pairs[:, ::-1]])
    D = np.concatenate([d, d])
    perm = g.permutation(len(P))
    o = np.lexsort((pairs[:, 1], pairs[:, 0], d))
    for m in (1, 100, len(pairs) - 1, 10000):
        p, dd = R.recon_select_best(c.ctx, P[perm], D[perm], m)
        assert np.array_equal(p, pairs[o][:m]) and np.array_equal(dd, d[o][:m])
    with pytest.raises(R.ReconError) as e:
        R.recon_select_best(c.ctx, [[0, N]], [0.0], 1)
    assert e.value.status == R.RECON_EINVAL


def test_sharding_is_refused_where_it_is_not_built(R):
    Xs = _wl(300, 50, 9)
    with pytest.raises(R.ReconError) as e:
        R.Recon(Xs, R.RECON_ISING, lam=1.0, shard_index=0, shard_count=2)  # NNDescent
    assert e.value.status == R.RECON_EUNSUPPORTED
    with pytest.raises(R.ReconError) as e:
        R.Recon(Xs, R.RECON_ISING, lam=1.0, knn_mode=R.RECON_KNN_SCREEN, shard_index=2, shard_count=2)
    assert e.value.status == R.RECON_EINVAL
    c = R.Recon(Xs, R.RECON_ISING, lam=1.0, knn_mode=R.RECON_KNN_SCREEN, shard_index=1, shard_count=2)
    with pytest.raises(R.ReconError) as e:
        c.gcd_step(4, 1.0)
    assert e.value.status == R.RECON_EUNSUPPORTED
