"""Parity at the full size of the precision workload: N=100,000 nodes, M=500
Gibbs-sampled spins on an Erdos-Renyi graph of mean degree 5 (couplings
N(0, 0.3^2)).  The oracle cannot score all 5e9 pairs, so:
  * 10^5 sampled pairs (half uniform, half the best found) are scored by the
    CUDA path and by the oracle one pair at a time;
  * on 64 random rows the CUDA scorer scores every pair of the row, and every
    pair better than the m-th best must be in the screen's best list (the
    subsample protocol of the recall measurement).
"""
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
def c3():
    return inputs.config("ising_n1e5_m500", device="cuda")


def test_precision_workload_sampled_pairs_and_rows(R, oracle, c3):
    wl = c3
    lam = wl.lam
    scr = R.Recon(wl.samples_major(), R.RECON_ISING, lam=lam, knn_mode=R.RECON_KNN_SCREEN)
    p, d = scr.best_pairs(16, 1.0)
    assert len(p) == wl.N and np.all(np.diff(d) >= 0)
    # planted couplings dominate the top of the list
    planted = {tuple(e) for e in wl.edges.tolist()}
    assert np.mean([tuple(x) in planted for x in p[:1000].tolist()]) > 0.95
    # 1. sampled pairs against the oracle
    pairs = np.concatenate([inputs.random_pairs(wl.N, 50000, 11), p[:50000]])
    dg, _ = scr.score(pairs)
    h = oracle.ising_fields_at_zero(wl.X)
    phi = np.repeat(h[:, None], wl.M, 1)
    g_ref, _ = oracle.ising_score_rows(wl.X, phi, pairs, lam)
    tol = REL * np.abs(g_ref) + FLOOR * g_ref.max()
    bad = np.abs(-dg.astype(np.float64) - g_ref) > tol
    assert not bad.any(), (int(bad.sum()), dg[bad][:5], g_ref[bad][:5])
    # 2. whole rows: nothing better than the m-th best is missing from the list
    cut = float(d[-1])
    found = {tuple(x) for x in p.tolist()}
    g = np.random.default_rng(5)
    for i in g.choice(wl.N, 64, replace=False):
        j = np.delete(np.arange(wl.N), i)
        rowp = np.stack([np.minimum(i, j), np.maximum(i, j)], 1).astype(np.int32)
        dr, _ = scr.score(rowp)
        must = rowp[dr < cut - 1e-4 * abs(cut)]
        assert all(tuple(x) in found for x in must.tolist())
