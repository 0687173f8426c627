"""The learned proposal on the GPU: its sketch and its loss gradient match the
FP64 oracle (which is pinned by finite differences); trained on one planted
graph it carries to another, and what it gains there over random lists is
measured on equal search seeds."""
import math

import numpy as np
import pytest

from oracle import mlp
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


def _bf16(a):
    import torch

    return torch.from_numpy(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).float().numpy()


def test_sketch_and_gradient_match_the_oracle(R):
    N, M = 150, 333
    edges = inputs.erdos_renyi(N, 3, inputs.rng(9, inputs.GRAPH))
    X = inputs.gibbs_ising(N, edges, np.full(len(edges), 0.3), np.zeros(N), M, 50, 9)
    ctx = R.Recon(np.ascontiguousarray(X.T), R.RECON_ISING, lam=10.0)
    sk, _ = R.recon_proposal_embed(ctx.ctx, N)
    s_ref = mlp.sketch(X, 7)
    assert np.allclose(sk, s_ref, rtol=1e-6, atol=1e-6)
    g = np.random.default_rng(3)
    n = R.recon_proposal_param_count()
    w = _bf16(g.normal(0, 0.15, n))  # exactly representable in the bf16 forward pass
    R.recon_proposal_weights(ctx.ctx, w)
    pairs = inputs.random_pairs(N, 700, 4)
    tau = g.normal(0, 1, len(pairs)).astype(np.float32)
    grad, loss = R.recon_proposal_grad(ctx.ctx, pairs, tau)
    L_ref, g_ref = mlp.grad(w.astype(np.float64), s_ref, pairs, tau.astype(np.float64))
    assert loss == pytest.approx(L_ref, rel=1e-4)
    scale = np.abs(g_ref).max()
    assert np.allclose(grad, g_ref, rtol=2e-3, atol=2e-4 * scale)


def test_trained_proposal_carries_to_another_graph(R):
    """Trained on exact scores of one planted graph (Omega redrawn at every
    step), the proposal seeds the first lists of another graph of the same kind
    (N = 2000, M = 1000, 4-regular, couplings +-0.3): its seeds hold far more of
    the exact best pairs than random lists, NNDescent from them finds more of
    the best pairs after its first iteration than from random lists on equal
    search seeds, and every seeding converges.  (The gain is the first
    iteration's: random lists catch up by the second or third, see the design
    notes.)  A proposal trained on a fixed Omega learns the nodes of its
    training graph and carries much less."""
    N, M, kappa, k = 2000, 1000, 2.0, 16
    lam = inputs.default_lambda(N, M)
    train = inputs.ising_workload("train", N, M, "regular", 4, "pm", 0.3, 0.0, 300, 4242, k, kappa, device="cuda")
    test = inputs.ising_workload("test", N, M, "regular", 4, "pm", 0.3, 0.0, 300, 2000, k, kappa, device="cuda")
    Xs = test.samples_major()
    exact = R.Recon(Xs, R.RECON_ISING, lam=lam, knn_mode=R.RECON_KNN_SCREEN)
    top, dtop = exact.best_pairs(k, kappa)
    truth = {tuple(p) for p, d in zip(top.tolist(), dtop) if d < 0}

    def trained(fixed):
        c = R.Recon(train.samples_major(), R.RECON_ISING, lam=lam)
        loss = R.recon_proposal_train(c.ctx, steps=1500, lr=3e-3, seed=7, fixed_sketch=fixed)
        w = R.recon_proposal_weights(c.ctx)
        c.close()
        return loss, w

    def seed_share(w):
        # share of the exact best pairs among each node's 8 largest |<e_i, e_j>|
        R.recon_proposal_weights(exact.ctx, w)
        _, emb = R.recon_proposal_embed(exact.ctx, N)
        S = np.abs(emb.astype(np.float64) @ emb.T.astype(np.float64))
        np.fill_diagonal(S, -1)
        top8 = np.argsort(-S, axis=1)[:, :8]
        seeds = {(min(i, j), max(i, j)) for i in range(N) for j in top8[i]}
        return len(truth & seeds) / len(truth)

    loss, w = trained(0)
    assert loss[-1] < 0.2 * loss[0]
    share = seed_share(w)
    _, w_fixed = trained(1)
    share_fixed = seed_share(w_fixed)
    print("seed share: per-step Omega", share, "fixed Omega", share_fixed, "random lists", 8 * N / (N * (N - 1) / 2))
    assert share > 0.08 and share > 1.8 * share_fixed

    def recall_after(seed_mode, iters, seed):
        c = R.Recon(Xs, R.RECON_ISING, lam=lam, seed_mode=seed_mode, max_knn_iters=iters, eps_knn=0.0, seed=seed)
        if seed_mode == R.RECON_SEED_LEARNED:
            R.recon_proposal_weights(c.ctx, w)
        p, _ = c.best_pairs(k, kappa)
        st = c.stats()
        c.close()
        return len(truth & {tuple(x) for x in p.tolist()}) / len(truth), st

    seeds = (11, 12, 13)
    curves = {}
    for name, mode in (("random", R.RECON_SEED_RANDOM), ("learned", R.RECON_SEED_LEARNED)):
        curves[name] = {it: [recall_after(mode, it, s)[0] for s in seeds] for it in (1, 2, 8)}
        print(name, {it: np.round(v, 4).tolist() for it, v in curves[name].items()})
    _, st = recall_after(R.RECON_SEED_LEARNED, 1, 11)
    assert st["seeded_nodes"] > N // 2
    assert np.mean(curves["learned"][1]) > np.mean(curves["random"][1]) + 0.015, curves
    for name in curves:
        assert np.mean(curves[name][8]) > 0.94, (name, curves[name][8])
