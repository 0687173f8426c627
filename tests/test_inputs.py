"""The seeded input generators against what fixes them independently: exact
enumeration of a small Ising model, the inverse precision matrix of the
Gaussian samplers, and the structure of the random graphs.  No GPU."""
import itertools

import numpy as np
import pytest

from paper_2401_01404_gb300 import inputs


def test_gibbs_matches_exact_enumeration():
    """P(x) ∝ exp(sum_i h_i x_i + sum_{i<j} w_ij x_i x_j) (the model whose
    conditionals App. A uses); the sampler's state frequencies on 5 spins."""
    N, M = 5, 60000
    edges = np.array([[0, 1], [1, 2], [2, 3], [3, 4], [0, 4], [1, 3]])
    w = np.array([0.5, -0.4, 0.3, 0.6, -0.2, 0.25])
    h = np.array([0.1, -0.2, 0.0, 0.3, -0.1])
    X = inputs.gibbs_ising(N, edges, w, h, M, 60, 5)
    states = np.array(list(itertools.product([-1, 1], repeat=N)))
    logp = states @ h + sum(wk * states[:, a] * states[:, b] for (a, b), wk in zip(edges, w))
    p = np.exp(logp - logp.max())
    p /= p.sum()
    idx = ((X.T + 1) // 2) @ (1 << np.arange(N - 1, -1, -1))
    freq = np.bincount(idx, minlength=2 ** N) / M
    chi2 = M * ((freq - p) ** 2 / p).sum()
    assert chi2 < 2 ** N + 6 * np.sqrt(2 * 2 ** N), chi2  # mean 31, sd ~8 under the model


def _cov_close(X, C, rel):
    S = X @ X.T / X.shape[1]
    return np.abs(S - C).max() <= rel * np.abs(C).max()


def test_torus_sampler_covariance():
    L1, L2, off, diag = 4, 5, -0.2, 1.8
    X = inputs.gaussian_torus_samples(L1, L2, off, diag, 100000, 3)
    N = L1 * L2
    Q = np.eye(N) * diag
    for a, b in inputs.torus(L1, L2).tolist():
        Q[a, b] = Q[b, a] = off
    assert _cov_close(X, np.linalg.inv(Q), 0.03)


def test_dense_sampler_covariance():
    g = np.random.default_rng(4)
    A = g.normal(0, 1, (8, 8))
    Q = A @ A.T + 8 * np.eye(8)
    X = inputs.gaussian_dense_samples(Q, 100000, 5)
    assert _cov_close(X, np.linalg.inv(Q), 0.03)


def test_er_precision_sampler_covariance():
    """The paper's synthetic Gaussian (off-diagonals ~ N(-10^3, 10^2) on an ER
    graph, W_ii = sum |W_ij| / (1 - 10^-3)^2): exact samples of N(0, W^-1)."""
    N = 16
    e, w, d = inputs.gaussian_er_precision(N, 5, -1000.0, 10.0, 1e-3, 9)
    W = np.diag(d)
    W[e[:, 0], e[:, 1]] = w
    W[e[:, 1], e[:, 0]] = w
    rowsum = np.abs(W - np.diag(d)).sum(1)
    assert np.allclose(d[rowsum > 0], rowsum[rowsum > 0] / (1 - 1e-3) ** 2)
    assert np.linalg.eigvalsh(W).min() > 0
    X = inputs.gaussian_precision_samples(N, e, w, d, 100000, 10)
    assert _cov_close(X, np.linalg.inv(W), 0.03)


def test_random_graphs_are_simple():
    g = inputs.rng(1, inputs.GRAPH)
    for N, deg in ((300, 3.0), (5000, 5.0)):
        e = inputs.erdos_renyi(N, deg, g)
        assert np.all(e[:, 0] < e[:, 1])
        assert len({tuple(x) for x in e.tolist()}) == len(e)
        assert abs(2 * len(e) / N - deg) < 4 * np.sqrt(deg / N) + 0.2
    e = inputs.random_regular(1000, 4, g)
    assert np.all(np.bincount(e.ravel(), minlength=1000) == 4)
    assert len({tuple(x) for x in e.tolist()}) == len(e) and np.all(e[:, 0] < e[:, 1])
