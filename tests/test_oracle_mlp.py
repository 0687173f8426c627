"""The oracle's proposal MLP: its backpropagated gradient equals central
finite differences of its loss (FP64), and its sketch is the random projection
it claims to be.  No GPU."""
import numpy as np

from oracle import mlp


def test_gradient_matches_finite_differences():
    g = np.random.default_rng(0)
    N = 12
    s = g.normal(0, 1, (N, mlp.S))
    w = g.normal(0, 0.2, mlp.H * mlp.S + mlp.H + mlp.E * mlp.H + mlp.E)
    pairs = np.array([[0, 1], [2, 5], [3, 4], [1, 7], [6, 11], [8, 9], [0, 10]])
    tau = g.normal(0, 1, len(pairs))
    L, gr = mlp.grad(w, s, pairs, tau)
    assert abs(L - mlp.loss(w, s, pairs, tau)) < 1e-12
    idx = g.choice(len(w), 60, replace=False)
    for q in idx:
        h = 1e-6
        wp, wm = w.copy(), w.copy()
        wp[q] += h
        wm[q] -= h
        fd = (mlp.loss(wp, s, pairs, tau) - mlp.loss(wm, s, pairs, tau)) / (2 * h)
        assert abs(fd - gr[q]) <= 1e-6 * max(1.0, abs(gr[q])), (q, fd, gr[q])


def test_sketch_is_a_random_sign_projection():
    M = 300
    Om = mlp.omega(M, 7)
    assert set(np.unique(Om)) == {-1.0, 1.0}
    assert abs(Om.mean()) < 0.05  # balanced signs
    g = np.random.default_rng(1)
    X = np.where(g.random((5, M)) < 0.5, 1, -1).astype(np.int8)
    s = mlp.sketch(X, 7)
    # every entry is (M - 2 * #disagreements) / sqrt(M)
    z = s * np.sqrt(M)
    assert np.allclose(z, np.round(z)) and np.all((np.round(z).astype(int) - M) % 2 == 0)
    # a node's sketch norm estimates 64 |x|^2 / M = 64 (Johnson-Lindenstrauss)
    assert abs((s * s).sum(1).mean() / 64 - 1) < 0.2
