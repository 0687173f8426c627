"""FP64 oracle of the learned proposal (test infrastructure only).

Plain NumPy, written from the definitions the library documents:
  sketch  s_i = Omega^T x_i / sqrt(M), Omega[m, c] = -1 where the top bit of
          SplitMix64(omega_seed + 2^32 c + m) is set, else +1, with
          omega_seed = SplitMix64(seed xor 0x0de9a5eed) (SplitMix64: Steele, Lea
          and Flood, OOPSLA 2014, implemented here on its own);
  MLP     a = W1 s + b1, h = relu(a), e = W2 h + b2;
  loss    mean over pairs of (<e_i, e_j> - tau_ij)^2,
and the gradient by explicit backpropagation.  Parameter layout:
W1 [128 x 64] | b1 [128] | W2 [32 x 128] | b2 [32].  Pinned by central finite
differences in tests/test_oracle_mlp.py.
"""
from __future__ import annotations

import numpy as np

S, H, E = 64, 128, 32
M64 = (1 << 64) - 1


def splitmix64(x: int) -> int:
    x = (x + 0x9E3779B97F4A7C15) & M64
    x = ((x ^ (x >> 30)) * 0xBF58476D1CE4E5B9) & M64
    x = ((x ^ (x >> 27)) * 0x94D049BB133111EB) & M64
    return x ^ (x >> 31)


def omega(M: int, seed: int) -> np.ndarray:
    """M x 64 matrix of +-1."""
    oseed = splitmix64(seed ^ 0x0DE9A5EED)
    out = np.empty((M, S))
    for c in range(S):
        for m in range(M):
            out[m, c] = -1.0 if splitmix64((oseed + (c << 32) + m) & M64) >> 63 else 1.0
    return out


def sketch(X: np.ndarray, seed: int) -> np.ndarray:
    """X node-major +-1 (N x M)."""
    X = np.asarray(X, dtype=np.float64)
    return X @ omega(X.shape[1], seed) / np.sqrt(X.shape[1])


def unpack(w: np.ndarray):
    w = np.asarray(w, dtype=np.float64)
    q = 0
    W1 = w[q:q + H * S].reshape(H, S); q += H * S
    b1 = w[q:q + H]; q += H
    W2 = w[q:q + E * H].reshape(E, H); q += E * H
    b2 = w[q:q + E]
    return W1, b1, W2, b2


def forward(w, s):
    W1, b1, W2, b2 = unpack(w)
    a = s @ W1.T + b1
    h = np.maximum(a, 0.0)
    return a, h, h @ W2.T + b2


def loss(w, s, pairs, tau) -> float:
    _, _, e = forward(w, s)
    p = np.asarray(pairs)
    r = (e[p[:, 0]] * e[p[:, 1]]).sum(1) - np.asarray(tau, dtype=np.float64)
    return float(np.mean(r * r))


def grad(w, s, pairs, tau):
    """(loss, gradient) by backpropagation."""
    W1, b1, W2, b2 = unpack(w)
    a, h, e = forward(w, s)
    p = np.asarray(pairs)
    r = (e[p[:, 0]] * e[p[:, 1]]).sum(1) - np.asarray(tau, dtype=np.float64)
    n = len(p)
    dp = 2.0 * r / n
    de = np.zeros_like(e)
    np.add.at(de, p[:, 0], dp[:, None] * e[p[:, 1]])
    np.add.at(de, p[:, 1], dp[:, None] * e[p[:, 0]])
    gW2 = de.T @ h
    gb2 = de.sum(0)
    dh = de @ W2
    da = dh * (a > 0)
    gW1 = da.T @ s
    gb1 = da.sum(0)
    return float(np.mean(r * r)), np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2])
