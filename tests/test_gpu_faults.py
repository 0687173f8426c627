"""Failure handling, injected on the host (no GPU fault): a cap on the device
memory a context may request makes the calls that need more fail with
RECON_ENOMEM, and a tensor-core screen (or a segmented scorer) whose loads are
never issued lets its bounded waits run out (about a second), so the launch
ends with an error word and the call returns RECON_ETIMEOUT.  Afterwards the GPU is untouched: a
fresh context gives the exact result."""
import os
import time

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


@pytest.fixture(scope="module")
def data():
    N, M = 600, 300
    edges = inputs.erdos_renyi(N, 3, inputs.rng(31, inputs.GRAPH))
    w = inputs.rng(31, inputs.COUPLINGS).normal(0, 0.5, len(edges))
    X = inputs.gibbs_ising(N, edges, w, np.zeros(N), M, 100, 31)
    return np.ascontiguousarray(X.T), inputs.default_lambda(N, M)


def _with_env(name, value, fn):
    os.environ[name] = value
    try:
        return fn()
    finally:
        del os.environ[name]


def test_allocation_cap_gives_enomem(R, data):
    Xs, lam = data
    # too small for the context's own state
    with pytest.raises(R.ReconError) as e:
        _with_env("RECON_FAULT_ALLOC_LIMIT", str(64 * 1024), lambda: R.Recon(Xs, R.RECON_ISING, lam=lam))
    assert e.value.status == R.RECON_ENOMEM
    # enough for the state, not for the search buffers
    c = _with_env("RECON_FAULT_ALLOC_LIMIT", str(4 << 20), lambda: R.Recon(Xs, R.RECON_ISING, lam=lam))
    with pytest.raises(R.ReconError) as e:
        c.best_pairs(16, 1.0)
    assert e.value.status == R.RECON_ENOMEM
    c.close()


@pytest.mark.parametrize("pair", [0, 1])
def test_stalled_screen_times_out_and_the_gpu_stays_usable(R, data, pair):
    """Both screen forms: in the CTA-pair form each CTA's waits give up on their
    own, and the pair meets at its closing cluster barrier before freeing TMEM."""
    Xs, lam = data
    ref = R.Recon(Xs, R.RECON_ISING, lam=lam, knn_mode=R.RECON_KNN_SCREEN)
    p0, d0 = ref.best_pairs(16, 1.0)
    c = _with_env("RECON_FAULT_SCREEN_STALL", "1",
                  lambda: R.Recon(Xs, R.RECON_ISING, lam=lam, knn_mode=R.RECON_KNN_SCREEN, screen_pair=pair))
    t0 = time.perf_counter()
    with pytest.raises(R.ReconError) as e:
        c.best_pairs(16, 1.0)
    assert e.value.status == R.RECON_ETIMEOUT
    assert time.perf_counter() - t0 < 30.0
    # the context refuses further work; a fresh one gives the same exact result
    with pytest.raises(R.ReconError) as e:
        c.best_pairs(16, 1.0)
    assert e.value.status == R.RECON_ESTATE
    c.close()
    fresh = R.Recon(Xs, R.RECON_ISING, lam=lam, knn_mode=R.RECON_KNN_SCREEN)
    p1, d1 = fresh.best_pairs(16, 1.0)
    assert np.array_equal(p0, p1) and np.array_equal(d0, d1)


def test_stalled_scorer_times_out_and_the_gpu_stays_usable(R, data):
    """The segmented scorer's row copies are never issued: each stage wait runs
    out (about a second), the launch sets its error word and the search
    returns RECON_ETIMEOUT; a fresh context gives the same result as before."""
    Xs, lam = data
    ex = R.RECON_KNN_EXHAUSTIVE  # every pair through the segmented scorer
    ref = R.Recon(Xs, R.RECON_ISING, lam=lam, knn_mode=ex)
    p0, d0 = ref.best_pairs(16, 1.0)
    c = _with_env("RECON_FAULT_SCORE_STALL", "1", lambda: R.Recon(Xs, R.RECON_ISING, lam=lam, knn_mode=ex))
    t0 = time.perf_counter()
    with pytest.raises(R.ReconError) as e:
        c.best_pairs(16, 1.0)
    assert e.value.status == R.RECON_ETIMEOUT
    assert time.perf_counter() - t0 < 60.0
    with pytest.raises(R.ReconError) as e:
        c.best_pairs(16, 1.0)
    assert e.value.status == R.RECON_ESTATE
    c.close()
    fresh = R.Recon(Xs, R.RECON_ISING, lam=lam, knn_mode=ex)
    p1, d1 = fresh.best_pairs(16, 1.0)
    assert np.array_equal(p0, p1) and np.array_equal(d0, d1)


def test_stalled_scorer_gives_up_once_for_the_whole_launch(R):
    """With many more segments than fit on the GPU at once, a stall still ends
    the launch in about one wait bound: the first warp that gives up raises the
    launch's error word, the waiting warps see it and later blocks skip their
    work (rather than each wave of blocks waiting its own second)."""
    N, M = 3000, 200
    edges = inputs.erdos_renyi(N, 3, inputs.rng(33, inputs.GRAPH))
    w = inputs.rng(33, inputs.COUPLINGS).normal(0, 0.5, len(edges))
    Xs = np.ascontiguousarray(inputs.gibbs_ising(N, edges, w, np.zeros(N), M, 50, 33).T)
    lam = inputs.default_lambda(N, M)
    ex = R.RECON_KNN_EXHAUSTIVE  # about 9000 segments of up to 512 pairs
    c = _with_env("RECON_FAULT_SCORE_STALL", "1", lambda: R.Recon(Xs, R.RECON_ISING, lam=lam, knn_mode=ex))
    t0 = time.perf_counter()
    with pytest.raises(R.ReconError) as e:
        c.best_pairs(16, 1.0)
    dt = time.perf_counter() - t0
    assert e.value.status == R.RECON_ETIMEOUT
    assert dt < 6.0, dt
    c.close()
    fresh = R.Recon(Xs, R.RECON_ISING, lam=lam, knn_mode=R.RECON_KNN_SCREEN)
    fresh.best_pairs(16, 1.0)
