"""recon_score_noalloc, the scoring call for callers that may not allocate
device memory while they run (for example next to a framework whose caching
allocator holds most of the GPU, or in a serving loop that forbids allocation):
it must return what recon_score returns, call after call, while staging its
data in the library's fixed static device array.  Collected last on purpose."""
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


def _close(a, b):
    a = -np.asarray(a, dtype=np.float64)
    b = -np.asarray(b, dtype=np.float64)
    tol = REL * np.abs(b) + FLOOR * max(float(np.max(b)), 1e-30)
    return np.all(np.abs(a - b) <= tol)


def test_noalloc_matches_recon_score_twice_in_a_row(R):
    wl = inputs.config("ising_n100_m200", N=300, M=500, sweeps=100)
    ctx = R.Recon(wl.samples_major(), R.RECON_ISING, lam=inputs.default_lambda(wl.N, wl.M))
    for call, seed in enumerate((3, 4)):
        pairs = inputs.random_pairs(wl.N, 5000 + 1000 * call, seed)
        d_ref, w_ref = ctx.score(pairs)
        st0 = ctx.stats()
        d, w = R.recon_score_noalloc(ctx.ctx, pairs)
        st1 = ctx.stats()
        assert _close(d, d_ref)
        assert np.allclose(w, w_ref, rtol=1e-5, atol=1e-6)
        # what the entry point is for: the call requested no device memory, and its
        # work is counted like recon_score's (pairs and Newton passes)
        assert st1["device_bytes"] == st0["device_bytes"] > 0
        assert st1["pair_evals"] - st0["pair_evals"] == len(pairs)
        assert st1["newton_passes"] >= st0["newton_passes"]


def test_noalloc_needs_no_allocation_room(R, monkeypatch):
    """A context whose allocation cap is what its own set-up took cannot grow
    recon_score's staging buffers for a larger list; recon_score_noalloc still
    scores that list."""
    wl = inputs.config("ising_n100_m200", N=200, M=300, sweeps=50)
    Xs = wl.samples_major()
    lam = inputs.default_lambda(wl.N, wl.M)
    probe = R.Recon(Xs, R.RECON_ISING, lam=lam)
    base = probe.stats()["device_bytes"]
    probe.close()
    monkeypatch.setenv("RECON_FAULT_ALLOC_LIMIT", str(base))
    ctx = R.Recon(Xs, R.RECON_ISING, lam=lam)
    monkeypatch.delenv("RECON_FAULT_ALLOC_LIMIT")
    pairs = inputs.random_pairs(wl.N, 20000, 6)
    with pytest.raises(R.ReconError) as e:
        ctx.score(pairs)
    assert e.value.status == R.RECON_ENOMEM
    ref = R.Recon(Xs, R.RECON_ISING, lam=lam)
    for _ in range(2):
        d, _ = R.recon_score_noalloc(ctx.ctx, pairs)
        assert _close(d, ref.score(pairs)[0])


def test_noalloc_gaussian_and_limits(R):
    X = inputs.gaussian_torus_samples(8, 9, -0.2, 1.8, 300, 4000)
    ctx = R.Recon(np.ascontiguousarray(X.T.astype(np.float32)), R.RECON_GAUSSIAN, lam=1.0)
    pairs = inputs.random_pairs(72, 2000, 5)
    for _ in range(2):
        d_ref, _ = ctx.score(pairs)
        d, _ = R.recon_score_noalloc(ctx.ctx, pairs)
        assert _close(d, d_ref)
    with pytest.raises(R.ReconError) as e:
        R.recon_score_noalloc(ctx.ctx, np.zeros((65537, 2), dtype=np.int32) + [0, 1])
    assert e.value.status == R.RECON_EINVAL
    with pytest.raises(R.ReconError) as e:
        R.recon_score_noalloc(ctx.ctx, [[0, 72]])
    assert e.value.status == R.RECON_EINVAL
    d, w = R.recon_score_noalloc(ctx.ctx, np.zeros((0, 2), dtype=np.int32))
    assert len(d) == 0
    # the context stays usable after the rejected calls
    d, _ = R.recon_score_noalloc(ctx.ctx, pairs[:10])
    assert _close(d, ctx.score(pairs[:10])[0])
