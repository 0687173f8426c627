"""Stored expected values (tests/golden/ising_n12_m64.json, written by
tests/golden/make_golden.py from the FP64 oracle alone): the oracle must keep
reproducing them, and the CUDA path must match them within the parity
tolerances (gains 1e-5 relative plus 1e-5 of the largest gain, objectives
1e-6 relative) without calling the oracle."""
import json
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
REL, FLOOR, OBJ_REL = 1e-5, 1e-5, 1e-6


@pytest.fixture(scope="module")
def golden():
    with open(os.path.join(HERE, "golden", "ising_n12_m64.json")) as f:
        d = json.load(f)
    d["X"] = np.asarray(d["X"], dtype=np.int8)
    for k in ("pairs", "best_pairs"):
        d[k] = np.asarray(d[k], dtype=np.int32)
    for k in ("gain", "w", "fields_w0"):
        d[k] = np.asarray(d[k], dtype=np.float64)
    return d


def test_oracle_reproduces_the_stored_values(oracle, golden):
    d = golden
    o = oracle.IsingOracle(d["X"], d["lambda"], w_clamp=d["w_clamp"])
    assert np.allclose(o.h, d["fields_w0"], rtol=1e-12, atol=1e-12)
    g, w = o.score(d["pairs"])
    assert np.allclose(g, d["gain"], rtol=1e-10, atol=1e-10 * float(d["gain"].max()))
    assert np.allclose(w, d["w"], rtol=1e-8, atol=1e-10)
    assert o.objective() == pytest.approx(d["objective_w0"], rel=1e-12)
    best = oracle.exhaustive_best(o.dist_matrix(), d["N"])
    assert np.array_equal(np.asarray(best), d["best_pairs"])
    o.update(d["best_pairs"])
    assert o.objective() == pytest.approx(d["objective_after_sweep"], rel=1e-12)


@pytest.mark.gpu
def test_cuda_path_matches_the_stored_values(golden):
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__

    __graft_entry__.build()
    from paper_2401_01404_gb300 import recon as R

    d = golden
    ctx = R.Recon(np.ascontiguousarray(d["X"].T), R.RECON_ISING, lam=d["lambda"], w_clamp=d["w_clamp"])
    assert ctx.objective() == pytest.approx(d["objective_w0"], rel=OBJ_REL)
    _, _, h = ctx.get_model()
    assert np.allclose(h, d["fields_w0"], rtol=1e-5, atol=1e-5)
    dd, w = ctx.score(d["pairs"])
    g = -np.asarray(dd, dtype=np.float64)
    tol = REL * np.abs(d["gain"]) + FLOOR * float(d["gain"].max())
    assert np.all(np.abs(g - d["gain"]) <= tol)
    assert np.allclose(w, d["w"], rtol=1e-3, atol=1e-4)
    ctx.cd_sweep(d["best_pairs"])
    assert ctx.objective() == pytest.approx(d["objective_after_sweep"], rel=OBJ_REL)
