"""The error bound the exact screen relies on (no GPU).  For the Ising model the
screen forms G_ij = sum_m (r_im x_jm + x_im r_jm) from rounded residuals
r~ = round(r) and exact spins x = +-1, so

    |G~_ij - G_ij| <= sum_m |r~_im - r_im| + sum_m |r~_jm - r_jm| = e_i + e_j

(before the accumulation's own rounding).  The rounding of both operand types
is emulated here from their definitions (bf16: 8 significant bits; E4M3: 4
significant bits, exponent bias 7, subnormal spacing 2^-9, round to nearest
even), the products are summed exactly in FP64, and the bound is checked for
every pair, next to the worst-case forms it replaces."""
import numpy as np
import pytest


def round_bf16(v):
    """float32 -> bf16 -> float32, round to nearest even."""
    b = np.asarray(v, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


def round_e4m3(v):
    """float32 -> E4M3 -> float64 (|v| < 448), round to nearest even."""
    v = np.asarray(v, dtype=np.float64)
    a = np.abs(v)
    e = np.floor(np.log2(np.where(a > 0, a, 1.0)))
    e = np.maximum(e, -6.0)  # below 2^-6 the spacing stays 2^-9 (subnormals)
    q = np.exp2(e - 3.0)
    return np.sign(v) * np.round(a / q) * q  # np.round: half to even


def _case(N, M, seed, spread):
    g = np.random.default_rng(seed)
    x = np.where(g.random((N, M)) < 0.5, -1.0, 1.0).astype(np.float32)
    # fields of various sizes, residuals r = x - tanh(phi) in FP32 as on the GPU
    phi = g.normal(0.0, spread, (N, M)).astype(np.float32)
    t = np.tanh(phi).astype(np.float32)
    r = (x - t).astype(np.float32)
    return x.astype(np.float64), r


def _g(ra, xa, rb, xb):
    return ra @ xb.T + xa @ rb.T  # exact enough: FP64 sums of |terms| < 2


@pytest.mark.parametrize("kind", ["bf16", "e4m3"])
@pytest.mark.parametrize("N,M,spread", [(40, 200, 0.3), (33, 500, 1.5), (25, 64, 4.0)])
def test_per_node_rounding_error_bounds_the_product(kind, N, M, spread):
    x, r = _case(N, M, 7 * N + M, spread)
    rr = (round_bf16(r) if kind == "bf16" else round_e4m3(r)).astype(np.float64)
    r64 = r.astype(np.float64)
    G = _g(r64, x, r64, x)
    Gt = _g(rr, x, rr, x)
    e = np.abs(rr - r64).sum(axis=1)
    bound = e[:, None] + e[None, :]
    assert np.all(np.abs(Gt - G) <= bound * (1 + 1e-12) + 1e-12)
    # the worst-case forms: 2^-8 sum|r| (bf16); 2^-4 sum|r| + 2^-10 per sample (E4M3)
    l1 = np.abs(r64).sum(axis=1)
    worst = l1 / 256.0 if kind == "bf16" else l1 / 16.0 + M / 1024.0
    assert np.all(e <= worst * (1 + 1e-9))
    # and the per-node form is the tighter one in practice
    assert e.sum() < 0.75 * worst.sum()


def test_emulated_roundings_match_their_definitions():
    # bf16 keeps 8 significant bits: 1 + 2^-8 ties to even (down), 1 + 3 2^-8 up
    assert round_bf16(np.float32(1 + 2 ** -8)) == 1.0
    assert round_bf16(np.float32(1 + 3 * 2 ** -8)) == np.float32(1 + 2 ** -6)
    # E4M3: spacing 2^-3 in [1, 2), 2^-9 below 2^-6, exact spins
    assert round_e4m3(1.0 + 2 ** -4) == 1.0  # tie to even
    assert round_e4m3(1.0 + 3 * 2 ** -4) == 1.25
    assert round_e4m3(2 ** -9 * 1.4) == 2 ** -9
    assert round_e4m3(-1.0) == -1.0 and round_e4m3(1.0) == 1.0
    v = np.linspace(-1.99, 1.99, 4001)
    rv = round_e4m3(v)
    assert np.all(np.abs(rv - v) <= np.maximum(np.abs(v) / 16.0, 2 ** -10) + 1e-15)
