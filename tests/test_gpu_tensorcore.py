"""GPU parity of the tensor-core normal-equation matrix (tcgen05, BF16 slices).

BF16X3 is held to its own definition: x = hi + lo with hi, lo the
round-to-nearest-even BF16 values of x and of x - hi (computed exactly here in
numpy), G_def = Z_hi^T M_hi Z_hi + ... summed as the three products
hi*hi + hi*lo + lo*hi in FP64, then symmetrised; the GPU differs from G_def
only by FP32 accumulation.  FP64_TC is held to the FP64 oracle's Gram at
FP64-level tolerance.  The mixed A-CholQR2 (BF16X3 or FP64_TC passes, FP64_TC
last) is held to the CHOL-EQR oracle with the FP64 path's tolerances.
"""
import numpy as np
import pytest

import oracle
from paper_1401_5171_gb300 import inputs

pytestmark = pytest.mark.gpu
U = 2.0 ** -53


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1401_5171_gb300 import oqr
    return torch, oqr, oqr.Oqr(0)


def dev(torch, oqr, x):
    return oqr.colmajor(torch.as_tensor(np.asarray(x), dtype=torch.float64).cuda())


def bf16_rne(x):
    """Round to the nearest BF16 value (8 significant bits), ties to even; exact in float64."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)                       # x = m 2^e, |m| in [0.5, 1)
    q = np.rint(m * 256.0)                   # 8 significant bits, numpy rint = ties to even
    return np.ldexp(q / 256.0, e)


def split_def(x):
    hi = bf16_rne(x)
    lo = bf16_rne(x - hi)
    return hi, lo


def lower_m(A):
    Ml = np.tril(A, -1) + 0.5 * np.diag(np.diag(A))
    return Ml


def test_bf16_rounding_definition_matches_torch():
    import torch
    x = np.random.default_rng(0).standard_normal(10000) * 10.0 ** np.random.default_rng(1).integers(-20, 20, 10000)
    t = torch.as_tensor(x.astype(np.float32)).to(torch.bfloat16).double().numpy()
    # through float32 first only differs when the float32 rounding creates a tie; compare on float32 inputs
    assert np.array_equal(bf16_rne(x.astype(np.float32).astype(np.float64)), t)


SHAPES = [(1, 1), (64, 5), (200, 20), (1000, 130), (2000, 20), (3000, 300)]


@pytest.mark.parametrize("m,n", SHAPES)
def test_tc_gram_bf16x3_definition(env, m, n):
    torch, oqr, ctx = env
    A, Z = inputs.paper_case(4, m, n, 1e4, 1e2, seed=m + 3 * n)
    G = ctx.oqr_gram(dev(torch, oqr, A), dev(torch, oqr, Z), prec=oqr.OQR_BF16X3).cpu().numpy()
    Mh, Ml = split_def(lower_m(A))
    Zh, Zl = split_def(Z)
    U1 = Mh @ Zh + Mh @ Zl + Ml @ Zh                 # the three products, FP64
    Uh, Ul = split_def(U1)
    C = Zh.T @ Uh + Zh.T @ Ul + Zl.T @ Uh
    Gdef = C + C.T
    scale = np.abs(Z).T @ np.abs(A) @ np.abs(Z)
    assert np.array_equal(G, G.T)
    # FP32 accumulation over pieces of 2048 plus the second product's split of U
    assert np.all(np.abs(G - Gdef) <= 2.0 ** -12 * scale + 1e-300)
    # and the method's own accuracy against the FP64 oracle: ~3 * 2^-16 per product
    assert np.all(np.abs(G - oracle.gram(A, Z)) <= 2.0 ** -11 * scale + 1e-300)


@pytest.mark.parametrize("m,n", SHAPES)
def test_tc_gram_fp64tc_matches_fp64(env, m, n):
    torch, oqr, ctx = env
    A, Z = inputs.paper_case(4, m, n, 1e6, 1e3, seed=m + 5 * n)
    P = A.copy()
    P[np.triu_indices(m, 1)] = np.nan            # upper triangle never used
    G = ctx.oqr_gram(dev(torch, oqr, P), dev(torch, oqr, Z), prec=oqr.OQR_FP64_TC).cpu().numpy()
    Gr = oracle.gram(A, Z)
    scale = np.abs(Z).T @ np.abs(A) @ np.abs(Z)
    assert np.array_equal(G, G.T)
    assert np.all(np.abs(G - Gr) <= 8 * m * U * scale + 1e-300)


def test_tc_gram_fp64tc_exact_integers(env):
    # integer A and Z whose products and sums are exact: the emulation must be exact too
    torch, oqr, ctx = env
    rng = np.random.default_rng(11)
    m, n = 700, 70
    B = rng.integers(-50, 51, size=(m, m)).astype(np.float64)
    A = np.tril(B) + np.tril(B, -1).T
    A[np.diag_indices(m)] = 2.0 * rng.integers(-50, 51, size=m)   # even diagonal: diag/2 exact
    Z = rng.integers(-30, 31, size=(m, n)).astype(np.float64)
    G = ctx.oqr_gram(dev(torch, oqr, A), dev(torch, oqr, Z), prec=oqr.OQR_FP64_TC).cpu().numpy()
    assert np.array_equal(G, Z.T @ A @ Z)


@pytest.mark.parametrize("prec,final", [(3, 3), (1, 3), (0, 3)])
def test_mixed_cholqr2_parity(env, prec, final):
    torch, oqr, ctx = env
    # kappa(A^{1/2} Z) ~ 1e2: the BF16X3 first pass completes
    A, Z = inputs.paper_case(4, 1500, 40, 1e4, 1e2, seed=77)
    Qr, Rr = oracle.oblique_qr(A, Z)
    Q, R, (st, info) = ctx.oqr_cholqr2(dev(torch, oqr, A), dev(torch, oqr, Z), prec=prec, final_prec=final)
    Q, R = Q.cpu().numpy(), R.cpu().numpy()
    assert np.all(np.tril(R, -1) == 0) and np.all(np.diag(R) > 0)
    assert np.linalg.norm(R - Rr) / np.linalg.norm(Rr) <= 1e-12
    assert oracle.orth_error(A, Q) <= max(1e-12, 10 * oracle.orth_error(A, Qr))


def test_fp64tc_cholqr2_config0(env):
    torch, oqr, ctx = env
    A, Z = inputs.config0(seed=0)
    Qr, Rr = oracle.oblique_qr(A, Z)
    Q, R, _ = ctx.oqr_cholqr2(dev(torch, oqr, A), dev(torch, oqr, Z), prec=oqr.OQR_FP64_TC,
                              final_prec=oqr.OQR_FP64_TC)
    Q, R = Q.cpu().numpy(), R.cpu().numpy()
    assert np.linalg.norm(R - Rr) / np.linalg.norm(Rr) <= 1e-12
    assert oracle.orth_error(A, Q) <= max(1e-12, 10 * oracle.orth_error(A, Qr))
