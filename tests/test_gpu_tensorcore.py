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
from split_defs import bf16_rne, e4m3_quantize, tc2_cols, tc2_rows

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


def split_def(x):
    hi = bf16_rne(x)
    lo = bf16_rne(x - hi)
    return hi, lo


def lower_m(A):
    Ml = np.tril(A, -1) + 0.5 * np.diag(np.diag(A))
    return Ml


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


@pytest.mark.parametrize("m,n", [(700, 24), (520, 80)])
def test_tc_gram_fp64tc_near_exact(env, m, n):
    # Held to Z^T A Z formed in extended precision (np.longdouble: 64- or 113-bit
    # significand), not to the FP64 oracle: the slices keep 55 bits of each
    # element relative to its 256-chunk maximum and the chunk sums are exact, so
    # what remains is the double-float (about 2^-48) accumulation of U = M Z and
    # C = Z^T U and the final FP64 sum.  Several 256-chunks, a ragged tail, and
    # two column chunks of 64 at n = 80.
    torch, oqr, ctx = env
    A, Z = inputs.paper_case(4, m, n, 1e6, 1e3, seed=m + 7 * n)
    G = ctx.oqr_gram(dev(torch, oqr, A), dev(torch, oqr, Z), prec=oqr.OQR_FP64_TC).cpu().numpy()
    Ml = lower_m(A).astype(np.longdouble)
    Zl = Z.astype(np.longdouble)
    C = Zl.T @ (Ml @ Zl)
    Gx = C + C.T
    scale = np.abs(Z).T @ np.abs(A) @ np.abs(Z)
    err = np.max(np.abs((G.astype(np.longdouble) - Gx) / scale))
    assert err <= 2.0 ** -44, err


@pytest.mark.parametrize("m,n", [(64, 5), (300, 20), (1000, 130), (2000, 200)])
def test_tc_gram_tc2_definition(env, m, n):
    # TC2 keeps the two leading FP64_TC slices: M~ per (row, 256-chunk), Z~ per (column, 256-chunk);
    # G_def = Z~^T U~ + (Z~^T U~)^T with U~ the same truncation of U_def = M~ Z~.  The GPU differs by
    # FP32 accumulation, and U~ by one truncation step where U and U_def straddle a boundary.
    torch, oqr, ctx = env
    A, Z = inputs.paper_case(4, m, n, 1e4, 1e2, seed=m + 11 * n)
    G = ctx.oqr_gram(dev(torch, oqr, A), dev(torch, oqr, Z), prec=oqr.OQR_TC2).cpu().numpy()
    Mt, Zt = tc2_rows(lower_m(A)), tc2_cols(Z)
    Ut = tc2_cols(Mt @ Zt)
    C = Zt.T @ Ut
    Gdef = C + C.T
    scale = np.abs(Z).T @ np.abs(A) @ np.abs(Z)
    assert np.array_equal(G, G.T)
    assert np.all(np.abs(G - Gdef) <= 2.0 ** -14 * scale + 1e-300)
    assert np.all(np.abs(G - oracle.gram(A, Z)) <= 2.0 ** -11 * scale + 1e-300)


def test_shared_split_matches_separate_steps(env):
    # A-CholQR2 with a TC2 then an FP64_TC pass splits A once for both passes; composing the same
    # steps from separate calls (each splitting A itself; the first pass solves with oqr_trsm_tc, the
    # last with oqr_trsm_last) must give bit-identical Q and R
    torch, oqr, ctx = env
    A, Z = inputs.paper_case(4, 1100, 70, 1e5, 1e2, seed=21)
    Ad, Zd = dev(torch, oqr, A), dev(torch, oqr, Z)
    Q, R, (st, _) = ctx.oqr_cholqr2(Ad, Zd, prec=oqr.OQR_TC2, final_prec=oqr.OQR_FP64_TC)
    G1 = ctx.oqr_gram(Ad, Zd, prec=oqr.OQR_TC2)
    R1, st1, _ = ctx.oqr_potrf(G1)
    Q1 = ctx.oqr_trsm_tc(Zd, R1)
    G2 = ctx.oqr_gram(Ad, Q1, prec=oqr.OQR_FP64_TC)
    R2, st2, _ = ctx.oqr_potrf(G2)
    Q2 = ctx.oqr_trsm_last(G2, Q1, R2)
    Rm = ctx.oqr_rprod(R2, R1)
    assert st == st1 == st2 == oqr.OQR_OK
    assert torch.equal(Q, Q2) and torch.equal(R, Rm)


@pytest.mark.parametrize("prec,final", [(3, 3), (1, 3), (0, 3), (4, 3)])
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


# ------------------------------------------------------------------- FP8 ----
def chunk_exponents(X, axis_len=128):
    """frexp exponent of each 128-row chunk's largest magnitude, per column (K x C input)."""
    K, C = X.shape
    out = np.zeros(((K + axis_len - 1) // axis_len, C), dtype=int)
    for kc in range(out.shape[0]):
        mx = np.abs(X[kc * axis_len:(kc + 1) * axis_len]).max(axis=0)
        out[kc] = np.where(mx > 0, np.frexp(mx)[1], 0)
    return out


def quantize_tall(X):
    E = chunk_exponents(X)
    Q = np.empty_like(X, dtype=np.float64)
    for kc in range(E.shape[0]):
        sl = slice(kc * 128, (kc + 1) * 128)
        Q[sl] = e4m3_quantize(X[sl], E[kc][None, :])
    return Q


def test_tc_gram_fp8_definition_integers(env):
    # integer M and Z are exact in E4M3 after their power-of-two scaling; U = M Z is
    # then exact, and only U's own quantization (defined above) enters G
    torch, oqr, ctx = env
    rng = np.random.default_rng(17)
    m, n = 700, 24
    B = rng.integers(-7, 8, size=(m, m)).astype(np.float64)
    A = np.tril(B) + np.tril(B, -1).T
    A[np.diag_indices(m)] = 2.0 * rng.integers(-7, 8, size=m)
    Z = rng.integers(-15, 16, size=(m, n)).astype(np.float64)
    M = np.tril(A, -1) + 0.5 * np.diag(np.diag(A))
    U = M @ Z
    Uq = quantize_tall(U)
    C = Z.T @ Uq
    Gdef = C + C.T
    G = ctx.oqr_gram(dev(torch, oqr, A), dev(torch, oqr, Z), prec=oqr.OQR_FP8).cpu().numpy()
    assert np.array_equal(G, G.T)
    assert np.max(np.abs(G - Gdef)) <= 1e-6 * np.abs(Gdef).max()


def test_tc_gram_fp8_error_bound(env):
    torch, oqr, ctx = env
    A, Z = inputs.paper_case(4, 1500, 40, 1e2, 1e1, seed=31)
    G = ctx.oqr_gram(dev(torch, oqr, A), dev(torch, oqr, Z), prec=oqr.OQR_FP8).cpu().numpy()
    Gr = oracle.gram(A, Z)
    # three E4M3 roundings (M, Z, U) at 2^-4 relative each, against |Z|^T |A| |Z|
    scale = np.abs(Z).T @ np.abs(A) @ np.abs(Z)
    assert np.all(np.abs(G - Gr) <= 0.25 * scale)
    assert np.linalg.norm(G - Gr) / np.linalg.norm(Gr) <= 0.1


def test_mixed_cholqr2_fp8_first_pass(env):
    torch, oqr, ctx = env
    A, Z = inputs.paper_case(4, 1200, 32, 1e1, 2.0, seed=41)    # kappa(A^{1/2} Z) ~ 2
    Qr, Rr = oracle.oblique_qr(A, Z)
    Q, R, (st, info) = ctx.oqr_cholqr2(dev(torch, oqr, A), dev(torch, oqr, Z), prec=oqr.OQR_FP8,
                                       final_prec=oqr.OQR_FP64_TC, raise_on_error=False)
    assert st == 0
    Q, R = Q.cpu().numpy(), R.cpu().numpy()
    assert np.linalg.norm(R - Rr) / np.linalg.norm(Rr) <= 1e-12
    assert oracle.orth_error(A, Q) <= max(1e-12, 10 * oracle.orth_error(A, Qr))


def test_precision_study_per_kappa(env):
    """Precision study at m=2048, n=64, kappa(A)=1e6: kappa(A^{1/2} Z) set to 1e1..1e7
    through case-2 columns of V (the n largest eigenvalues) and kappa(Z).  Reports the
    Gram error of BF16X3 and FP8 and the orthogonality of the mixed A-CholQR2 variants
    against the FP64 oracle; asserts what the method guarantees."""
    torch, oqr, ctx = env
    m, n = 2048, 64
    rows = []
    for kz in (1e1, 1e3, 1e5, 1e7):
        A, Z = inputs.paper_case(2, m, n, 1e6, kz, seed=int(np.log10(kz)))
        Qr, Rr = oracle.oblique_qr(A, Z)
        kap = np.linalg.cond(Rr)
        Gr = oracle.gram(A, Z)
        Ad, Zd = dev(torch, oqr, A), dev(torch, oqr, Z)
        eg = {}
        for name, prec in (("bf16x3", oqr.OQR_BF16X3), ("fp8", oqr.OQR_FP8)):
            G = ctx.oqr_gram(Ad, Zd, prec=prec).cpu().numpy()
            eg[name] = np.linalg.norm(G - Gr, 2) / np.linalg.norm(Gr, 2)
        orth = {}
        for name, kw in (("bf16x3->fp64tc", dict(prec=1, final_prec=3)),
                         ("fp8->fp64tc", dict(prec=2, final_prec=3)),
                         ("shifted bf16x3->fp64tc->fp64tc", dict(shifted=1, prec=1, prec_mid=3, final_prec=3)),
                         ("shifted fp8->fp64tc->fp64tc", dict(shifted=1, prec=2, prec_mid=3, final_prec=3))):
            Q, R, (st, info) = ctx.oqr_cholqr2(Ad, Zd, raise_on_error=False, **kw)
            orth[name] = oracle.orth_error(A, Q.cpu().numpy()) if st == 0 else float("inf")
        rows.append((kap, eg, orth))
        print(f"\nkappa(A^1/2 Z)={kap:.1e}: Gram error bf16x3 {eg['bf16x3']:.1e} fp8 {eg['fp8']:.1e}; orth " +
              ", ".join(f"{k} {v:.1e}" for k, v in orth.items()))
        assert eg["bf16x3"] <= 1e-4 and eg["fp8"] <= 0.2
        if kap <= 1e3:
            assert orth["bf16x3->fp64tc"] <= max(1e-12, 10 * oracle.orth_error(A, Qr))
        if kap <= 1e7:
            assert orth["shifted bf16x3->fp64tc->fp64tc"] <= max(1e-12, 10 * oracle.orth_error(A, Qr))


# ------------------------------------------------------- host-buffer path ----
@pytest.mark.parametrize("prec,final", [(4, 3), (0, 0), (3, 3)])
def test_cholqr2_host_matches_device(env, prec, final):
    # host buffers: A's lower triangle copied in 256-column panels (m = 1100: a ragged last panel), the
    # split of A made panel by panel; Q and R must equal the device-buffer call bit for bit
    import torch
    torch_, oqr, ctx = env
    m, n = 1100, 70
    A, Z = inputs.paper_case(4, m, n, 1e5, 1e2, seed=33)
    Qd, Rd, (st, _) = ctx.oqr_cholqr2(dev(torch, oqr, A), dev(torch, oqr, Z), prec=prec, final_prec=final)
    Ah = torch.from_numpy(np.asfortranarray(A)).t().contiguous().pin_memory().t()
    Ah[torch.triu_indices(m, m, 1).unbind()] = float("nan")        # the upper triangle is never read
    Zh = torch.from_numpy(np.asfortranarray(Z)).t().contiguous().pin_memory().t()
    Qh, Rh, (sth, info) = ctx.oqr_cholqr2_host(Ah, Zh, prec=prec, final_prec=final)
    assert st == sth == oqr.OQR_OK
    assert torch.equal(Qh, Qd.cpu()) and torch.equal(Rh, Rd.cpu())


def test_cholqr2_host_padded_pageable(env):
    # leading dimensions larger than m and n, pageable (not pinned) host memory
    import torch
    torch_, oqr, ctx = env
    m, n = 700, 24
    A, Z = inputs.paper_case(4, m, n, 1e4, 1e2, seed=34)
    Apad = np.zeros((m + 5, m), order="F"); Apad[:m] = A
    Zpad = np.zeros((m + 3, n), order="F"); Zpad[:m] = Z
    Ah = torch.from_numpy(Apad)[:m]
    Zh = torch.from_numpy(Zpad)[:m]
    Qh = torch.zeros((n, m + 2), dtype=torch.float64).t()[:m]
    Rh = torch.zeros((n, n + 1), dtype=torch.float64).t()[:n]
    Qh2, Rh2, (st, _) = ctx.oqr_cholqr2_host(Ah, Zh, Q=Qh, R=Rh, prec=oqr.OQR_TC2, final_prec=oqr.OQR_FP64_TC)
    Qr, Rr = oracle.oblique_qr(A, Z)
    assert st == oqr.OQR_OK
    assert np.linalg.norm(Rh.numpy() - Rr) / np.linalg.norm(Rr) <= 1e-12
    assert oracle.orth_error(A, Qh.numpy()) <= max(1e-12, 10 * oracle.orth_error(A, Qr))
