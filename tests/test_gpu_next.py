"""GPU parity of the paths beyond the normal-equation core: the generalized least-squares solve (Sec. 1),
its symmetric product with A, A-CholQR2 reusing A Z, tridiagonal A (Sec. 8's second workload) and
PRE-CHOLQR (Sec. 3, Algorithm 2).  Each is compared with the CPU oracle element by element on small and
ragged sizes, and checked by properties at the benchmark's size.
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


def dev(torch, x, oqr):
    return oqr.colmajor(torch.as_tensor(np.asarray(x), dtype=torch.float64).cuda())


def host(x):
    return np.asfortranarray(x.cpu().numpy())


# ------------------------------------------------------------------ C = A B --
@pytest.mark.parametrize("m,k", [(1, 1), (63, 3), (64, 8), (65, 1), (1000, 11), (4097, 2)])
def test_symm_matches_oracle(env, m, k):
    """Tiles of 64 with ragged edges, one tile, several groups of 8 right-hand sides; the upper triangle
    of A holds NaN (never read)."""
    torch, oqr, ctx = env
    rng = np.random.default_rng(m + 13 * k)
    Bm = rng.standard_normal((m, m))
    A = Bm + Bm.T
    B = rng.standard_normal((m, k))
    P = A.copy()
    P[np.triu_indices(m, 1)] = np.nan
    C = host(ctx.oqr_symm(dev(torch, P, oqr), dev(torch, B, oqr)))
    Cr = oracle.symm_times(A, B)
    assert np.all(np.abs(C - Cr) <= 4 * m * U * (np.abs(A) @ np.abs(B)) + 1e-300)


def test_symm_exact_integers(env):
    torch, oqr, ctx = env
    rng = np.random.default_rng(3)
    m, k = 777, 5
    Bm = rng.integers(-4, 5, size=(m, m)).astype(np.float64)
    A = Bm + Bm.T
    B = rng.integers(-4, 5, size=(m, k)).astype(np.float64)
    assert np.array_equal(host(ctx.oqr_symm(dev(torch, A, oqr), dev(torch, B, oqr))), oracle.symm_times(A, B))


# ------------------------------------------------------------------- GLLS --
def test_glls_matches_oracle(env):
    """x = R^{-1} Q^T A b (Sec. 1) from the GPU's A-CholQR2, against the oracle's GLLS on config 0.

    The solution's sensitivity to the factorization is about kappa(R)^2 u (R's forward error, about
    kappa(R) u, amplified by R^{-1}), so the bound is 10 u kappa(R)^2 relative to ||x||."""
    torch, oqr, ctx = env
    A, Z = inputs.config0(seed=0)
    rng = np.random.default_rng(21)
    B = rng.standard_normal((A.shape[0], 3))
    Xr = oracle.glls(A, Z, B)
    _, Rr = oracle.oblique_qr(A, Z)
    kappa = np.linalg.cond(Rr)
    Ad = dev(torch, A, oqr)
    Q, R, _ = ctx.oqr_cholqr2(Ad, dev(torch, Z, oqr))
    X = host(ctx.oqr_glls(Ad, Q, R, dev(torch, B, oqr)))
    assert np.linalg.norm(X - Xr) / np.linalg.norm(Xr) <= max(1e-12, 10 * U * kappa ** 2)


def test_glls_consistent_system_and_normal_equations(env):
    """b = Z x0 returns x0; for a random b the residual is A-orthogonal to range(Z)."""
    torch, oqr, ctx = env
    A, Z = inputs.paper_case(4, 1500, 40, 1e4, 1e2, seed=31)
    rng = np.random.default_rng(31)
    x0 = rng.standard_normal((40, 1))
    Ad, Zd = dev(torch, A, oqr), dev(torch, Z, oqr)
    Q, R, _ = ctx.oqr_cholqr2(Ad, Zd)
    X = host(ctx.oqr_glls(Ad, Q, R, dev(torch, Z @ x0, oqr)))
    assert np.abs(X - x0).max() <= 1e-9 * np.abs(x0).max()
    b = rng.standard_normal((1500, 2))
    X = host(ctx.oqr_glls(Ad, Q, R, dev(torch, b, oqr)))
    g = Z.T @ A @ (b - Z @ X)
    assert np.abs(g).max() <= 1e-9 * (np.abs(Z).T @ np.abs(A) @ np.abs(b)).max()


def test_glls_full_size_normal_equations(env):
    """m = 32768, n = 256 (the benchmark's instance) with the mixed A-CholQR2's (Q, R): the residual of
    the solution is A-orthogonal to range(Z), measured with torch's FP64 GEMMs."""
    torch, oqr, ctx = env
    m, n = 32768, 256
    Af, _ = inputs.dense_spd(m, 1e6, seed=101, device="cuda")
    Z = inputs.tall_z(m, n, 1e2, seed=102, device="cuda")
    A = oqr.colmajor(Af)
    Q, R, _ = ctx.oqr_cholqr2(A, oqr.colmajor(Z.clone()), prec=4, final_prec=3)
    g = torch.Generator(device="cuda").manual_seed(5)
    b = oqr.colmajor(torch.randn((m, 1), dtype=torch.float64, device="cuda", generator=g))
    x = ctx.oqr_glls(A, Q, R, b)
    r = b - Z @ x
    grad = Z.T @ (Af @ r)
    scale = (Z.abs().T @ (Af.abs() @ b.abs())).max()
    assert (grad.abs().max() / scale).item() <= 1e-10
    del Af, A
    torch.cuda.empty_cache()


# ------------------------------------------------------- A-CholQR2 reusing W --
def test_cholqr2_reuse_w_against_its_restatement(env):
    """A-CholQR2 with W = A Z kept (A Q_1 = W R_1^{-1}) on config 0 and on a ragged shape, against the same
    steps restated on the CPU: R and the orthogonality within 100 x the restatement's own error (the
    variant is not exact: its loss of orthogonality keeps one factor of kappa), and never worse than
    one-pass CHOLQR."""
    torch, oqr, ctx = env
    for A, Z in (inputs.config0(seed=0), inputs.paper_case(4, 777, 33, 1e4, 1e3, seed=6)):
        Qr, Rr = oracle.oblique_qr(A, Z)
        Qc, Rc = oracle.cholqr2_reuse_w(A, Z)
        Q, R, (st, info) = ctx.oqr_cholqr2(dev(torch, A, oqr), dev(torch, Z, oqr), reuse_w=1, check=1)
        Q, R = host(Q), host(R)
        assert st == 0 and np.all(np.tril(R, -1) == 0) and np.all(np.diag(R) > 0)
        relR, relRc = (np.linalg.norm(X - Rr) / np.linalg.norm(Rr) for X in (R, Rc))
        orth, orthc = oracle.orth_error(A, Q), oracle.orth_error(A, Qc)
        assert relR <= max(1e-12, 100 * relRc)
        assert orth <= max(1e-13, 100 * orthc)
        assert orth <= oracle.orth_error(A, oracle.cholqr(A, Z)[0])
        assert oracle.repres_error(Z, Q, R) <= 1e-13


def test_cholqr2_reuse_w_rejects_other_options(env):
    torch, oqr, ctx = env
    A, Z = inputs.paper_case(4, 200, 8, 1e2, 1e1, seed=2)
    for kw in ({"shifted": 1}, {"prec": 3, "final_prec": 3}, {"passes": 3}):
        _, _, (st, _) = ctx.oqr_cholqr2(dev(torch, A, oqr), dev(torch, Z, oqr), reuse_w=1, raise_on_error=False,
                                        **kw)
        assert st == oqr.OQR_ERR_UNSUPPORTED


# ------------------------------------------------------------- tridiagonal A --
def _tri(torch, d, e):
    return (torch.as_tensor(np.ascontiguousarray(d), dtype=torch.float64).cuda(),
            torch.as_tensor(np.ascontiguousarray(e if len(e) else np.zeros(1)), dtype=torch.float64).cuda())


@pytest.mark.parametrize("prec", [0, 3])
@pytest.mark.parametrize("m,n", [(1, 1), (2, 2), (63, 20), (300, 37), (1000, 130), (2049, 64)])
def test_gram_tridiag_matches_oracle(env, m, n, prec):
    """G = Z^T T Z for tridiagonal T, FP64 (DFMA GEMM) and FP64-accurate tensor cores, against the oracle's
    Gram of the dense T; exactly symmetric."""
    torch, oqr, ctx = env
    rng = np.random.default_rng(m + n)
    d = 2.0 + rng.random(m)
    e = rng.standard_normal(m - 1)
    Z = rng.standard_normal((m, n))
    dd, ed = _tri(torch, d, e)
    G = host(ctx.oqr_gram_tridiag(dd, ed, dev(torch, Z, oqr), prec=prec))
    T = oracle.tridiag_dense(d, e)
    Gr = oracle.gram(T, Z)
    assert np.array_equal(G, G.T)
    scale = np.abs(Z).T @ np.abs(T) @ np.abs(Z)
    assert np.all(np.abs(G - Gr) <= 8 * U * scale * max(m, 2)), np.max(np.abs(G - Gr) / scale)


@pytest.mark.parametrize("kw", [{"passes": 1}, {}, {"shifted": 1}, {"prec": 4, "final_prec": 3},
                                {"prec": 3, "final_prec": 3}, {"shifted": 1, "prec": 3, "final_prec": 3}])
def test_cholqr2_tridiag_matches_oracle(env, kw):
    """The normal-equation method on a tridiagonal A against the tridiagonal oracle (m = 3000, n = 48,
    kappa(T) = 1e4, kappa(Z) = 1e2); one-pass CHOLQR is held to 100 x its own CPU restatement's error."""
    torch, oqr, ctx = env
    m, n = 3000, 48
    d, e = inputs.tridiag_spd(m, 1e4)
    _, Z = inputs.paper_case(4, m, n, 1e2, 1e2, seed=77)
    Qr, Rr = oracle.oblique_qr_tridiag(d, e, Z)
    dd, ed = _tri(torch, d, e)
    Q, R, (st, info) = ctx.oqr_cholqr2_tridiag(dd, ed, dev(torch, Z, oqr), check=1, **kw)
    Q, R = host(Q), host(R)
    assert st == 0
    assert np.all(np.tril(R, -1) == 0) and np.all(np.diag(R) > 0)
    relR = np.linalg.norm(R - Rr) / np.linalg.norm(Rr)
    orth = oracle.orth_error_tridiag(d, e, Q)
    if kw.get("passes") == 1:
        T = oracle.tridiag_dense(d, e)
        Qc, Rc = oracle.cholqr(T, Z)
        assert relR <= max(1e-12, 100 * np.linalg.norm(Rc - Rr) / np.linalg.norm(Rr))
        assert orth <= max(1e-12, 100 * oracle.orth_error(T, Qc))
    else:
        assert relR <= 1e-12
        assert orth <= max(1e-12, 10 * oracle.orth_error_tridiag(d, e, Qr))
        assert 0 <= info.orth_err <= 1e-12              # the library's own check of the result
    assert oracle.repres_error(Z, Q, R) <= 1e-13


@pytest.mark.parametrize("n", [64, 256])
def test_cholqr2_tridiag_paper_size(env, n):
    """Sec. 8's tridiagonal workload, m = 100000: the mixed A-CholQR2 (TC2 then FP64-accurate pass) and
    the FP64 one against the tridiagonal oracle's R, with Q^T T Q - I and Z - Q R measured by torch on the
    GPU."""
    torch, oqr, ctx = env
    m = 100000
    d, e = inputs.tridiag_spd(m, 1e4)
    Zt = inputs.tall_z(m, n, 1e2, seed=9, device="cuda")
    Zh = Zt.cpu().numpy()
    _, Rr = oracle.oblique_qr_tridiag(d, e, Zh)
    Rr = torch.as_tensor(Rr).cuda()
    kappa = np.linalg.cond(Rr.cpu().numpy())
    dd, ed = _tri(torch, d, e)
    for kw in ({"prec": 4, "final_prec": 3}, {}):
        Q, R, (st, _) = ctx.oqr_cholqr2_tridiag(dd, ed, oqr.colmajor(Zt.clone()), **kw)
        assert st == 0
        TQ = dd[:, None] * Q
        TQ[1:] += ed[:m - 1, None] * Q[:-1]
        TQ[:-1] += ed[:m - 1, None] * Q[1:]
        E = Q.T @ TQ - torch.eye(n, dtype=torch.float64, device="cuda")
        orth = torch.linalg.eigvalsh(0.5 * (E + E.T)).abs().max().item()
        relR = (torch.linalg.matrix_norm(R - Rr) / torch.linalg.matrix_norm(Rr)).item()
        rep = (torch.linalg.matrix_norm(Zt - Q @ R, 2) / torch.linalg.matrix_norm(Zt, 2)).item()
        assert relR <= max(1e-12, 100 * U * kappa), (kw, relR)
        assert orth <= 1e-12 and rep <= 1e-13, (kw, orth, rep)


# ------------------------------------------------------------- PRE-CHOLQR --
@pytest.mark.parametrize("m,n", [(1, 1), (5, 3), (256, 256), (300, 20), (2000, 20), (4097, 64), (3000, 300),
                                 (70001, 8), (9000, 1)])
def test_tsqr_matches_lapack(env, m, n):
    """The Euclidean Householder TSQR (one leaf; odd and even node counts; a deep tree; n = 1) against
    LAPACK's QR with its signs normalised: S within 1e-13 of R_lapack, Y orthonormal to working precision
    and within kappa(Z) u of Q_lapack."""
    torch, oqr, ctx = env
    rng = np.random.default_rng(m + 7 * n)
    Z = rng.standard_normal((m, n)) @ np.diag(np.logspace(0, 3, n))
    Y, S = ctx.oqr_tsqr(dev(torch, Z, oqr))
    Y, S = host(Y), host(S)
    Ql, Rl = np.linalg.qr(Z)
    D = np.where(np.diag(Rl) < 0, -1.0, 1.0)
    Ql, Rl = Ql * D, (Rl.T * D).T
    assert np.all(np.tril(S, -1) == 0) and np.all(np.diag(S) > 0)
    assert np.linalg.norm(S - Rl) / np.linalg.norm(Rl) <= 1e-13
    assert np.abs(Y.T @ Y - np.eye(n)).max() <= 20 * np.sqrt(m) * n * U
    assert np.abs(Y - Ql).max() <= 100 * np.linalg.cond(Z) * U
    assert np.linalg.norm(Z - Y @ S) / np.linalg.norm(Z) <= 10 * n * U


@pytest.mark.parametrize("m,n", [(3000, 100), (1500, 64)])
def test_blocked_householder_ill_conditioned(env, m, n):
    """The blocked Householder QR (n > 32: TSQR panels, reconstructed Householder vectors, GEMM updates) at
    kappa(Z) = 1e12: Y orthonormal and Z = Y S to working precision, as Householder QR is backward stable
    whatever kappa(Z); at kappa(Z) = 1e3 (the same sizes) S is LAPACK's R within 1e-13."""
    torch, oqr, ctx = env
    _, Z = inputs.paper_case(4, m, n, 1.0, 1e12, seed=m + n)
    Y, S = ctx.oqr_tsqr(dev(torch, Z, oqr))
    Y, S = host(Y), host(S)
    assert np.all(np.tril(S, -1) == 0) and np.all(np.diag(S) > 0)
    assert np.linalg.norm(Y.T @ Y - np.eye(n), 2) <= 20 * np.sqrt(m) * n * U
    assert np.linalg.norm(Z - Y @ S, 2) / np.linalg.norm(Z, 2) <= 10 * n * U
    _, Z = inputs.paper_case(4, m, n, 1.0, 1e3, seed=m + n)
    _, S = ctx.oqr_tsqr(dev(torch, Z, oqr))
    _, Rl = np.linalg.qr(Z)
    Rl = (Rl.T * np.where(np.diag(Rl) < 0, -1.0, 1.0)).T
    assert np.linalg.norm(host(S) - Rl) / np.linalg.norm(Rl) <= 1e-13


def _pre_orth_bound(A, Q, m, n):
    """Thm 3.1's bound c m n^2 u ||Q||_2^2 ||A||_2 with c = 1."""
    return m * n * n * U * np.linalg.norm(Q, 2) ** 2 * np.linalg.eigvalsh(A).max()


@pytest.mark.parametrize("final_prec", [0, 3])
def test_precholqr_config0_parity(env, final_prec):
    """PRE-CHOLQR (Algorithm 2) on config 0, FP64 and FP64-accurate CHOLQR pass: the oracle's (Q, R)."""
    torch, oqr, ctx = env
    A, Z = inputs.config0(seed=0)
    m, n = Z.shape
    Qr, Rr = oracle.oblique_qr(A, Z)
    Q, R, (st, _) = ctx.oqr_precholqr(dev(torch, A, oqr), dev(torch, Z, oqr), final_prec=final_prec)
    Q, R = host(Q), host(R)
    assert st == 0 and np.all(np.tril(R, -1) == 0) and np.all(np.diag(R) > 0)
    kappa = np.linalg.cond(Rr)
    assert np.linalg.norm(R - Rr) / np.linalg.norm(Rr) <= max(1e-12, 100 * U * kappa)
    orth = oracle.orth_error(A, Q)
    assert orth <= min(_pre_orth_bound(A, Q, m, n), max(1e-11, 100 * oracle.orth_error(A, Qr)))
    assert oracle.repres_error(Z, Q, R) <= 1e-13


@pytest.mark.parametrize("n", [20, 80])
def test_precholqr_orthogonality_independent_of_kappa_z(env, n):
    """Thm 3.1: PRE-CHOLQR's loss of orthogonality does not grow with kappa(Z).  The same A (m = 2000,
    kappa(A) = 1e4), kappa(Z) = 1e2 and 1e8: the orthogonality stays within 10x, inside the theorem's
    bound, while one-pass CHOLQR at kappa(Z) = 1e8 breaks down or loses at least 1000x more; R is the
    oracle's within 100 u kappa(R).  n = 20: the TSQR; n = 80: the blocked Householder QR."""
    torch, oqr, ctx = env
    m = 2000
    orths = []
    for kz in (1e2, 1e8):
        A, Z = inputs.paper_case(4, m, n, 1e4, kz, seed=8)
        Qr, Rr = oracle.oblique_qr(A, Z)
        Ad = dev(torch, A, oqr)
        Q, R, (st, _) = ctx.oqr_precholqr(Ad, dev(torch, Z, oqr))
        Q, R = host(Q), host(R)
        assert st == 0
        assert np.linalg.norm(R - Rr) / np.linalg.norm(Rr) <= max(1e-12, 100 * U * np.linalg.cond(Rr))
        orths.append(oracle.orth_error(A, Q))
        assert orths[-1] <= _pre_orth_bound(A, Q, m, n)
        assert oracle.repres_error(Z, Q, R) <= 1e-13
        if kz == 1e8:   # one-pass CHOLQR breaks down or loses orthogonality (Thm 2.1: u kappa^2)
            Q1, _, (st1, _) = ctx.oqr_cholqr(Ad, dev(torch, Z, oqr), raise_on_error=False)
            assert st1 == oqr.OQR_ERR_NOT_SPD or oracle.orth_error(A, host(Q1)) >= 1e3 * orths[-1]
    assert orths[1] <= 10 * orths[0] + 1e-15, orths


def test_precholqr_in_place_and_tridiagonal(env):
    """Q aliasing Z, and PRE-CHOLQR on a tridiagonal A against the tridiagonal oracle (kappa(Z) = 1e8)."""
    torch, oqr, ctx = env
    A, Z = inputs.paper_case(4, 900, 30, 1e3, 1e2, seed=5)
    Qr, Rr = oracle.oblique_qr(A, Z)
    Zd = dev(torch, Z, oqr)
    Q, R, _ = ctx.oqr_precholqr(dev(torch, A, oqr), Zd, Q=Zd)
    assert Q.data_ptr() == Zd.data_ptr()
    assert np.linalg.norm(host(R) - Rr) / np.linalg.norm(Rr) <= 1e-12
    m, n = 5000, 40
    d, e = inputs.tridiag_spd(m, 1e4)
    _, Z = inputs.paper_case(4, m, n, 1e2, 1e8, seed=15)
    Qr, Rr = oracle.oblique_qr_tridiag(d, e, Z)
    dd, ed = _tri(torch, d, e)
    Q, R, (st, _) = ctx.oqr_precholqr_tridiag(dd, ed, dev(torch, Z, oqr))
    Q, R = host(Q), host(R)
    assert st == 0
    assert np.linalg.norm(R - Rr) / np.linalg.norm(Rr) <= max(1e-12, 100 * U * np.linalg.cond(Rr))
    assert oracle.orth_error_tridiag(d, e, Q) <= max(1e-12, 100 * oracle.orth_error_tridiag(d, e, Qr))


# ---------------------------------------------------------- A-CGS2 at full size --
def test_cgs2_full_size_stable_in_kappa_z(env):
    """Block A-CGS2 at m = 32768, n = 256, kappa(A) = 1e6, kappa(Z) = 1e8 (config 1's hardest cell): Thm 6.4
    bounds its loss of orthogonality by c m^{3/2} n u ||A|| ||Q||^2, independent of kappa(Z), as A-CholQR2's;
    held to 10x A-CholQR2's orthogonality on the same instance (both measured by torch's FP64 GEMMs)."""
    torch, oqr, ctx = env
    m, n = 32768, 256
    Af, _ = inputs.dense_spd(m, 1e6, seed=301, device="cuda")
    A = oqr.colmajor(Af)
    Z = oqr.colmajor(inputs.tall_z(m, n, 1e8, seed=311, device="cuda"))
    orth = {}
    for name in ("oqr_cholqr2", "oqr_cgs2"):
        Q, R, (st, _) = getattr(ctx, name)(A, Z)
        assert st == 0
        E = Q.T @ (Af @ Q) - torch.eye(n, dtype=torch.float64, device="cuda")
        orth[name] = torch.linalg.eigvalsh(0.5 * (E + E.T)).abs().max().item()
        rep = (torch.linalg.matrix_norm(Z - Q @ R, 2) / torch.linalg.matrix_norm(Z, 2)).item()
        assert rep <= 1e-13, (name, rep)
    assert orth["oqr_cgs2"] <= max(1e-12, 10 * orth["oqr_cholqr2"]), orth
    del Af, A
    torch.cuda.empty_cache()
