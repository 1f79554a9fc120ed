"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

The oracle is CHOL-EQR (Algorithm 3) in plain C; the unique oblique QR it
returns is what every normal-equation variant must reach.  Tolerances
(FP64 path, kappa(A^{1/2} Z) <= 1e3): ||R - R_ref|| / ||R|| <= 1e-12 and
||Q^T A Q - I||_2 <= max(1e-12, 10 x the oracle's own), with the
orthogonality of the GPU's Q measured on the CPU in long double.  One-pass
A-CholQR is held to 100 x the error of the same algorithm restated on the
CPU (Thm 2.1: its error grows like kappa^2).  Step kernels are compared
element by element with the oracle's definitions.
"""
import math

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


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


# --------------------------------------------------------------- step kernels --
@pytest.mark.parametrize("m,n", [(1, 1), (7, 3), (128, 64), (300, 37), (1000, 130), (2000, 20), (513, 257)])
def test_gram_matches_oracle(env, m, n):
    torch, oqr, ctx = env
    rng = np.random.default_rng(m * 7 + n)
    B = rng.standard_normal((m, m))
    A = B + B.T + 2 * m * np.eye(m)
    Z = rng.standard_normal((m, n))
    P = A.copy()
    P[np.triu_indices(m, 1)] = np.nan          # the upper triangle is never used
    G = host(ctx.oqr_gram(dev(torch, P, oqr), dev(torch, Z, oqr)))
    Gr = oracle.gram(A, Z)
    assert np.array_equal(G, G.T)              # exactly symmetric by construction
    scale = np.abs(Z).T @ np.abs(A) @ np.abs(Z)
    assert np.all(np.abs(G - Gr) <= 4 * m * U * scale + 1e-300)


def test_gram_odd_leading_dimension_plain_path(env):
    torch, oqr, ctx = env
    m, n = 301, 45
    rng = np.random.default_rng(5)
    B = rng.standard_normal((m, m))
    A = B @ B.T
    Z = rng.standard_normal((m, n))
    # lda = m + 2 = 303: its byte stride is not a multiple of 16, so TMA cannot address A
    Ab = torch.zeros((m, m + 2), dtype=torch.float64, device="cuda")
    Ab[:, :m] = torch.as_tensor(A.T)
    Am = Ab.t()[:m]
    assert Am.stride(0) == 1 and Am.stride(1) == m + 2
    Zm = dev(torch, Z, oqr)
    G = host(ctx.oqr_gram(Am, Zm))
    scale = np.abs(Z).T @ np.abs(A) @ np.abs(Z)
    assert np.all(np.abs(G - oracle.gram(A, Z)) <= 4 * m * U * scale)


@pytest.mark.parametrize("n", [1, 5, 32, 33, 100, 257, 512])
def test_potrf_matches_oracle(env, n):
    torch, oqr, ctx = env
    rng = np.random.default_rng(n)
    B = rng.standard_normal((n, n))
    G = B @ B.T + n * np.eye(n)
    P = G.copy()
    P[np.triu_indices(n, 1)] = np.nan
    R, st, info = ctx.oqr_potrf(dev(torch, P, oqr))
    assert st == oqr.OQR_OK and info == 0
    R = host(R)
    Rr = oracle.chol_upper(G)
    assert np.all(np.tril(R, -1) == 0)
    assert rel(R, Rr) < 1e-13


def test_potrf_pascal_exact(env):
    torch, oqr, ctx = env
    n = 12
    P = np.array([[math.comb(i + j, i) for j in range(n)] for i in range(n)], dtype=np.float64)
    R, st, _ = ctx.oqr_potrf(dev(torch, P, oqr))
    assert st == oqr.OQR_OK
    assert np.array_equal(host(R), oracle.chol_upper(P))


@pytest.mark.parametrize("n,col", [(4, 3), (40, 35), (70, 1)])
def test_potrf_breakdown_column(env, n, col):
    torch, oqr, ctx = env
    d = np.ones(n)
    d[col - 1] = -1.0
    G = np.diag(d)
    with pytest.raises(oracle.OracleBreakdown) as e:
        oracle.chol_upper(G)
    R, st, info = ctx.oqr_potrf(dev(torch, G, oqr))
    assert st == oqr.OQR_ERR_NOT_SPD and info == e.value.column == col


def test_potrf_shift(env):
    torch, oqr, ctx = env
    n = 50
    rng = np.random.default_rng(3)
    B = rng.standard_normal((n, n))
    G = B @ B.T + np.eye(n)
    R, st, _ = ctx.oqr_potrf(dev(torch, G, oqr), shift=2.5)
    assert rel(host(R), oracle.chol_upper(G + 2.5 * np.eye(n))) < 1e-13


@pytest.mark.parametrize("m,n", [(1, 1), (63, 20), (1000, 33), (3000, 64), (3000, 65), (2000, 129), (4097, 300),
                                 (640, 512)])
def test_trsm_tc_matches_oracle(env, m, n):
    # blocked solve: FP64-accurate tensor-core products off the diagonal, FP64 substitution in the
    # 64 x 64 diagonal blocks; single block, a ragged last block and several blocks
    torch, oqr, ctx = env
    rng = np.random.default_rng(m + 7 * n)
    R = np.triu(rng.standard_normal((n, n))) + 3 * np.eye(n)
    Z = rng.standard_normal((m, n))
    Qr = oracle.trsm_right_upper(Z, R)
    Q = host(ctx.oqr_trsm_tc(dev(torch, Z, oqr), dev(torch, R, oqr)))
    assert rel(Q, Qr) < 1e-13
    Zd = dev(torch, Z, oqr)
    ctx.oqr_trsm_tc(Zd, dev(torch, R, oqr), Q=Zd)
    assert rel(host(Zd), Qr) < 1e-13


def test_trsm_tc_rowwise_backward_error(env):
    # R the Cholesky factor of an ill-conditioned Gram (kappa(R) ~ 1e6): every row q of Q = Z / R
    # satisfies |z - q R| <= c u |q| |R| up to a modest constant, as row-wise substitution does (Sec. 2)
    torch, oqr, ctx = env
    A, Z = inputs.paper_case(4, 2500, 150, 1e4, 1e5, seed=4)
    R = oracle.chol_upper(oracle.gram(A, Z))
    Q = host(ctx.oqr_trsm_tc(dev(torch, Z, oqr), dev(torch, R, oqr)))
    Qf = host(ctx.oqr_trsm(dev(torch, Z, oqr), dev(torch, R, oqr)))
    res = np.abs(Z - Q @ R).max(axis=1) / (np.abs(Q) @ np.abs(R)).max(axis=1)
    res_f = np.abs(Z - Qf @ R).max(axis=1) / (np.abs(Qf) @ np.abs(R)).max(axis=1)
    assert res.max() <= 4 * 150 * 2.0 ** -53, (res.max(), res_f.max())


def _near_identity_gram(rng, n, frob):
    """G = I + E, E symmetric with ||E||_F = frob, and R = chol(G) (upper, from the oracle)."""
    E = rng.standard_normal((n, n))
    E = E + E.T
    G = np.eye(n) + frob * E / np.linalg.norm(E)
    return G, oracle.chol_upper(G)


@pytest.mark.parametrize("m,n", [(1, 1), (63, 20), (1000, 33), (3000, 65), (2000, 130), (4097, 256)])
def test_trsm_last_near_identity(env, m, n):
    # ||G - I||_F <= 0.5: Q = Z R^{-1} as one FP64-accurate product with the explicit inverse.  R's
    # condition is at most sqrt(3), so the result matches the substitution at rounding level and every
    # row's backward error |z - q R| stays within a small multiple of n u |q| |R|
    torch, oqr, ctx = env
    rng = np.random.default_rng(3 * m + n)
    G, R = _near_identity_gram(rng, n, 0.45)
    Z = rng.standard_normal((m, n))
    Qr = oracle.trsm_right_upper(Z, R)
    Gd, Rd = dev(torch, G, oqr), dev(torch, R, oqr)
    Q = host(ctx.oqr_trsm_last(Gd, dev(torch, Z, oqr), Rd))
    assert rel(Q, Qr) < 1e-14
    res = np.abs(Z - Q @ R).max(axis=1) / (np.abs(Q) @ np.abs(R)).max(axis=1)
    assert res.max() <= 4 * n * U
    Zd = dev(torch, Z, oqr)
    ctx.oqr_trsm_last(Gd, Zd, Rd, Q=Zd)  # in place
    assert np.array_equal(host(Zd), Q)
    if m * n >= 1000:  # the product route ran, not the substitution (their roundings differ somewhere)
        assert not np.array_equal(Q, host(ctx.oqr_trsm(dev(torch, Z, oqr), Rd)))


@pytest.mark.parametrize("m,n", [(63, 20), (3000, 65), (2000, 130)])
def test_trsm_last_far_from_identity_is_the_rowwise_solve(env, m, n):
    # ||G - I||_F > 0.5 (here 0.6, and a Gram of condition ~1e6): FP64 row-wise substitution runs, bit for bit
    torch, oqr, ctx = env
    rng = np.random.default_rng(5 * m + n)
    cases = [_near_identity_gram(rng, n, 0.6)]
    A, Zc = inputs.paper_case(4, 2 * n + 10, n, 1e4, 1e3, seed=n)
    Gc = oracle.gram(A, Zc)
    cases.append((Gc, oracle.chol_upper(Gc)))
    for G, R in cases:
        Z = rng.standard_normal((m, n))
        Gd, Rd = dev(torch, G, oqr), dev(torch, R, oqr)
        Q = host(ctx.oqr_trsm_last(Gd, dev(torch, Z, oqr), Rd))
        assert np.array_equal(Q, host(ctx.oqr_trsm(dev(torch, Z, oqr), Rd)))
        assert rel(Q, oracle.trsm_right_upper(Z, R)) < 1e-9


@pytest.mark.parametrize("m,n", [(1, 1), (63, 20), (1000, 33), (2000, 20), (4097, 300), (640, 512)])
def test_trsm_matches_oracle(env, m, n):
    torch, oqr, ctx = env
    rng = np.random.default_rng(m + n)
    R = np.triu(rng.standard_normal((n, n))) + 3 * np.eye(n)
    Z = rng.standard_normal((m, n))
    Q = host(ctx.oqr_trsm(dev(torch, Z, oqr), dev(torch, R, oqr)))
    Qr = oracle.trsm_right_upper(Z, R)
    assert rel(Q, Qr) < 1e-13
    # in place
    Zd = dev(torch, Z, oqr)
    ctx.oqr_trsm(Zd, dev(torch, R, oqr), Q=Zd)
    assert rel(host(Zd), Qr) < 1e-13


def test_trsm_exact_integers(env):
    torch, oqr, ctx = env
    rng = np.random.default_rng(4)
    m, n = 200, 70
    R = np.triu(rng.integers(-3, 4, size=(n, n))).astype(np.float64)
    np.fill_diagonal(R, 2.0 ** rng.integers(0, 3, size=n))
    Q0 = rng.integers(-2, 3, size=(m, n)).astype(np.float64)
    Z = Q0 @ R
    assert np.abs(Z).max() < 2 ** 40
    assert np.array_equal(host(ctx.oqr_trsm(dev(torch, Z, oqr), dev(torch, R, oqr))), Q0)


@pytest.mark.parametrize("n", [1, 9, 64, 200])
def test_rprod_exact(env, n):
    torch, oqr, ctx = env
    rng = np.random.default_rng(n)
    Uu = np.triu(rng.integers(-5, 6, size=(n, n))).astype(np.float64)
    S = np.triu(rng.integers(-5, 6, size=(n, n))).astype(np.float64)
    assert np.array_equal(host(ctx.oqr_rprod(dev(torch, Uu, oqr), dev(torch, S, oqr))), oracle.upper_times_upper(Uu, S))


# --------------------------------------------------------------- whole path --
def factor(ctx, name, torch, oqr, A, Z, **kw):
    Q, R, (st, info) = getattr(ctx, name)(dev(torch, A, oqr), dev(torch, Z, oqr), **kw)
    return host(Q), host(R), info


@pytest.mark.parametrize("name,kw", [("oqr_cholqr2", {}), ("oqr_cholqr2", {"shifted": 1}),
                                     ("oqr_cgs2", {}), ("oqr_cgs2", {"block": 7})])
def test_config0_parity(env, name, kw):
    torch, oqr, ctx = env
    A, Z = inputs.config0(seed=0)
    Qr, Rr = oracle.oblique_qr(A, Z)
    orth_ref = oracle.orth_error(A, Qr)
    Q, R, info = factor(ctx, name, torch, oqr, A, Z, **kw)
    assert np.all(np.tril(R, -1) == 0) and np.all(np.diag(R) > 0)
    assert rel(R, Rr) <= 1e-12
    assert oracle.orth_error(A, Q) <= max(1e-12, 10 * orth_ref)
    assert rel(Q, Qr) <= 1e-10
    assert oracle.repres_error(Z, Q, R) <= 1e-13


def test_config0_one_pass_cholqr(env):
    torch, oqr, ctx = env
    A, Z = inputs.config0(seed=0)
    Qr, Rr = oracle.oblique_qr(A, Z)
    Qc, Rc = oracle.cholqr(A, Z)                       # the same algorithm on the CPU
    Q, R, _ = factor(ctx, "oqr_cholqr", torch, oqr, A, Z)
    assert rel(R, Rr) <= max(100 * rel(Rc, Rr), 1e-12)
    assert oracle.orth_error(A, Q) <= max(100 * oracle.orth_error(A, Qc), 1e-12)
    assert oracle.repres_error(Z, Q, R) <= 1e-13


@pytest.mark.parametrize("case", [1, 2, 3, 4, 5])
def test_paper_cases_cholqr2(env, case):
    # Sec. 7 cases at m=80, n=10, kappa(A)=1e6, kappa(Z)=1e3.  The attainable
    # accuracy is set by ||A|| ||Q||^2 (Thm 4.1; between sigma_1/sigma_n and
    # kappa(A), Sec. 7), so R is held to max(1e-12, 100 u ||A|| ||Q||^2).
    torch, oqr, ctx = env
    A, Z = inputs.paper_case(case, 80, 10, 1e6, 1e3 if case != 5 else None, seed=40 + case)
    Qr, Rr = oracle.oblique_qr(A, Z)
    floor = 100 * U * np.linalg.eigvalsh(A).max() * np.linalg.norm(Qr, 2) ** 2
    Q, R, _ = factor(ctx, "oqr_cholqr2", torch, oqr, A, Z)
    assert rel(R, Rr) <= max(1e-12, floor)
    assert oracle.orth_error(A, Q) <= max(1e-12, 10 * oracle.orth_error(A, Qr))
    if case == 5:                                  # exact factors: R = I, Q = Z
        assert np.abs(R - np.eye(10)).max() <= max(1e-12, floor)


@pytest.mark.parametrize("m,n", [(1, 1), (2, 2), (5, 1), (64, 64), (129, 65), (1000, 130), (777, 100)])
def test_ragged_and_edge_shapes(env, m, n):
    torch, oqr, ctx = env
    A, Z = inputs.paper_case(4, m, n, 1e3, 1e1, seed=m + n)
    Qr, Rr = oracle.oblique_qr(A, Z)
    Q, R, _ = factor(ctx, "oqr_cholqr2", torch, oqr, A, Z)
    assert rel(R, Rr) <= 1e-12
    assert oracle.orth_error(A, Q) <= 1e-12


def test_in_place_and_upper_triangle_garbage(env):
    torch, oqr, ctx = env
    A, Z = inputs.paper_case(4, 500, 40, 1e4, 1e2, seed=9)
    Qr, Rr = oracle.oblique_qr(A, Z)
    P = A.copy()
    P[np.triu_indices(500, 1)] = np.nan
    Ad, Zd = dev(torch, P, oqr), dev(torch, Z, oqr)
    Q, R, _ = ctx.oqr_cholqr2(Ad, Zd, Q=Zd)
    assert Q.data_ptr() == Zd.data_ptr()
    assert rel(host(R), Rr) <= 1e-12 and oracle.orth_error(A, host(Q)) <= 1e-12


def test_not_spd_reports_breakdown(env):
    torch, oqr, ctx = env
    m, n = 200, 10
    A = np.eye(m)
    A[3, 3] = -1.0                                 # indefinite A
    Z = np.zeros((m, n))
    Z[:n, :n] = np.eye(n)
    Q, R, (st, info) = ctx.oqr_cholqr(dev(torch, A, oqr), dev(torch, Z, oqr), raise_on_error=False)
    assert st == oqr.OQR_ERR_NOT_SPD and info.info == 4


def test_check_matches_oracle(env):
    torch, oqr, ctx = env
    A, Z = inputs.config0(seed=1)
    Q, R, _ = factor(ctx, "oqr_cholqr", torch, oqr, A, Z)   # one pass: visible loss of orthogonality
    o2, oF, E = ctx.oqr_check(dev(torch, A, oqr), dev(torch, Q, oqr), want_E=True)
    Er = oracle.orth_defect(A, Q)
    ref2 = float(np.max(np.abs(np.linalg.eigvalsh(0.5 * (Er + Er.T)))))
    assert abs(o2 - ref2) <= 0.05 * ref2 + 1e-14
    assert abs(oF - np.linalg.norm(Er)) <= 0.01 * np.linalg.norm(Er) + 1e-14
    _, _, (st, info) = ctx.oqr_cholqr2(dev(torch, A, oqr), dev(torch, Z, oqr), check=1)
    assert 0 <= info.orth_err < 1e-12


# ---------------------------------------------------- full size, properties --
FULL_PATHS = {
    # name: (kwargs of oqr_cholqr2)
    "fp64": {},
    "fp64_shifted": {"shifted": 1},
    "mixed_tc2_fp64tc": {"prec": 4, "final_prec": 3},        # the benchmark's headline path
    "all_fp64tc": {"prec": 3, "final_prec": 3},
    "bf16x3_fp64tc": {"prec": 1, "final_prec": 3},
    "shifted_all_fp64tc": {"shifted": 1, "prec": 3, "final_prec": 3},
}


@pytest.fixture(scope="module")
def full_size(env):
    """m=32768, n=256, kappa(A)=1e6, kappa(Z)=1e2: the benchmark's workload, and the R of the
    FP64 (DFMA) A-CholQR2, the path pinned to the oracle element by element at small sizes."""
    torch, oqr, ctx = env
    m, n = 32768, 256
    Af, _ = inputs.dense_spd(m, 1e6, seed=101, device="cuda")
    Z = inputs.tall_z(m, n, 1e2, seed=102, device="cuda")
    A = oqr.colmajor(Af)
    _, R64, (st, _) = ctx.oqr_cholqr2(A, oqr.colmajor(Z.clone()))
    assert st == 0
    G = Z.T @ (Af @ Z)
    ev = torch.linalg.eigvalsh(0.5 * (G + G.T)).clamp_min(0).sqrt().sort().values
    yield {"Af": Af, "A": A, "Z": Z, "R64": R64, "ev": ev}
    torch.cuda.empty_cache()


@pytest.mark.parametrize("path", list(FULL_PATHS))
def test_config1_full_size_properties(env, full_size, path):
    """Every A-CholQR2 path at the benchmark's launch configuration (m=32768, n=256).

    No oracle runs at this size: Q^T A Q = I, Z = Q R, R upper with a positive
    diagonal and sigma(R)^2 = eig(Z^T A Z) (Thm 1.1) together fix (Q, R); each is
    measured with torch's own FP64 GEMM/eigensolver on the GPU.  R is also
    compared with the DFMA path's R within max(1e-12, 100 u kappa(R)): the
    forward error of a normal-equation R grows with kappa(A^{1/2} Z) (Thm 2.1).
    """
    torch, oqr, ctx = env
    Af, A, Z, R64, ev = (full_size[k] for k in ("Af", "A", "Z", "R64", "ev"))
    n = Z.shape[1]
    Q, R, (st, info) = ctx.oqr_cholqr2(A, oqr.colmajor(Z.clone()), **FULL_PATHS[path])
    assert st == 0
    E = Q.T @ (Af @ Q) - torch.eye(n, dtype=torch.float64, device="cuda")
    orth = torch.linalg.eigvalsh(0.5 * (E + E.T)).abs().max().item()
    rep = (torch.linalg.matrix_norm(Z - Q @ R, 2) / torch.linalg.matrix_norm(Z, 2)).item()
    assert torch.all(torch.tril(R, -1) == 0) and torch.all(torch.diagonal(R) > 0)
    sv = torch.linalg.svdvals(R).sort().values
    assert torch.max((sv - ev).abs() / ev.max()).item() < 1e-10
    kappa = (ev[-1] / ev[0]).item()
    relR = (torch.linalg.matrix_norm(R - R64) / torch.linalg.matrix_norm(R64)).item()
    assert relR <= max(1e-12, 100 * U * kappa), (relR, kappa)
    assert orth < 1e-11 and rep < 1e-13, (orth, rep)


def test_repres_planted_residual(env):
    """oqr_repres on Z' = Q R + E with a planted rank-one E and a clear top singular value of Z':
    both ratios against numpy's norms."""
    torch, oqr, ctx = env
    rng = np.random.default_rng(71)
    m, n = 900, 40
    Uz, _ = np.linalg.qr(rng.standard_normal((m, n)))
    Wz, _ = np.linalg.qr(rng.standard_normal((n, n)))
    sig = np.concatenate([[10.0], np.linspace(1.0, 0.1, n - 1)])
    Z = (Uz * sig) @ Wz.T
    Qh, Rh = np.linalg.qr(Z)
    D = np.sign(np.diag(Rh))
    Q, R = Qh * D, (Rh.T * D).T                        # Z = Q R, R upper with a positive diagonal
    u, v = rng.standard_normal(m), rng.standard_normal(n)
    E = 1e-5 * np.outer(u / np.linalg.norm(u), v / np.linalg.norm(v))   # far above Q R's rounding
    Zp = Z + E
    r2, rf = ctx.oqr_repres(*(oqr.colmajor(torch.as_tensor(x).cuda()) for x in (Zp, Q, R)))
    ref2 = np.linalg.norm(Zp - Q @ R, 2) / np.linalg.norm(Zp, 2)
    refF = np.linalg.norm(Zp - Q @ R) / np.linalg.norm(Zp)
    assert abs(r2 - ref2) <= 1e-6 * ref2
    assert abs(rf - refF) <= 1e-6 * refF


def test_repres_of_factorization(env):
    """The representativity of an A-CholQR2 result is at the rounding level (Sec. 7: about 1e-15)."""
    torch, oqr, ctx = env
    A, Z = inputs.paper_case(4, 700, 30, 1e6, 1e4, seed=3)
    Ad, Zd = (oqr.colmajor(torch.as_tensor(x).cuda()) for x in (A, Z))
    Q, R, _ = ctx.oqr_cholqr2(Ad, Zd)
    r2, rf = ctx.oqr_repres(Zd, Q, R)
    ref = oracle.repres_error(Z, Q.cpu().numpy(), R.cpu().numpy())
    assert r2 <= max(4 * ref, 1e-15) and r2 <= 1e-13
    assert rf <= 1e-13


# ------------------------------------------------------------- shift value --
@pytest.mark.parametrize("prec", ["fp64", "fp64tc", "bf16x3", "tc2"])
def test_shift_value_matches_its_formula(env, prec):
    """The shift of shifted A-CholQR3's first pass, recomputed on the CPU from its definition.

    FP64 or FP64-accurate first pass: s = 11 u (m n + n (n + 1)) ||A||_F ||Z||_F^2, u = 2^-53
    (||A||_F of the symmetric A whose lower triangle is read).  BF16X3 or TC2 first pass:
    s = 11 u_eff trace(G), u_eff = 2^-16, G that pass's low-precision Z^T A Z, whose trace agrees
    with the exact trace(Z^T A Z) to about 2^-16.  A wrong constant, norm or unit roundoff
    changes s by far more than these tolerances.
    """
    torch, oqr, ctx = env
    m, n = 1500, 48
    A, Z = inputs.paper_case(4, m, n, 1e4, 1e6, seed=17)
    P = np.tril(A)                                       # the upper triangle must not enter ||A||_F
    P[np.triu_indices(m, 1)] = 7.0
    # (first pass, later passes): a low-precision first pass is followed by FP64-accurate passes
    code = {"fp64": (0, 0), "fp64tc": (3, 3), "bf16x3": (1, 3), "tc2": (4, 3)}[prec]
    _, _, (st, info) = ctx.oqr_cholqr2(dev(torch, P, oqr), dev(torch, Z, oqr), shifted=1, prec=code[0],
                                       prec_mid=code[1], final_prec=code[1])
    assert st == 0
    if prec in ("fp64", "fp64tc"):
        ref = 11 * U * (m * n + n * (n + 1)) * np.linalg.norm(A) * np.linalg.norm(Z) ** 2
        assert abs(info.shift - ref) <= 1e-12 * ref, (info.shift, ref)
    else:
        ref = 11 * 2.0 ** -16 * np.trace(Z.T @ A @ Z)
        assert abs(info.shift - ref) <= 1e-3 * ref, (info.shift, ref)
