"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test pins one oracle function to something other than itself: exact
integer arithmetic, closed forms, a library routine in a special case the
paper names (A = I reduces to the Euclidean QR, Sec. 1), Theorem 1.1's
singular-value identities, test case 5's exact factors (Sec. 7), planted
factors, and a 50-digit brute force on tiny inputs.  The mutation test at the
end checks that plausible mistakes planted in the oracle fail these pins.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1401_5171_gb300 import inputs

U = 2.0 ** -53


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300)


# ---------------------------------------------------------------- Cholesky --
def pascal(n):
    return np.array([[math.comb(i + j, i) for j in range(n)] for i in range(n)], dtype=np.float64)


def test_chol_pascal_exact():
    # Symmetric Pascal matrix P = L L^T, L_ij = binom(i, j): the upper factor is L^T exactly.
    n = 12
    L = np.array([[math.comb(i, j) for j in range(n)] for i in range(n)], dtype=np.float64)
    C = oracle.chol_upper(pascal(n))
    assert np.array_equal(C, L.T)


def test_chol_reads_lower_triangle_only():
    rng = np.random.default_rng(1)
    B = rng.standard_normal((30, 30))
    A = B @ B.T + 30 * np.eye(30)
    P = A.copy()
    P[np.triu_indices(30, 1)] = np.nan
    assert np.array_equal(oracle.chol_upper(A), oracle.chol_upper(P))


def test_chol_matches_lapack():
    rng = np.random.default_rng(2)
    B = rng.standard_normal((60, 60))
    A = B @ B.T + np.eye(60)
    C = oracle.chol_upper(A)
    assert rel(C, np.linalg.cholesky(A).T) < 1e-12
    assert np.all(np.tril(C, -1) == 0) and np.all(np.diag(C) > 0)


@pytest.mark.parametrize("A,col", [
    (np.diag([1.0, 2.0, -1.0, 3.0]), 3),
    (np.array([[1.0, 2.0], [2.0, 1.0]]), 2),
    (np.array([[0.0, 0.0], [0.0, 1.0]]), 1),
    (np.array([[1.0, 0.0], [0.0, np.nan]]), 2),
])
def test_chol_breakdown_column(A, col):
    with pytest.raises(oracle.OracleBreakdown) as e:
        oracle.chol_upper(A)
    assert e.value.column == col


# ------------------------------------------------------------ Gram / products --
def int_sym(rng, m, lo=-5, hi=6):
    B = rng.integers(lo, hi, size=(m, m))
    return np.tril(B) + np.tril(B, -1).T


def test_symm_times_and_gram_exact_integers():
    rng = np.random.default_rng(3)
    m, n = 17, 5
    Ai = int_sym(rng, m)
    Zi = rng.integers(-4, 5, size=(m, n))
    A = Ai.astype(np.float64)
    A_poison = A.copy()
    A_poison[np.triu_indices(m, 1)] = 1e300       # upper triangle is never read
    Bx = [[sum(int(Ai[i, k]) * int(Zi[k, c]) for k in range(m)) for c in range(n)] for i in range(m)]
    Gx = [[sum(int(Zi[i, r]) * Bx[i][c] for i in range(m)) for c in range(n)] for r in range(n)]
    assert np.array_equal(oracle.symm_times(A_poison, Zi), np.array(Bx, dtype=np.float64))
    assert np.array_equal(oracle.gram(A_poison, Zi), np.array(Gx, dtype=np.float64))


def test_gram_not_symmetric_input_orientation():
    # G = Z^T A Z, not Z A Z^T or Z^T A^T Z with a transposed lower triangle.
    A = np.array([[2.0, 0.0], [1.0, 3.0]])  # lower triangle: a21 = 1 -> A = [[2,1],[1,3]]
    Z = np.array([[1.0, 2.0], [0.0, 1.0]])
    As = np.array([[2.0, 1.0], [1.0, 3.0]])
    assert np.array_equal(oracle.gram(A, Z), Z.T @ As @ Z)


def test_trsm_exact_integers():
    rng = np.random.default_rng(4)
    m, n = 23, 7
    R = np.triu(rng.integers(-3, 4, size=(n, n))).astype(np.float64)
    np.fill_diagonal(R, 2.0 ** rng.integers(0, 3, size=n))
    Q0 = rng.integers(-6, 7, size=(m, n)).astype(np.float64)
    Z = Q0 @ R                                    # exact: small integers
    assert np.array_equal(oracle.trsm_right_upper(Z, R), Q0)


def test_trsm_matches_scipy():
    import scipy.linalg as sl
    rng = np.random.default_rng(5)
    m, n = 40, 9
    R = np.triu(rng.standard_normal((n, n))) + 4 * np.eye(n)
    Z = rng.standard_normal((m, n))
    ref = sl.solve_triangular(R, Z.T, trans="T", lower=False).T
    assert rel(oracle.trsm_right_upper(Z, R), ref) < 1e-13


def test_upper_times_upper_exact():
    rng = np.random.default_rng(6)
    n = 9
    Uu = np.triu(rng.integers(-5, 6, size=(n, n))).astype(np.float64)
    S = np.triu(rng.integers(-5, 6, size=(n, n))).astype(np.float64)
    assert np.array_equal(oracle.upper_times_upper(Uu, S), Uu @ S)


# --------------------------------------------------------------- Householder --
def sign_fix(Q, R):
    s = np.sign(np.diag(R))
    s[s == 0] = 1
    return Q * s, R * s[:, None]


def test_householder_matches_lapack():
    rng = np.random.default_rng(7)
    W = rng.standard_normal((50, 8))
    Y, Rh = oracle.householder_qr(W)
    Yr, Rr = sign_fix(*np.linalg.qr(W))
    Yo, Ro = sign_fix(Y, Rh)
    assert rel(Ro, Rr) < 1e-13 and rel(Yo, Yr) < 1e-13
    assert np.abs(Y.T @ Y - np.eye(8)).max() < 1e-14
    assert rel(Y @ Rh, W) < 1e-14


# ---------------------------------------------------------------- the oracle --
def test_identity_metric_is_euclidean_qr():
    # Sec. 1: for A = I the oblique QR is the standard QR factorization.
    rng = np.random.default_rng(8)
    Z = rng.standard_normal((70, 6)) @ np.diag(10.0 ** np.arange(6))
    Q, R = oracle.oblique_qr(np.eye(70), Z)
    Qr, Rr = sign_fix(*np.linalg.qr(Z))
    assert rel(R, Rr) < 1e-13 and rel(Q, Qr) < 1e-12


def test_hand_worked_examples():
    A = np.array([[4.0, 2.0], [2.0, 3.0]])
    Q, R = oracle.oblique_qr(A, np.eye(2))
    Rx = np.array([[2.0, 1.0], [0.0, math.sqrt(2.0)]])
    assert np.allclose(R, Rx, rtol=0, atol=1e-15)
    assert np.allclose(Q, np.linalg.inv(Rx), rtol=0, atol=1e-15)
    A3 = np.diag([1.0, 4.0, 9.0])
    Z3 = np.array([[1.0, 0.0], [0.0, 1.0], [0.0, 0.0]])
    Q3, R3 = oracle.oblique_qr(A3, Z3)
    assert np.allclose(R3, np.diag([1.0, 2.0]), atol=1e-15)
    assert np.allclose(Q3, np.array([[1.0, 0.0], [0.0, 0.5], [0.0, 0.0]]), atol=1e-15)
    # a column that is a multiple of another after A-orthogonalisation: z2 = z1 + 3 e2
    A4 = np.array([[2.0, 1.0], [1.0, 2.0]])
    Z4 = np.array([[1.0, 1.0], [0.0, 3.0]])
    # A Z = [[2, 5], [1, 7]], G = Z^T A Z = [[2, 5], [5, 26]] -> R = [[sqrt2, 5/sqrt2], [0, sqrt(26 - 12.5)]]
    Q4, R4 = oracle.oblique_qr(A4, Z4)
    R4x = np.array([[math.sqrt(2), 5 / math.sqrt(2)], [0, math.sqrt(13.5)]])
    assert np.allclose(R4, R4x, rtol=1e-15, atol=1e-15)


def _mp_reference(A, Z, dps=50):
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = dps
    m, n = Z.shape
    Am = mpmath.matrix([[A[max(i, j), min(i, j)] for j in range(m)] for i in range(m)])
    Zm = mpmath.matrix(Z.tolist())
    G = Zm.T * Am * Zm
    R = mpmath.cholesky(G).T
    Q = Zm * R ** -1
    return (np.array(Q.tolist(), dtype=np.float64), np.array(R.tolist(), dtype=np.float64))


@pytest.mark.parametrize("seed,m,n,ka,kz", [(0, 6, 3, 1e2, 1e1), (1, 8, 4, 1e6, 1e3),
                                            (2, 12, 4, 1e10, 1e2), (3, 5, 5, 1e4, 1e4)])
def test_brute_force_50_digits(seed, m, n, ka, kz):
    A, Z = inputs.paper_case(4, m, n, ka, kz, seed=seed)
    Q, R = oracle.oblique_qr(A, Z)
    Qm, Rm = _mp_reference(A, Z)
    kap = np.linalg.cond(Rm)
    assert rel(R, Rm) < 50 * m * n * U * kap
    assert rel(Q, Qm) < 50 * m * n * U * kap * math.sqrt(ka)


def test_singular_values_theorem_1_1():
    rng = np.random.default_rng(9)
    m, n = 60, 6
    A, Z = inputs.paper_case(4, m, n, 1e4, 1e2, seed=11)
    w, V = np.linalg.eigh(A)
    Ah = (V * np.sqrt(w)) @ V.T
    Q, R = oracle.oblique_qr(A, Z)
    sR = np.linalg.svd(R, compute_uv=False)
    sAZ = np.linalg.svd(Ah @ Z, compute_uv=False)
    assert np.max(np.abs(sR - sAZ) / sAZ) < 1e-11
    Zhat = np.linalg.qr(Z)[0]
    sAZh = np.linalg.svd(Ah @ Zhat, compute_uv=False)
    sQ = np.linalg.svd(Q, compute_uv=False)
    assert np.max(np.abs(sQ - 1.0 / sAZh[::-1]) * sAZh[::-1]) < 1e-11


@pytest.mark.parametrize("ka", [1e2, 1e6, 1e10])
def test_case5_exact_factors(ka):
    # Sec. 7, case 5: Z is A-orthonormal, so R = I and Q = Z.
    A, Z = inputs.paper_case(5, 80, 10, ka, seed=12)
    Q, R = oracle.oblique_qr(A, Z)
    tol = 1e3 * 80 * U * ka
    assert np.abs(R - np.eye(10)).max() < tol
    assert np.abs(Q - Z).max() / np.abs(Z).max() < tol


def test_planted_factors():
    rng = np.random.default_rng(13)
    m, n = 50, 5
    A, _ = inputs.paper_case(4, m, n, 1e3, seed=14)
    C = np.linalg.cholesky(A).T
    Y0 = inputs.haar(rng, m, n)
    Q0 = np.linalg.solve(C, Y0)
    R0 = np.triu(rng.standard_normal((n, n)))
    np.fill_diagonal(R0, np.abs(np.diag(R0)) + 0.5)
    Q, R = oracle.oblique_qr(A, Q0 @ R0)
    assert rel(R, R0) < 1e-11 and rel(Q, Q0) < 1e-10


@pytest.mark.parametrize("case", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("ka", [1e1, 1e5, 1e10, 1e15])
def test_paper_cases_theorem_4_1_bounds(case, ka):
    # Sec. 7 sweep (m=80, n=10, kappa(Z) = kappa(A)^{1/2}) against the bounds of
    # Thm 4.1 for CHOL-EQR with the unknown constant c taken as 1:
    #   ||Q^T A Q - I||_2 <= c m n u ||A|| ||Q||^2,
    #   ||Z - Q R||_A    <= c m n^2 u ||A||^{1/2} || |Q| |R| ||_2.
    # ||.||_A of the residual is read from the Gram D^T A D, not from A^{1/2}.
    m, n = 80, 10
    A, Z = inputs.paper_case(case, m, n, ka, seed=20 + case)
    Q, R = oracle.oblique_qr(A, Z)
    assert np.all(np.tril(R, -1) == 0) and np.all(np.diag(R) > 0)
    normA = np.linalg.eigvalsh(A).max()
    assert oracle.orth_error(A, Q) <= m * n * U * normA * np.linalg.norm(Q, 2) ** 2
    D = oracle.repres_residual(Z, Q, R)
    repA = math.sqrt(max(np.linalg.eigvalsh(oracle.gram(A, D)).max(), 0.0))
    assert repA <= m * n * n * U * math.sqrt(normA) * np.linalg.norm(np.abs(Q) @ np.abs(R), 2)
    # and the 2-norm representativity stays near u for these cases
    assert np.linalg.norm(D, 2) / np.linalg.norm(Z, 2) < 1e3 * U


def test_upper_triangle_of_A_ignored():
    A, Z = inputs.paper_case(4, 40, 5, 1e4, seed=30)
    P = A.copy()
    P[np.triu_indices(40, 1)] = -7.0
    Q1, R1 = oracle.oblique_qr(A, Z)
    Q2, R2 = oracle.oblique_qr(P, Z)
    assert np.array_equal(Q1, Q2) and np.array_equal(R1, R2)


def test_not_spd_reports_column():
    A = np.diag([1.0, 1.0, -2.0, 1.0])
    with pytest.raises(oracle.OracleBreakdown) as e:
        oracle.oblique_qr(A, np.eye(4)[:, :2])
    assert e.value.column == 3


# ------------------------------------------------------------------ checks --
def test_orth_defect_and_residual_exact():
    A = np.diag([1.0, 4.0, 9.0])
    Q = np.array([[2.0, 0.0], [0.0, 1.0], [0.0, 0.0]])
    # Q^T A Q = diag(4, 4) -> E = diag(3, 3)
    assert np.array_equal(oracle.orth_defect(A, Q), np.diag([3.0, 3.0]))
    Z = np.array([[1.0, 2.0], [3.0, 4.0], [5.0, 6.0]])
    R = np.array([[1.0, 1.0], [0.0, 1.0]])
    Qz = np.array([[1.0, 1.0], [3.0, 1.0], [5.0, 1.0]])
    assert np.array_equal(oracle.repres_residual(Z, Qz, R), np.zeros((3, 2)))


def test_cholqr_restatement_agrees_when_well_conditioned():
    A, Z = inputs.paper_case(4, 100, 8, 1e3, 1e1, seed=31)
    Q0, R0 = oracle.oblique_qr(A, Z)
    Q1, R1 = oracle.cholqr(A, Z)
    assert rel(R1, R0) < 1e-12 and rel(Q1, Q0) < 1e-11


def test_cpu_method_cholqr2_reaches_the_oracle():
    """The CPU A-CholQR2 restatement (the benchmark's timed baseline of the method) reaches the oracle's
    unique (Q, R) on config 0; ragged row blocks (m not a multiple of 64)
    and column counts not a multiple of the 8-column step are covered."""
    A, Z = inputs.config0(seed=0)
    Qr, Rr = oracle.oblique_qr(A, Z)
    Q, R = oracle.cpu_cholqr2(A, Z)
    assert np.linalg.norm(R - Rr) / np.linalg.norm(Rr) <= 1e-12
    assert oracle.orth_error(A, Q) <= 1e-12
    # ragged sizes: m = 203 (3 row blocks, the last 11 rows; 203 = 25*8 + 3 columns of A)
    A, Z = inputs.paper_case(4, 203, 9, 1e3, 1e2, seed=8)
    Qr, Rr = oracle.oblique_qr(A, Z)
    Q, R = oracle.cpu_cholqr2(A, Z)
    assert np.linalg.norm(R - Rr) / np.linalg.norm(Rr) <= 1e-12
    assert oracle.orth_error(A, Q) <= 1e-12


def test_glls_oracle_pins():
    """The oracle's GLLS (x = R^{-1} Q^T A b, Sec. 1) against what fixes it: a consistent system returns
    its planted solution, A = I reduces to LAPACK's least squares, and the residual is A-orthogonal to
    range(Z) (the normal equations Z^T A (b - Z x) = 0)."""
    rng = np.random.default_rng(12)
    A, Z = inputs.paper_case(4, 300, 12, 1e3, 1e2, seed=12)
    x0 = rng.standard_normal((12, 2))
    X = oracle.glls(A, Z, Z @ x0)
    assert np.abs(X - x0).max() <= 1e-10 * np.abs(x0).max()
    B = rng.standard_normal((300, 3))
    X = oracle.glls(np.eye(300), Z, B)
    Xl = np.linalg.lstsq(Z, B, rcond=None)[0]
    assert np.abs(X - Xl).max() <= 1e-10 * np.abs(Xl).max()
    X = oracle.glls(A, Z, B)
    g = Z.T @ A @ (B - Z @ X)
    assert np.abs(g).max() <= 1e-10 * (np.abs(Z).T @ np.abs(A) @ np.abs(B)).max()


def test_tridiag_oracle_pins():
    """The tridiagonal oracle (CHOL-EQR with T's bidiagonal Cholesky factor) against the dense oracle on
    the same T, against LAPACK's QR for T = I, and against the closed form of an eigenvector basis:
    Z = V_k diag(lambda_k^(-1/2)) with T v_k = lambda_k v_k gives Z^T T Z = I, so R = I and Q = Z."""
    m, n = 300, 11
    d, e = inputs.tridiag_spd(m, 1e4)
    T = oracle.tridiag_dense(d, e)
    lam = np.linalg.eigvalsh(T)
    assert abs(lam.max() / lam.min() / 1e4 - 1) < 1e-9
    _, Z = inputs.paper_case(4, m, n, 1e2, 1e3, seed=14)
    Qd, Rd = oracle.oblique_qr(T, Z)
    Qt, Rt = oracle.oblique_qr_tridiag(d, e, Z)
    assert np.linalg.norm(Rt - Rd) / np.linalg.norm(Rd) <= 1e-13
    assert np.linalg.norm(Qt - Qd) / np.linalg.norm(Qd) <= 1e-12
    assert abs(oracle.orth_error_tridiag(d, e, Qt) - oracle.orth_error(T, Qt)) <= 1e-15
    Qi, Ri = oracle.oblique_qr_tridiag(np.ones(m), np.zeros(m - 1), Z)
    Ql, Rl = np.linalg.qr(Z)
    D = np.sign(np.diag(Rl))
    assert np.abs(Ri - (Rl.T * D).T).max() <= 1e-13 * np.abs(Rl).max()
    assert np.abs(Qi - Ql * D).max() <= 10 * 1e3 * 2.0 ** -53 * 300    # Q is kappa(Z) u sensitive
    ks = [1, 2, 5, 150, 299, 300]
    V = inputs.laplacian_eigvec(m, ks)
    lamk = (d[0] - 2.0) + 2.0 - 2.0 * np.cos(np.asarray(ks) * np.pi / (m + 1))
    Z5 = V / np.sqrt(lamk)
    Q5, R5 = oracle.oblique_qr_tridiag(d, e, Z5)
    assert np.abs(R5 - np.eye(len(ks))).max() <= 1e-10
    assert np.abs(Q5 - Z5).max() <= 1e-10 * np.abs(Z5).max()
    with pytest.raises(oracle.OracleBreakdown) as err:
        oracle.oblique_qr_tridiag(np.array([1.0, 1.0, 1.0]), np.array([0.0, 2.0]), Z[:3, :2])
    assert err.value.column == 3


def test_reuse_w_restatement_pins():
    """The CPU restatement of A-CholQR2 with W reused (not in the paper): on a well-conditioned instance it
    reaches the oracle's unique (Q, R); on case 5 (Z^T A Z = I exactly) it returns R = I, Q = Z; and its
    orthogonality lies between CholQR2's and one-pass CholQR's on an ill-conditioned instance (the second
    pass corrects the Gram's kappa^2 loss but keeps A Z's rounding)."""
    A, Z = inputs.paper_case(4, 400, 10, 1e2, 1e1, seed=3)
    Qr, Rr = oracle.oblique_qr(A, Z)
    Q, R = oracle.cholqr2_reuse_w(A, Z)
    assert np.linalg.norm(R - Rr) / np.linalg.norm(Rr) <= 1e-13
    A5, Z5 = inputs.paper_case(5, 80, 10, 1e6, None, seed=45)
    Q5, R5 = oracle.cholqr2_reuse_w(A5, Z5)
    assert np.abs(R5 - np.eye(10)).max() <= 1e-9
    A, Z = inputs.config0(seed=0)
    Q, R = oracle.cholqr2_reuse_w(A, Z)
    Q1, _ = oracle.cholqr(A, Z)
    Q2, _ = oracle.cpu_cholqr2(A, Z)
    o_reuse, o_one, o_two = oracle.orth_error(A, Q), oracle.orth_error(A, Q1), oracle.orth_error(A, Q2)
    assert o_two <= 10 * o_reuse and o_reuse <= o_one, (o_two, o_reuse, o_one)
