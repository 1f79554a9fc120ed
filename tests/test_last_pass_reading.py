"""CPU pins of the reading behind the last tensor-core pass's solve.

The last pass of A-CholQR2 (or of shifted A-CholQR3) factors G = R^T R with
G close to I.  The library then forms Q = Z R^{-1} as one product with the
explicit inverse whenever ||G - I||_F <= 0.5, and keeps row-wise substitution
(Algorithm 1, line 4) otherwise.  These tests pin the two facts that rule
rests on, with the oracle's Cholesky and substitution and numpy's product:
  - ||G - I||_F <= 0.5 puts every eigenvalue of G in [0.5, 1.5], so
    cond(R)^2 = cond(G) <= 3;
  - for such an R the explicit inverse gives the substitution's result to a
    few units of rounding, with every row's backward error |z - q R| within
    the row-wise substitution's bound (Sec. 2's model, reading 2).
"""
import numpy as np
import pytest

import oracle

U = 2.0 ** -53


def near_identity(rng, n, frob):
    E = rng.standard_normal((n, n))
    E = E + E.T
    return np.eye(n) + frob * E / np.linalg.norm(E)


@pytest.mark.parametrize("n", [1, 2, 7, 40, 129])
def test_defect_bound_limits_the_condition(n):
    rng = np.random.default_rng(11 + n)
    cases = [near_identity(rng, n, 0.5)]
    # the extreme placements of the whole defect: one eigenvalue moved by -0.5 or +0.5
    for sgn in (-1.0, 1.0):
        G = np.eye(n)
        G[0, 0] += sgn * 0.5
        cases.append(G)
    for G in cases:
        assert np.linalg.norm(G - np.eye(n)) <= 0.5 * (1 + 1e-12)
        ev = np.linalg.eigvalsh(G)
        assert ev.min() >= 0.5 - 1e-12 and ev.max() <= 1.5 + 1e-12
        R = oracle.chol_upper(G)
        assert np.linalg.cond(R) ** 2 <= 3.0 * (1 + 1e-9)


@pytest.mark.parametrize("m,n", [(1, 1), (300, 20), (2000, 64), (1500, 130)])
def test_explicit_inverse_matches_substitution_near_identity(m, n):
    rng = np.random.default_rng(5 * m + n)
    G = near_identity(rng, n, 0.45)
    R = oracle.chol_upper(G)
    Z = rng.standard_normal((m, n))
    Rinv = oracle.trsm_right_upper(np.eye(n), R)  # R^{-1} by the same row-wise substitution
    Qi = Z @ Rinv
    Qs = oracle.trsm_right_upper(Z, R)
    assert np.linalg.norm(Qi - Qs) <= 1e-14 * np.linalg.norm(Qs)
    bw = np.abs(Z - Qi @ R).max(axis=1) / (np.abs(Qi) @ np.abs(R)).max(axis=1)
    assert bw.max() <= 4 * n * U
