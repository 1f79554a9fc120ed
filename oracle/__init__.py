"""CPU FP64 oracle for QR factorization in an oblique inner product.

TEST INFRASTRUCTURE ONLY: the slow, plain reference that the CUDA path is
checked against (arXiv:1401.5171).  Only the tests, the smoke check and the
benchmark's CPU-baseline arm may import this package; the CUDA library never
does.  The arithmetic lives in ``oqr_oracle.c`` (plain C, FP64, no blocking);
this module only builds it with gcc and marshals numpy arrays.

Every matrix argument is a 2-D float64 numpy array; it is passed column-major
(Fortran order, leading dimension = number of rows), copied if needed.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oqr_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "cpu_method.c")]   # the oracle, and the CPU restatement of the method
_LIB = os.path.join(_HERE, "liboqr_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, IEEE semantics, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or any(os.path.getmtime(_LIB) < os.path.getmtime(s) for s in _SRCS):
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-fno-fast-math", "-std=c99", *_SRCS, "-o", _LIB + ".tmp", "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            path = os.environ.get("OQR_ORACLE_LIB")   # a planted-mistake build (mutation test)
            if not path:
                path = build()
            lib = ctypes.CDLL(path)
            dp = ctypes.POINTER(ctypes.c_double)
            i, l = ctypes.c_int, ctypes.c_long
            lib.orc_chol_upper.argtypes = [i, dp, l, dp, l]
            lib.orc_chol_upper.restype = i
            lib.orc_symm_times.argtypes = [i, i, dp, l, dp, l, dp, l]
            lib.orc_gram.argtypes = [i, i, dp, l, dp, l, dp, l]
            lib.orc_trsm_right_upper.argtypes = [i, i, dp, l, dp, l, dp, l]
            lib.orc_upper_times_upper.argtypes = [i, dp, l, dp, l, dp, l]
            lib.orc_cholqr.argtypes = [i, i, dp, l, dp, l, dp, l, dp, l]
            lib.orc_cholqr.restype = i
            lib.orc_householder_qr.argtypes = [i, i, dp, l, dp, l, dp, l]
            lib.orc_oblique_qr.argtypes = [i, i, dp, l, dp, l, dp, l, dp, l]
            lib.orc_oblique_qr.restype = i
            lib.orc_orth_defect.argtypes = [i, i, dp, l, dp, l, dp, l]
            lib.orc_repres_residual.argtypes = [i, i, dp, l, dp, l, dp, l, dp, l]
            lib.orc_oblique_qr_tridiag.argtypes = [i, i, dp, dp, dp, l, dp, l, dp, l]
            lib.orc_oblique_qr_tridiag.restype = i
            lib.orc_orth_defect_tridiag.argtypes = [i, i, dp, dp, dp, l, dp, l]
            lib.orc_cpu_cholqr2.argtypes = [i, i, dp, l, dp, l, dp, l, dp, l]
            lib.orc_cpu_cholqr2.restype = i
            lib.orc_cpu_threads.argtypes = []
            lib.orc_cpu_threads.restype = i
            _lib = lib
    return _lib


def _f(x):
    x = np.asarray(x, dtype=np.float64)
    if x.ndim == 1:
        x = x.reshape(-1, 1)
    return np.asfortranarray(x)


def _p(x):
    return x.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ld(x):
    return max(1, x.shape[0])


class OracleBreakdown(RuntimeError):
    """Cholesky breakdown: the 1-based column is in ``.column``."""

    def __init__(self, what, column):
        super().__init__(f"{what}: Cholesky breakdown at column {column}")
        self.column = column


def chol_upper(A):
    """C upper with A = C^T C (lower triangle of A read)."""
    A = _f(A)
    n = A.shape[0]
    C = np.zeros((n, n), order="F")
    info = _load().orc_chol_upper(n, _p(A), _ld(A), _p(C), _ld(C))
    if info:
        raise OracleBreakdown("chol_upper", info)
    return C


def symm_times(A, Z):
    A, Z = _f(A), _f(Z)
    m, n = Z.shape
    B = np.zeros((m, n), order="F")
    _load().orc_symm_times(m, n, _p(A), _ld(A), _p(Z), _ld(Z), _p(B), _ld(B))
    return B


def gram(A, Z):
    """G = Z^T A Z (Algorithm 1, lines 1-2)."""
    A, Z = _f(A), _f(Z)
    m, n = Z.shape
    G = np.zeros((n, n), order="F")
    _load().orc_gram(m, n, _p(A), _ld(A), _p(Z), _ld(Z), _p(G), _ld(G))
    return G


def trsm_right_upper(Z, R):
    """Q = Z R^{-1}, row by row (Algorithm 1, line 4)."""
    Z, R = _f(Z), _f(R)
    m, n = Z.shape
    Q = np.zeros((m, n), order="F")
    _load().orc_trsm_right_upper(m, n, _p(Z), _ld(Z), _p(R), _ld(R), _p(Q), _ld(Q))
    return Q


def upper_times_upper(U, S):
    U, S = _f(U), _f(S)
    n = U.shape[0]
    R = np.zeros((n, n), order="F")
    _load().orc_upper_times_upper(n, _p(U), _ld(U), _p(S), _ld(S), _p(R), _ld(R))
    return R


def cholqr(A, Z):
    """CHOLQR (Algorithm 1) restated on the CPU; returns (Q, R)."""
    A, Z = _f(A), _f(Z)
    m, n = Z.shape
    Q = np.zeros((m, n), order="F")
    R = np.zeros((n, n), order="F")
    info = _load().orc_cholqr(m, n, _p(A), _ld(A), _p(Z), _ld(Z), _p(Q), _ld(Q), _p(R), _ld(R))
    if info:
        raise OracleBreakdown("cholqr", info)
    return Q, R


def householder_qr(W):
    """Euclidean Householder QR, thin Y and R_h (signs as produced)."""
    W = _f(W).copy(order="F")
    m, n = W.shape
    Y = np.zeros((m, n), order="F")
    Rh = np.zeros((n, n), order="F")
    _load().orc_householder_qr(m, n, _p(W), _ld(W), _p(Y), _ld(Y), _p(Rh), _ld(Rh))
    return Y, Rh


def oblique_qr(A, Z):
    """The oracle: (Q, R) of Z = QR with Q^T A Q = I by CHOL-EQR (Algorithm 3)."""
    A, Z = _f(A), _f(Z)
    m, n = Z.shape
    Q = np.zeros((m, n), order="F")
    R = np.zeros((n, n), order="F")
    info = _load().orc_oblique_qr(m, n, _p(A), _ld(A), _p(Z), _ld(Z), _p(Q), _ld(Q), _p(R), _ld(R))
    if info:
        raise OracleBreakdown("oblique_qr", info)
    return Q, R


def orth_defect(A, Q):
    """E = Q^T A Q - I, summed in long double."""
    A, Q = _f(A), _f(Q)
    m, n = Q.shape
    E = np.zeros((n, n), order="F")
    _load().orc_orth_defect(m, n, _p(A), _ld(A), _p(Q), _ld(Q), _p(E), _ld(E))
    return E


def repres_residual(Z, Q, R):
    """D = Z - Q R, summed in long double."""
    Z, Q, R = _f(Z), _f(Q), _f(R)
    m, n = Z.shape
    D = np.zeros((m, n), order="F")
    _load().orc_repres_residual(m, n, _p(Z), _ld(Z), _p(Q), _ld(Q), _p(R), _ld(R), _p(D), _ld(D))
    return D


def orth_error(A, Q):
    """||Q^T A Q - I||_2 (Sec. 7's orthogonality measure)."""
    E = orth_defect(A, Q)
    return float(np.max(np.abs(np.linalg.eigvalsh(0.5 * (E + E.T))))) if E.size else 0.0


def repres_error(Z, Q, R):
    """||Z - Q R||_2 / ||Z||_2 (Sec. 7's representativity measure)."""
    D = repres_residual(Z, Q, R)
    return float(np.linalg.norm(D, 2) / np.linalg.norm(np.asarray(Z), 2))


def cpu_cholqr2(A, Z):
    """A-CholQR2 (Algorithm 1 twice, R = R_2 R_1) restated on the CPU with row-block loops over all host
    cores: the benchmark's timed CPU baseline of the method itself (not the oracle).  A is read in full."""
    A, Z = _f(A), _f(Z)
    m, n = Z.shape
    Q = np.zeros((m, n), order="F")
    R = np.zeros((n, n), order="F")
    info = _load().orc_cpu_cholqr2(m, n, _p(A), _ld(A), _p(Z), _ld(Z), _p(Q), _ld(Q), _p(R), _ld(R))
    if info:
        raise OracleBreakdown("cpu_cholqr2", info)
    return Q, R


def cpu_threads():
    """OpenMP threads the CPU code uses (all host cores unless OMP_NUM_THREADS says otherwise)."""
    return int(_load().orc_cpu_threads())


def glls(A, Z, B):
    """The generalized least-squares solution of Sec. 1, x = R^{-1} Q^T A b for each column b of B, from the
    oracle's own (Q, R) (CHOL-EQR), its product with A and a back substitution with R."""
    Q, R = oblique_qr(A, Z)
    C = symm_times(A, _f(B))
    Y = np.asarray(Q).T @ C
    n = R.shape[0]
    X = np.zeros_like(Y)
    for i in range(n - 1, -1, -1):               # R x = y, last row first
        X[i] = (Y[i] - R[i, i + 1:] @ X[i + 1:]) / R[i, i]
    return X


def _vec1(x):
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64).ravel())
    return x if x.size else np.zeros(1)


def oblique_qr_tridiag(d, e, Z):
    """The oracle for tridiagonal A = T (diagonal d, off-diagonal e): CHOL-EQR (Algorithm 3) with T's
    bidiagonal Cholesky factor."""
    Z = _f(Z)
    m, n = Z.shape
    d, e = _vec1(d), _vec1(e)
    Q = np.zeros((m, n), order="F")
    R = np.zeros((n, n), order="F")
    info = _load().orc_oblique_qr_tridiag(m, n, _p(d), _p(e), _p(Z), _ld(Z), _p(Q), _ld(Q), _p(R), _ld(R))
    if info:
        raise OracleBreakdown("oblique_qr_tridiag", info)
    return Q, R


def orth_error_tridiag(d, e, Q):
    """||Q^T T Q - I||_2 for tridiagonal T, the defect summed in long double."""
    Q = _f(Q)
    m, n = Q.shape
    d, e = _vec1(d), _vec1(e)
    E = np.zeros((n, n), order="F")
    _load().orc_orth_defect_tridiag(m, n, _p(d), _p(e), _p(Q), _ld(Q), _p(E), _ld(E))
    return float(np.max(np.abs(np.linalg.eigvalsh(0.5 * (E + E.T))))) if E.size else 0.0


def tridiag_dense(d, e):
    """The dense T of a tridiagonal (d, e), for comparisons with the dense oracle at small m."""
    m = len(d)
    T = np.diag(np.asarray(d, dtype=np.float64))
    if m > 1:
        T += np.diag(np.asarray(e, dtype=np.float64)[:m - 1], -1) + np.diag(np.asarray(e, dtype=np.float64)[:m - 1], 1)
    return T


def cholqr2_reuse_w(A, Z):
    """A-CholQR2 with the first pass's W = A Z kept (not in the paper), restated on the CPU from the oracle's
    pinned steps: W = A Z; R_1 = chol(Z^T W); Q_1 = Z / R_1; W_1 = W / R_1; R_2 = chol(Q_1^T W_1);
    Q = Q_1 / R_2; R = R_2 R_1.  The reference for the GPU variant's own rounding, not the oracle of the
    result (that is oblique_qr)."""
    A, Z = _f(A), _f(Z)
    W = symm_times(A, Z)
    R1 = chol_upper(Z.T @ W)
    Q1 = trsm_right_upper(Z, R1)
    W1 = trsm_right_upper(W, R1)
    R2 = chol_upper(Q1.T @ W1)
    return trsm_right_upper(Q1, R2), upper_times_upper(R2, R1)
