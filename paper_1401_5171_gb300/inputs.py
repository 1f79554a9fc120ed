"""Seeded synthetic inputs for oblique QR (the test-matrix recipe of Sec. 7).

This module only draws random numbers and builds test matrices; it holds none
of the factorization's arithmetic.  Both the CPU oracle's tests and the CUDA
path's tests and benchmark take their inputs from here.

Recipe (Sec. 7 of Lowery & Langou):
  * A = V D V^T with D = diag(d), d_i = 10^(alpha (i-1)), alpha =
    log10(kappa_A) / (m - 1): log-evenly spaced eigenvalues from 1 to kappa_A.
  * Z = U Sigma W^T with log-evenly spaced singular values from 1 to kappa_Z,
    W a random orthonormal n x n matrix, and U either random orthonormal
    (case 4) or chosen columns of V (cases 1, 2, 3, 5).
  * "Random orthonormal" is MATLAB's orth(randn(m)); here the QR factor of a
    Gaussian matrix with the signs fixed so that R has a positive diagonal,
    which is Haar distributed.

Large A (m in the tens of thousands, or thousands of batched instances)
cannot use a Haar V: its QR costs O(m^3).  ``dense_spd`` builds instead
  A = H_2 H_1 S (sum_i d_pi(i) c_i c_i^T) S H_1 H_2
with c_i the orthonormal DCT-II basis vectors, pi a random permutation, S a
random +-1 diagonal and H_j = I - 2 u_j u_j^T two random Householder
reflectors.  A is dense, its eigenvectors are delocalised, its spectrum is
exactly the recipe's d (up to rounding), and the eigenvectors are known in
closed form, so cases 1-5 remain constructible.  With a random U the pair
(A, Z) has the same distribution up to an orthogonal change of basis as with
a Haar V.  The O(m^2) work runs in torch on the requested device; every
random draw comes from numpy's PCG64 so that a seed means the same inputs
everywhere.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "eigenvalues", "singular_values", "haar", "paper_case", "config0",
    "DenseSPD", "dense_spd", "tall_z", "batch_shapes", "tridiag_spd", "laplacian_eigvec",
]


def eigenvalues(m: int, kappa: float) -> np.ndarray:
    """d_i = 10^(alpha (i-1)), alpha = log10(kappa)/(m-1), i = 1..m (ascending)."""
    if m == 1:
        return np.ones(1)
    alpha = math.log10(kappa) / (m - 1)
    return 10.0 ** (alpha * np.arange(m, dtype=np.float64))


def singular_values(n: int, kappa: float) -> np.ndarray:
    """Log-evenly spaced singular values from 1 up to kappa (ascending)."""
    return eigenvalues(n, kappa)


def haar(rng: np.random.Generator, m: int, n: int | None = None) -> np.ndarray:
    """m x n matrix with orthonormal columns: QR of a Gaussian, diag(R) > 0."""
    n = m if n is None else n
    g = rng.standard_normal((m, n))
    q, r = np.linalg.qr(g)
    s = np.sign(np.diag(r))
    s[s == 0] = 1.0
    return np.asfortranarray(q * s)


def _case_columns(case: int, m: int, n: int) -> np.ndarray:
    """Indices (into ascending eigenvalues) of V's columns that span Z in cases 1, 2, 3, 5."""
    if case == 1:
        return np.arange(n)                      # n smallest eigenvalues
    if case == 2:
        return np.arange(m - n, m)               # n largest eigenvalues
    if case in (3, 5):
        lo = (n + 1) // 2                        # ceil(n/2) smallest and floor(n/2) largest
        return np.concatenate([np.arange(lo), np.arange(m - (n - lo), m)])
    raise ValueError(case)


def paper_case(case: int, m: int, n: int, kappa_a: float, kappa_z: float | None = None,
               seed: int = 0):
    """Test case 1-5 of Sec. 7 with a Haar V.  Returns (A, Z) as float64 arrays.

    kappa_z defaults to sqrt(kappa_a), as in Sec. 7's sweep.  In case 5 Z is
    A-orthonormal (singular values d^{-1/2} on the chosen eigenvectors), so the
    exact factors are R = I and Q = Z.
    """
    rng = np.random.default_rng(seed)
    kappa_z = math.sqrt(kappa_a) if kappa_z is None else kappa_z
    V = haar(rng, m)
    d = eigenvalues(m, kappa_a)
    A = np.asfortranarray((V * d) @ V.T)
    W = haar(rng, n)
    if case == 4:
        U = haar(rng, m, n)
        sig = singular_values(n, kappa_z)
    else:
        idx = _case_columns(case, m, n)
        U = V[:, idx]
        sig = d[idx] ** -0.5 if case == 5 else singular_values(n, kappa_z)
    Z = np.asfortranarray((U * sig) @ W.T)
    return A, Z


def config0(seed: int = 0, m: int = 2000, n: int = 20):
    """Plain FP64 workload: m=2000, n=20, kappa(A)=1e4 (logspace(0,4,m)), random U, kappa(Z)=1e3."""
    return paper_case(4, m, n, 1e4, 1e3, seed=seed)


@dataclass
class DenseSPD:
    """Random orthogonal eigenbasis V = H_2 H_1 S C_pi and spectrum d of a dense SPD A."""
    m: int
    d: np.ndarray           # ascending eigenvalues
    freq: np.ndarray        # freq[i]: DCT frequency carrying eigenvalue d[i]
    sign: np.ndarray        # S
    u: np.ndarray           # (2, m) unit Householder vectors


def _dense_spd_params(m: int, kappa: float, rng: np.random.Generator) -> DenseSPD:
    d = eigenvalues(m, kappa)
    freq = rng.permutation(m)
    sign = rng.choice(np.array([-1.0, 1.0]), size=m)
    u = rng.standard_normal((2, m))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    return DenseSPD(m, d, freq, sign, u)


def eigvecs(p: DenseSPD, idx, torch_mod=None, device="cpu"):
    """Columns V[:, idx] (eigenvectors of eigenvalues d[idx]) of a dense_spd matrix, as numpy."""
    m = p.m
    k = np.arange(m, dtype=np.float64)
    cols = []
    for i in np.atleast_1d(idx):
        f = p.freq[i]
        s = math.sqrt(1.0 / m) if f == 0 else math.sqrt(2.0 / m)
        v = s * np.cos(math.pi * f * (2.0 * k + 1.0) / (2.0 * m))
        v = p.sign * v
        for j in (0, 1):                       # V = H_2 H_1 S C: apply H_1 first
            uj = p.u[j]
            v = v - 2.0 * uj * (uj @ v)
        cols.append(v)
    return np.stack(cols, axis=1)


def dense_spd(m: int, kappa: float, seed: int, device="cpu", dtype=None, out=None):
    """Dense SPD A (m x m) with eigenvalues eigenvalues(m, kappa); see module docstring.

    Returns (A, params) with A a torch float64 tensor on ``device`` holding the
    full symmetric matrix (row-major storage of a symmetric matrix is also its
    column-major storage).  ``out`` may supply preallocated storage.
    """
    import torch

    rng = np.random.default_rng(seed)
    p = _dense_spd_params(m, kappa, rng)
    dt = torch.float64
    # f(t) = 1/2 sum_i w_i s_i^2 cos(pi i t / m), t = 0..2m-1, w_i the eigenvalue at frequency i
    w = np.empty(m)
    w[p.freq] = p.d
    s2 = np.full(m, 2.0 / m)
    s2[0] = 1.0 / m
    x = np.zeros(2 * m)
    x[:m] = 0.5 * w * s2
    f = torch.fft.fft(torch.tensor(x, dtype=dt)).real.to(device)
    sign = torch.tensor(p.sign, dtype=dt, device=device)
    A = out if out is not None else torch.empty((m, m), dtype=dt, device=device)
    kk = torch.arange(m, device=device)
    rows = max(1, min(m, (1 << 26) // max(m, 1)))
    for r0 in range(0, m, rows):
        r1 = min(m, r0 + rows)
        k = kk[r0:r1, None]
        blk = f[(k - kk[None, :]).abs()] + f[k + kk[None, :] + 1]
        A[r0:r1] = blk * sign[r0:r1, None] * sign[None, :]
    for j in (0, 1):
        u = torch.tensor(p.u[j], dtype=dt, device=device)
        wv = A @ u
        gam = torch.dot(u, wv)
        for r0 in range(0, m, rows):
            r1 = min(m, r0 + rows)
            A[r0:r1] += (-2.0 * u[r0:r1, None]) * wv[None, :] + (-2.0 * wv[r0:r1, None]) * u[None, :] \
                + (4.0 * gam) * u[r0:r1, None] * u[None, :]
    return A, p


def tall_z(m: int, n: int, kappa_z: float, seed: int, device="cpu", U=None):
    """Z = U diag(sigma) W^T (torch float64 on ``device``), U Haar unless given (m x n numpy)."""
    import torch

    rng = np.random.default_rng(seed)
    if U is None:
        U = haar(rng, m, n)          # on the host: one m x n QR
    U = torch.as_tensor(np.asarray(U), dtype=torch.float64, device=device)
    W = torch.tensor(haar(rng, n), dtype=torch.float64, device=device)
    sig = torch.tensor(singular_values(n, kappa_z), dtype=torch.float64, device=device)
    return (U * sig) @ W.T


def batch_shapes(count: int, seed: int, m_range=(64, 4096), n_range=(4, 64),
                 log_kappa_a=(0.0, 6.0), log_kappa_z=(0.0, 6.0)):
    """Instance table of a batch: m, n uniform integers (inclusive, n <= m), kappas log-uniform."""
    rng = np.random.default_rng(seed)
    m = rng.integers(m_range[0], m_range[1] + 1, size=count)
    n = rng.integers(n_range[0], n_range[1] + 1, size=count)
    n = np.minimum(n, m)
    ka = 10.0 ** rng.uniform(*log_kappa_a, size=count)
    kz = 10.0 ** rng.uniform(*log_kappa_z, size=count)
    seeds = rng.integers(0, 2**31 - 1, size=count)
    return m.astype(np.int64), n.astype(np.int64), ka, kz, seeds


def batch_instances(count: int, seed: int, device="cpu", m_range=(64, 4096), n_range=(4, 64),
                    log_kappa_a=(0.0, 6.0), log_kappa_z=(0.0, 6.0)):
    """A batch in the recipe of the batched workload: per instance m, n uniform
    integers, kappa(A) and kappa(Z) log-uniform, A from dense_spd and Z from
    tall_z with the instance's own seed.  Returns (As, Zs, table) with A_b, Z_b
    column-major torch float64 tensors on ``device``."""
    import torch
    m, n, ka, kz, seeds = batch_shapes(count, seed, m_range, n_range, log_kappa_a, log_kappa_z)
    As, Zs = [], []
    for b in range(count):
        A, _ = dense_spd(int(m[b]), float(ka[b]), seed=int(seeds[b]), device=device)
        As.append(A.t())                       # column-major view; the library reads its lower triangle
        Z = tall_z(int(m[b]), int(n[b]), float(kz[b]), seed=int(seeds[b]) + 1, device=device)
        Zs.append(Z.t().contiguous().t())
    return As, Zs, {"m": m, "n": n, "kappa_A": ka, "kappa_Z": kz, "seed": seeds}


def tridiag_spd(m: int, kappa: float):
    """Tridiagonal SPD T for Sec. 8's tridiagonal workload (the paper does not give its entries): the
    1-D Laplacian tridiag(-1, 2, -1) shifted by mu I, with mu chosen so that kappa(T) = kappa exactly.
    Its eigenvalues are mu + 2 - 2 cos(k pi / (m + 1)), k = 1..m.  Returns (d, e) as float64 arrays
    (e has m - 1 entries)."""
    if m == 1:
        return np.ones(1), np.zeros(0)
    a = 2.0 - 2.0 * math.cos(math.pi / (m + 1))        # smallest Laplacian eigenvalue
    b = 2.0 + 2.0 * math.cos(math.pi / (m + 1))        # largest
    mu = (b - kappa * a) / (kappa - 1.0) if kappa > 1.0 else 1.0
    return np.full(m, 2.0 + mu), np.full(m - 1, -1.0)


def laplacian_eigvec(m: int, ks) -> np.ndarray:
    """Orthonormal eigenvectors of tridiag(-1, 2, -1) (any diagonal shift), v_k(i) =
    sqrt(2 / (m + 1)) sin(i k pi / (m + 1)), i, k = 1..m; columns for the given k (1-based)."""
    i = np.arange(1, m + 1, dtype=np.float64)[:, None]
    k = np.asarray(ks, dtype=np.float64)[None, :]
    return np.sqrt(2.0 / (m + 1)) * np.sin(i * k * math.pi / (m + 1))
