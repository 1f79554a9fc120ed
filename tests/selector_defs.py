"""CPU definitions of the batched selector's features, for the GPU tests (test infrastructure).

Written from the feature list in include/oqr.h (OQR_BATCHED_SELECTOR): the features of one instance from
its FP64 Gram G0 = Z^T A Z (the oracle's), the Cholesky factor R1 of G0 (the oracle's) or the breakdown
column, and a sketch W (n x 2n) of standard normal deviates drawn with SplitMix64 (Steele, Lea and Flood,
2014) on counters 2c and 2c + 1, c = j n + i, and the Box-Muller transform.
"""
import numpy as np

SEED = np.uint64(0x0123456789ABCDEF)
GAMMA = np.uint64(0x9E3779B97F4A7C15)


def splitmix64_at(counter):
    """Output number counter (0-based) of SplitMix64 seeded with SEED (uint64 arithmetic, wrapping)."""
    with np.errstate(over="ignore"):
        z = SEED + (np.asarray(counter, dtype=np.uint64) + np.uint64(1)) * GAMMA
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def sketch(n, k):
    """W (n x k): W[i, j] = sqrt(-2 ln u1) cos(2 pi u2), u1 from counter 2c (top 53 bits + 1, times 2^-53),
    u2 from counter 2c + 1 (top 53 bits times 2^-53), c = j n + i."""
    i = np.arange(n, dtype=np.uint64)[:, None]
    j = np.arange(k, dtype=np.uint64)[None, :]
    c = j * np.uint64(n) + i
    u1 = ((splitmix64_at(np.uint64(2) * c) >> np.uint64(11)) + np.uint64(1)).astype(np.float64) * 2.0 ** -53
    u2 = (splitmix64_at(np.uint64(2) * c + np.uint64(1)) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def features(m, n, G0, R1=None, breakdown=0):
    """The 16 features (f13..f15 zero); R1 is the Cholesky factor of G0, or None with its breakdown column."""
    f = np.zeros(16)
    d = np.diag(G0).copy()
    f[0], f[1], f[2] = np.log10(m) / 4, np.log10(n) / 2, n / m
    f[3] = np.log10(d.max() / d.min()) / 6 if d.min() > 0 else 4.0
    C = G0 / np.sqrt(np.outer(d, d))
    f[4] = np.abs(C - np.diag(np.diag(C))).max() if n > 1 else 0.0
    try:
        piv = np.diag(np.linalg.cholesky(C)) ** 2
        f[7], f[8] = -np.log10(piv.min()) / 6, np.log10(piv.max()) / 6
    except np.linalg.LinAlgError:
        f[5] = 1.0                                   # the column is not reproduced here
    f[9] = np.log10(d.sum() / d.max()) / 3
    if R1 is None:
        f[10], f[11] = 1.0, breakdown / n
    else:
        W = sketch(n, 2 * n)
        X = np.linalg.solve(R1, W)
        f[12] = np.log10(np.linalg.norm(R1) * np.linalg.norm(X) / np.linalg.norm(W)) / 8
    return f
