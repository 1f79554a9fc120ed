"""Definitions of the low-precision splits, written out in float64 for the tests.

bf16_rne: round to the nearest value with 8 significant bits, ties to even
(BF16).  e4m3_quantize: the E4M3 value (4 significant bits, ties to even,
subnormal steps of 2^-9 below 2^-6) of x 2^(8-e), scaled back.  Both are exact
in float64; tests/test_split_definitions.py pins them to torch's conversions.
emu_digits: the balanced base-256 digits of the FP64-accurate slicing, and
tc2_rows / tc2_cols: the value that the two leading slices keep of every
element, per 256-long chunk (integer arithmetic, exact).
"""
import numpy as np


def bf16_rne(x):
    """Round to the nearest BF16 value (8 significant bits), ties to even; exact in float64."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)                       # x = m 2^e, |m| in [0.5, 1)
    q = np.rint(m * 256.0)                   # 8 significant bits, numpy rint = ties to even
    return np.ldexp(q / 256.0, e)



def e4m3_quantize(x, e):
    """Value of the E4M3 code of x 2^(8-e), scaled back by 2^(e-8): 4 significant
    bits, round to nearest even, subnormal steps of 2^-9 below 2^-6 (exact in float64)."""
    v = np.ldexp(np.asarray(x, dtype=np.float64), 8 - e)
    m, ex = np.frexp(v)                                   # v = m 2^ex, |m| in [0.5, 1)
    normal = np.abs(v) >= 2.0 ** -6
    qn = np.ldexp(np.rint(m * 16.0) / 16.0, ex)           # 4 significant bits
    qs = np.rint(v * 512.0) / 512.0                       # subnormal grid 2^-9
    return np.ldexp(np.where(normal, qn, qs), e - 8)


def chunk_exponent(amax):
    """e with amax = f 2^e, f in [0.5, 1) (frexp); 0 for amax = 0."""
    return np.where(amax > 0, np.frexp(amax)[1], 0)


def emu_digits(x, e, S=7):
    """Digits d_0..d_{S-1} with RNE(x 2^(55-e)) = sum_s d_s 2^(8(6-s)) for |x| < 2^e:
    d_1..d_6 in [-128, 127] (balanced base 256), d_0 the rest.  Returns an int64
    array of shape (S,) + x.shape."""
    x = np.asarray(x, dtype=np.float64)
    Y = np.rint(np.ldexp(x, 55 - np.asarray(e))).astype(np.int64)   # exact scaling, ties to even
    d = np.zeros((7,) + x.shape, dtype=np.int64)
    for s in range(6, 0, -1):
        r = np.bitwise_and(Y, 255)
        r = np.where(r > 127, r - 256, r)
        d[s] = r
        Y = (Y - r) >> 8
    d[0] = Y
    return d[:S]


def _tc2_value(x, e):
    d = emu_digits(x, e, 2)
    return np.ldexp(d[0] + np.ldexp(d[1].astype(np.float64), -8), np.asarray(e) - 7)


def tc2_rows(M, chunk=256):
    """Value kept by the two leading slices of every element of M, with one
    exponent per (row, 256-long chunk of columns) as in the FP64_TC/TC2 split."""
    M = np.asarray(M, dtype=np.float64)
    out = np.zeros_like(M)
    for k0 in range(0, M.shape[1], chunk):
        blk = M[:, k0:k0 + chunk]
        e = chunk_exponent(np.abs(blk).max(axis=1))[:, None]
        out[:, k0:k0 + chunk] = _tc2_value(blk, e)
    return out


def tc2_cols(X, chunk=256):
    """tc2_rows with one exponent per (column, chunk of rows)."""
    return tc2_rows(np.asarray(X).T, chunk).T

