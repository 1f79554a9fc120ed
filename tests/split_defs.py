"""Definitions of the low-precision splits, written out in float64 for the tests.

bf16_rne: round to the nearest value with 8 significant bits, ties to even
(BF16).  e4m3_quantize: the E4M3 value (4 significant bits, ties to even,
subnormal steps of 2^-9 below 2^-6) of x 2^(8-e), scaled back.  Both are exact
in float64; tests/test_split_definitions.py pins them to torch's conversions.
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


