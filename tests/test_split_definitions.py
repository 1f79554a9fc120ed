"""Pins the float64 split definitions used by the GPU tests to torch's own
BF16 and FP8 E4M3 conversions (library routines) on float32-representable inputs."""
import numpy as np
import torch

from split_defs import bf16_rne, e4m3_quantize, chunk_exponent, emu_digits, tc2_cols, tc2_rows


def test_bf16_definition_matches_torch():
    rng = np.random.default_rng(0)
    x = (rng.standard_normal(20000) * 10.0 ** rng.integers(-20, 20, 20000)).astype(np.float32).astype(np.float64)
    t = torch.as_tensor(x.astype(np.float32)).to(torch.bfloat16).double().numpy()
    assert np.array_equal(bf16_rne(x), t)


def test_e4m3_definition_matches_torch():
    rng = np.random.default_rng(1)
    x = (rng.standard_normal(20000) * 30).astype(np.float32).astype(np.float64)
    x = x[np.abs(x) < 448]
    t = torch.as_tensor(x.astype(np.float32)).to(torch.float8_e4m3fn).double().numpy()
    assert np.array_equal(e4m3_quantize(x, 8), t)          # e = 8: scale 2^(8-e) = 1
    # a power-of-two chunk scale commutes with the rounding
    assert np.array_equal(e4m3_quantize(x * 2.0 ** 5, 13), t * 2.0 ** 5)


def test_emu_digits_reconstruct_and_range():
    # the digits are the balanced base-256 expansion of RNE(x 2^(55-e)): they rebuild it exactly,
    # d_1..d_6 stay in [-128, 127], |d_0| <= 128, and the rebuilt value is within 2^(e-56) of x
    rng = np.random.default_rng(5)
    x = rng.standard_normal(4000) * np.exp(rng.uniform(-30, 30, 4000))
    e = np.frexp(np.abs(x))[1] + rng.integers(0, 3, size=x.size)       # |x| < 2^e
    d = emu_digits(x, e)
    Y = np.rint(np.ldexp(x, 55 - e)).astype(np.int64)
    rebuilt = sum(d[s].astype(object) * (256 ** (6 - s)) for s in range(7))
    assert all(int(a) == int(b) for a, b in zip(rebuilt, Y))
    assert np.all((d[1:] >= -128) & (d[1:] <= 127)) and np.all(np.abs(d[0]) <= 128)
    val = sum(np.ldexp(d[s].astype(np.float64), e - 7 - 8 * s) for s in range(7))
    assert np.all(np.abs(val - x) <= np.ldexp(1.0, e - 56))


def test_tc2_keeps_16_bits_of_the_chunk_maximum():
    # two slices leave |d_2 2^-16 + d_3 2^-24 + ...| <= 128 2^-16 / (1 - 2^-8) of x 2^(7-e):
    # |x - x_tc2| <= 2^(e-16) 256/255 per chunk
    rng = np.random.default_rng(6)
    M = rng.standard_normal((40, 600)) * np.exp(rng.uniform(-5, 5, (40, 600)))
    T = tc2_rows(M)
    for k0 in range(0, 600, 256):
        blk = M[:, k0:k0 + 256]
        e = chunk_exponent(np.abs(blk).max(axis=1))[:, None]
        assert np.all(np.abs(T[:, k0:k0 + 256] - blk) <= np.ldexp(256.0 / 255.0, e - 16))
    # integers below 2^8 relative to the chunk maximum's scale are kept exactly
    Z = rng.integers(-100, 101, size=(256, 3)).astype(np.float64)
    assert np.array_equal(tc2_cols(Z), Z)

