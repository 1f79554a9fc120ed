"""Pins the float64 split definitions used by the GPU tests to torch's own
BF16 and FP8 E4M3 conversions (library routines) on float32-representable inputs."""
import numpy as np
import torch

from split_defs import bf16_rne, e4m3_quantize


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
