"""Pins of the CPU definitions the selector's GPU tests use (tests/selector_defs.py), on the CPU."""
import numpy as np

import selector_defs as sd


def test_splitmix64_published_outputs():
    """SplitMix64 seeded with 0 starts 0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4 (the generator's reference
    implementation); the definition is checked with that seed."""
    keep = sd.SEED
    try:
        sd.SEED = np.uint64(0)
        assert int(sd.splitmix64_at(0)) == 0xE220A8397B1DCDAF
        assert int(sd.splitmix64_at(1)) == 0x6E789E6AA1B965F4
    finally:
        sd.SEED = keep


def test_sketch_is_standard_normal():
    W = sd.sketch(64, 128)
    assert W.shape == (64, 128)
    assert abs(W.mean()) < 0.03 and abs(W.std() - 1.0) < 0.03
    assert np.array_equal(W, sd.sketch(64, 128))          # a function of the counters only


def test_features_on_known_matrices():
    """G0 = diag(1, 10^6): spread log10(1e6)/6 = 1, no coherence, pivots of C all 1; R1 = sqrt(G0) gives
    kappa_sketch ~ 1e3 within the sketch's scatter."""
    G0 = np.diag([1.0, 1e6])
    f = sd.features(100, 2, G0, R1=np.sqrt(G0))
    assert abs(f[3] - 1.0) < 1e-12 and f[4] == 0.0 and abs(f[7]) < 1e-12 and abs(f[8]) < 1e-12
    assert 2.0 / 8 < f[12] < 4.0 / 8
    f = sd.features(100, 2, G0, R1=None, breakdown=2)
    assert f[10] == 1.0 and f[11] == 1.0 and f[12] == 0.0
