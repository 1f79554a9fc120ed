"""Pins of the selector network's CPU oracle (oracle/mlp.py) to mathematics:
central finite differences of the loss, and the closed form of the
zero-weight network (logits = b3, so d loss / d b3 = mean(softmax(b3) - e_y))."""
import numpy as np

from oracle import mlp


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(0)
    p = rng.standard_normal(mlp.COUNT) * 0.3
    X = rng.standard_normal((9, 16))
    y = rng.integers(0, 4, size=9)
    _, g = mlp.loss_and_grad(p, X, y)
    idx = rng.choice(mlp.COUNT, size=200, replace=False)
    for i in idx:
        h = 1e-6 * max(1.0, abs(p[i]))
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (mlp.loss_only(pp, X, y) - mlp.loss_only(pm, X, y)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 + 1e-5 * abs(fd)


def test_zero_weight_closed_form():
    p = np.zeros(mlp.COUNT)
    b3 = np.array([0.5, -1.0, 2.0, 0.0])
    p[-4:] = b3
    X = np.random.default_rng(1).standard_normal((5, 16))
    y = np.array([0, 2, 2, 3, 1])
    loss, g = mlp.loss_and_grad(p, X, y)
    sm = np.exp(b3 - b3.max())
    sm /= sm.sum()
    assert np.allclose(g[-4:], sm - np.bincount(y, minlength=4) / 5.0)
    assert np.isclose(loss, np.mean(-np.log(sm[y])))
    assert np.all(g[:-4] == 0)                   # no signal through zero weights
