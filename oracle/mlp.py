"""CPU FP64 restatement of the selector network (test infrastructure only).

The selector is not in the paper; this module states what the CUDA kernels
compute so that their outputs and gradients can be checked: an MLP
16 -> 64 -> 64 -> 4 with ReLU, logits z = W3 h2 + b3, and the mean softmax
cross-entropy loss over a minibatch.  Parameters use the library's flat
layout W1[64][16], b1[64], W2[64][64], b2[64], W3[4][64], b3[4].  The
gradient is written out by the chain rule; tests pin it to central finite
differences and to the closed form of the zero-weight network.
"""
import numpy as np

F, H, O = 16, 64, 4
SIZES = [("W1", (H, F)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (O, H)), ("b3", (O,))]
COUNT = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    out, o = {}, 0
    for name, shape in SIZES:
        k = int(np.prod(shape))
        out[name] = p[o:o + k].reshape(shape)
        o += k
    return out


def forward(p, X):
    """Returns (logits, cache) for feature rows X (B x 16)."""
    w = unpack(p)
    X = np.asarray(X, dtype=np.float64)
    a1 = X @ w["W1"].T + w["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ w["W2"].T + w["b2"]
    h2 = np.maximum(a2, 0.0)
    z = h2 @ w["W3"].T + w["b3"]
    return z, (X, h1, h2)


def loss_and_grad(p, X, y):
    """Mean softmax cross-entropy and its gradient w.r.t. the flat parameters."""
    w = unpack(p)
    z, (X, h1, h2) = forward(p, X)
    B = z.shape[0]
    zs = z - z.max(axis=1, keepdims=True)
    e = np.exp(zs)
    sm = e / e.sum(axis=1, keepdims=True)
    y = np.asarray(y)
    loss = float(np.mean(-np.log(sm[np.arange(B), y])))
    dz = sm.copy()
    dz[np.arange(B), y] -= 1.0
    dz /= B
    g = {"W3": dz.T @ h2, "b3": dz.sum(axis=0)}
    dh2 = (dz @ w["W3"]) * (h2 > 0)
    g["W2"] = dh2.T @ h1
    g["b2"] = dh2.sum(axis=0)
    dh1 = (dh2 @ w["W2"]) * (h1 > 0)
    g["W1"] = dh1.T @ X
    g["b1"] = dh1.sum(axis=0)
    return loss, np.concatenate([g[name].ravel() for name, _ in SIZES])


def loss_only(p, X, y):
    z, _ = forward(p, X)
    zs = z - z.max(axis=1, keepdims=True)
    lse = np.log(np.exp(zs).sum(axis=1)) + z.max(axis=1)
    return float(np.mean(lse - z[np.arange(z.shape[0]), np.asarray(y)]))
