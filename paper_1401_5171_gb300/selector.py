"""Learned selector over the normal-equation variants: training-set generation, training and marshalling.

The selector itself runs inside the C library (``oqr_batched`` in ``OQR_BATCHED_SELECTOR`` mode): every
instance of a batch first runs one FP64-accurate pass on the tensor cores; 16 features of that pass's
Gram G0 and Cholesky factor R1 go through the MLP 16 -> 64 -> 64 -> 4 (BF16 inference), whose argmax says
how the instance finishes:

  0  one pass         Q = Z R1^{-1}                        (its result is checked)
  1  two passes       one more FP64-accurate pass          (A-CholQR2)
  2  shifted          chol(G0 + s I), then two more passes (shifted A-CholQR3)
  3  FP64 A-CholQR2   (DFMA)                               -- also the end of the fallback chain

A failed check or a breakdown goes to shifted A-CholQR3 on the tensor cores, then to FP64 A-CholQR2.

This module makes the network's training data and trains it, with the library's own kernels: the
features come from ``oqr_batched_features`` (the same first pass), and the label of an instance is the
cheapest option whose measured ||Q^T A Q - I||_2 meets the tolerance, measured by running the three
tensor-core programs on the batch (``oqr_batched_mixed`` with its check).  Those programs produce exactly
the selector's options: the same first pass, then the same later passes.  Training is Adam on the mean
cross-entropy (``oqr_mlp_grad``, ``oqr_mlp_adam``).  Nothing here computes a factorization.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np

CLASSES = 4
ONE, TWO, SHIFTED, FP64 = 0, 1, 2, 3
# the tensor-core program of each option (oqr_batch_program), for labelling
PROGRAMS = {ONE: 0, TWO: 2, SHIFTED: 3}          # OQR_BATCH_CHOLQR_TC, _CHOLQR2_TC, _SCHOLQR3_TC
WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "selector_weights.json")

# the selector's workload: kappa(A) log-uniform to 1e6, kappa(Z) log-uniform to 1e12 (random U), so that
# kappa(A^{1/2} Z) spreads over 1e0 .. 1e12
KAPPA_A = (0.0, 6.0)
KAPPA_Z = (0.0, 12.0)


def init_params(seed: int = 0):
    """He-initialised flat parameters (numpy float32), layout W1[64][16] b1[64] W2[64][64] b2[64] W3[4][64] b3[4]."""
    rng = np.random.default_rng(seed)
    parts = []
    for fan_in, fan_out in ((16, 64), (64, 64), (64, 4)):
        parts.append(rng.standard_normal((fan_out, fan_in)) * math.sqrt(2.0 / fan_in))
        parts.append(np.zeros(fan_out))
    return np.concatenate([p.ravel() for p in parts]).astype(np.float32)


def batch(count, seed, device="cuda", m_range=(64, 1024), n_range=(4, 64), log_kappa_a=KAPPA_A,
          log_kappa_z=KAPPA_Z):
    """A batch of the selector's workload (inputs.batch_instances with its kappa laws)."""
    from . import inputs
    return inputs.batch_instances(count, seed, device=device, m_range=m_range, n_range=n_range,
                                  log_kappa_a=log_kappa_a, log_kappa_z=log_kappa_z)


def option_orth(ctx, As, Zs):
    """||Q^T A Q - I||_2 of options 0-2 on every instance (inf after a breakdown): (count, 3) numpy array."""
    out = np.zeros((len(Zs), 3))
    for k in (ONE, TWO, SHIFTED):
        _, _, st, orth = ctx.oqr_batched_mixed(As, Zs, program=[PROGRAMS[k]] * len(Zs), check=True)
        o = orth.cpu().numpy()
        o[st.cpu().numpy() != 0] = np.inf
        out[:, k] = o
    return out


def labels_from(orth, tol=1e-12):
    """The cheapest option meeting tol; where none does, the shifted option (the most robust one)."""
    y = np.full(len(orth), SHIFTED, dtype=np.int32)
    for b in range(len(orth)):
        for k in (ONE, TWO, SHIFTED):
            if orth[b, k] <= tol:
                y[b] = k
                break
    return y


def make_set(ctx, count, seed, batch_size=1024, tol=1e-12, **kw):
    """Method-generated training data: features and labels of `count` instances, made batch by batch."""
    import torch
    X, y, orths = [], [], []
    for i, s in enumerate(range(0, count, batch_size)):
        As, Zs, _ = batch(min(batch_size, count - s), seed * 100003 + i, **kw)
        X.append(ctx.oqr_batched_features(As, Zs))
        o = option_orth(ctx, As, Zs)
        orths.append(o)
        y.append(torch.as_tensor(labels_from(o, tol), device=X[-1].device))
        del As, Zs
        torch.cuda.empty_cache()
    return {"X": torch.cat(X), "y": torch.cat(y), "orth": np.concatenate(orths)}


def train(ctx, X, y, epochs=60, lr=3e-3, batch=512, seed=0, params=None):
    """Adam on the mean cross-entropy, all arithmetic in the library's kernels."""
    import torch
    dev = X.device
    P = torch.as_tensor(init_params(seed) if params is None else params, device=dev).clone()
    m = torch.zeros_like(P)
    v = torch.zeros_like(P)
    n = X.shape[0]
    g = torch.Generator().manual_seed(seed)
    losses, t = [], 0
    for _ in range(epochs):
        perm = torch.randperm(n, generator=g).to(dev)
        acc = 0.0
        for i in range(0, n, batch):
            idx = perm[i:i + batch]
            grad, loss = ctx.oqr_mlp_grad(X[idx].contiguous(), y[idx].contiguous(), P)
            t += 1
            ctx.oqr_mlp_adam(P, grad, m, v, lr, t)
            acc += float(loss.item()) * len(idx)
        losses.append(acc / n)
    return P, losses


def choose(ctx, X, P):
    """Argmax option per feature row (BF16 inference kernel)."""
    _, choice = ctx.oqr_mlp_forward(X, P, bf16=True, want_logits=False)
    return choice


def solve_batch(ctx, As, Zs, P, tol=1e-12, check_all=False, stream=None):
    """The selector over a batch through the C ABI (oqr_batched, OQR_BATCHED_SELECTOR); returns
    (Qs, Rs, status, orth, choice) with orth NaN where the instance was not checked."""
    import torch

    from . import oqr as _oqr
    dev = Zs[0].device
    orth = torch.empty(len(Zs), dtype=torch.float64, device=dev)
    choice = torch.empty(len(Zs), dtype=torch.int32, device=dev)
    Qs, Rs, st = ctx.oqr_batched(As, Zs, mode=_oqr.OQR_BATCHED_SELECTOR, params=P, tol=tol, check_all=check_all,
                                 orth=orth, choice=choice, stream=stream)
    return Qs, Rs, st, orth, choice


def save(P, path=WEIGHTS, meta=None):
    with open(path, "w") as f:
        json.dump({"layout": "W1[64][16] b1[64] W2[64][64] b2[64] W3[4][64] b3[4]", "meta": meta or {},
                   "params": [float(x) for x in P.detach().cpu().numpy()]}, f)


def load(path=WEIGHTS, device="cuda"):
    import torch
    with open(path) as f:
        return torch.tensor(json.load(f)["params"], dtype=torch.float32, device=device)
