"""Learned selector over the normal-equation variants (host-side driver).

For each instance the selector reads 16 features from the instance's cheap
BF16X3 normal-equation matrix (oqr_features), runs the MLP 16 -> 64 -> 64 -> 4
(oqr_mlp_forward, BF16 inference) and picks one option, cheapest first:

  0  one FP64-accurate pass          (A-CholQR, tensor cores)
  1  TC2 pass + FP64-accurate pass    (mixed A-CholQR2, one split of A for both)
  2  shifted A-CholQR3, all three passes FP64-accurate on the tensor cores
  3  FP64 A-CholQR2 (DFMA)           -- also the fallback

A choice of option 0 or 1 is checked (||Q^T A Q - I||_2 <= tol, measured on
the FP64-accurate tensor-core Gram); if the check fails or a Cholesky breaks
down, the instance is refactored with option 3, and if that does not meet tol
either (an unshifted normal-equation method needs kappa(A^{1/2} Z)^2 u < 1),
with the shifted FP64 A-CholQR3 and then option 2, keeping the most
orthogonal result.  A choice of option 2 or 3 is the network's answer for an
ill-conditioned instance and is accepted once it completes.  Training labels are the cheapest option
whose measured orthogonality meets tol on method-generated instances; the
network is trained on the GPU by the library's own kernels (oqr_mlp_grad,
oqr_mlp_adam).  Every arithmetic step runs in the CUDA library.
"""
from __future__ import annotations

import json
import math
import time

import numpy as np

OPTIONS = [
    ("oqr_cholqr", {"final_prec": 3}),
    ("oqr_cholqr2", {"prec": 4, "final_prec": 3}),
    ("oqr_cholqr2", {"shifted": 1, "prec": 3, "prec_mid": 3, "final_prec": 3}),
    ("oqr_cholqr2", {}),
    ("oqr_cholqr2", {"shifted": 1}),   # last resort, not a class of the network
]
FALLBACK = 3
LAST_RESORT = 4
CLASSES = 4


def init_params(seed: int = 0):
    """He-initialised flat parameters (numpy float32)."""
    rng = np.random.default_rng(seed)
    parts = []
    for fan_in, fan_out in ((16, 64), (64, 64), (64, 4)):
        parts.append(rng.standard_normal((fan_out, fan_in)) * math.sqrt(2.0 / fan_in))
        parts.append(np.zeros(fan_out))
    return np.concatenate([p.ravel() for p in parts]).astype(np.float32)


def run_option(ctx, k, A, Z, Q=None, R=None, check=True):
    """Option k with the orthogonality check on the FP64-accurate tensor-core Gram."""
    name, kw = OPTIONS[k]
    Q, R, (st, info) = ctx._qr(name, A, Z, Q=Q, R=R, raise_on_error=False, check=2 if check else 0, **kw)
    return Q, R, st, (info.orth_err if st == 0 else float("inf"))


def label_instance(ctx, A, Z, tol=1e-12):
    """The cheapest option meeting tol; if none does, the most orthogonal option that
    completes (the shifted mixed A-CholQR3 when every option breaks down).  Also
    returns the orthogonality each option reached (inf for a breakdown)."""
    orth = []
    for k in range(CLASSES):
        _, _, st, o = run_option(ctx, k, A, Z)
        orth.append(o)
    for k, o in enumerate(orth):
        if o <= tol:
            return k, orth
    if np.all(np.isinf(orth)):
        return 2, orth
    return int(np.argmin(orth)), orth


def instances(count, seed, device="cuda", m_range=(64, 512), n_range=(4, 32), log_kappa_a=(0.0, 6.0),
              log_kappa_z=(0.0, 12.0)):
    """Yields (A, Z) of the selector's workload one at a time (kappa(A^{1/2} Z) log-uniform
    up to ~1e12 through kappa(Z) with a random U), so that large sets need not be resident."""
    from . import inputs
    m, n, ka, kz, seeds = inputs.batch_shapes(count, seed, m_range, n_range, log_kappa_a, log_kappa_z)
    for b in range(count):
        A, _ = inputs.dense_spd(int(m[b]), float(ka[b]), seed=int(seeds[b]), device=device)
        Z = inputs.tall_z(int(m[b]), int(n[b]), float(kz[b]), seed=int(seeds[b]) + 1, device=device)
        yield A.t(), Z.t().contiguous().t()


def make_set(ctx, count, seed, device="cuda", tol=1e-12, keep=False, **kw):
    """Method-generated instances with features and labels (torch tensors on device)."""
    import torch
    X = torch.empty((count, 16), dtype=torch.float32, device=device)
    y = torch.empty(count, dtype=torch.int32, device=device)
    orth = np.zeros((count, CLASSES))
    As, Zs = [], []
    for b, (A, Z) in enumerate(instances(count, seed, device, **kw)):
        ctx.oqr_features(A, Z, out=X[b])
        lab, o = label_instance(ctx, A, Z, tol)
        y[b] = lab
        orth[b] = o
        if keep:
            As.append(A)
            Zs.append(Z)
    torch.cuda.synchronize()
    return {"As": As, "Zs": Zs, "X": X, "y": y, "orth": orth}


def train(ctx, X, y, epochs=400, lr=3e-3, batch=256, seed=0, params=None):
    """Adam on the mean cross-entropy, all arithmetic in the library's kernels."""
    import torch
    dev = X.device
    P = torch.as_tensor(init_params(seed) if params is None else params, device=dev).clone()
    m = torch.zeros_like(P)
    v = torch.zeros_like(P)
    n = X.shape[0]
    g = torch.Generator().manual_seed(seed)
    losses, t = [], 0
    for ep in range(epochs):
        perm = torch.randperm(n, generator=g).to(dev)
        for i in range(0, n, batch):
            idx = perm[i:i + batch]
            grad, loss = ctx.oqr_mlp_grad(X[idx].contiguous(), y[idx].contiguous(), P)
            t += 1
            ctx.oqr_mlp_adam(P, grad, m, v, lr, t)
        losses.append(float(loss.item()))
    return P, losses


def choose(ctx, X, P):
    """Argmax option per feature row (BF16 inference kernel)."""
    _, choice = ctx.oqr_mlp_forward(X, P, bf16=True, want_logits=False)
    return choice


def solve(ctx, A, Z, P, tol=1e-12):
    """Selected factorization with check and fallback; returns (Q, R, info)."""
    import torch
    f = ctx.oqr_features(A, Z).reshape(1, 16)
    k = int(choose(ctx, f, P)[0].item())
    # options 0 and 1 are only right for well-conditioned instances: their result is checked;
    # options 2 and 3 are the network's answer for hard instances and are accepted once they complete
    risky = k in (0, 1)
    Q, R, st, o = run_option(ctx, k, A, Z, check=risky)
    ok = st == 0 and (o <= tol or not risky)
    fell = not ok
    used = k
    # fallback chain: FP64 A-CholQR2, then the shifted methods, keeping the most orthogonal result
    for fb in (FALLBACK, LAST_RESORT, 2):
        if ok:
            break
        if fb == k:
            continue
        Q2, R2, st2, o2 = run_option(ctx, fb, A, Z)
        if st2 == 0 and (st != 0 or o2 < o):
            Q, R, st, o, used = Q2, R2, st2, o2, fb
        ok = st == 0 and o <= tol
    return Q, R, {"choice": k, "fallback": fell, "used": used, "orth": o, "status": st}


# options -> programs of the batched tensor-core path (option 3, FP64 A-CholQR2, is oqr_batched mode 0)
BATCH_PROGRAMS = {0: 0, 1: 1, 2: 3}   # OQR_BATCH_CHOLQR_TC, OQR_BATCH_CHOLQR2_TC2, OQR_BATCH_SCHOLQR3_TC


def solve_batch(ctx, As, Zs, P, tol=1e-12, stream=None):
    """The selector over a batch.  Per-instance features (oqr_features), one MLP forward over the batch,
    then the chosen tensor-core programs in one checked oqr_batched_mixed call and the FP64 A-CholQR2
    choices in one oqr_batched call.  Options 0 and 1 are accepted when their check meets tol, option 2
    and 3 once they complete (the network's answer for hard instances).  Every other instance goes down
    the fallback chain in batches: shifted A-CholQR3 on the tensor cores (checked), then FP64 A-CholQR2,
    keeping the most orthogonal completed result.  Returns (Qs, Rs, info) with per-instance lists
    choice, used, orth (nan where the result was not checked) and status."""
    import torch
    from . import oqr as _oqr
    B = len(Zs)
    dev = Zs[0].device
    X = torch.empty((B, 16), dtype=torch.float32, device=dev)
    for b in range(B):
        ctx.oqr_features(As[b], Zs[b], out=X[b], stream=stream)
    choice = [int(c) for c in choose(ctx, X, P).cpu().tolist()]
    Qs = [_oqr.empty_colmajor(z.shape[0], z.shape[1], dev) for z in Zs]
    Rs = [_oqr.empty_colmajor(z.shape[1], z.shape[1], dev) for z in Zs]
    used = [None] * B
    orth = [float("inf")] * B
    status = [1] * B
    accepted = [False] * B

    def run_tc(idx, programs):
        Qt = [_oqr.empty_colmajor(Zs[b].shape[0], Zs[b].shape[1], dev) for b in idx]
        Rt = [_oqr.empty_colmajor(Zs[b].shape[1], Zs[b].shape[1], dev) for b in idx]
        _, _, st, o = ctx.oqr_batched_mixed([As[b] for b in idx], [Zs[b] for b in idx], program=programs,
                                            Qs=Qt, Rs=Rt, stream=stream, check=True)
        return Qt, Rt, st.cpu().tolist(), o.cpu().tolist()

    def run_fp64(idx):
        Qt = [_oqr.empty_colmajor(Zs[b].shape[0], Zs[b].shape[1], dev) for b in idx]
        Rt = [_oqr.empty_colmajor(Zs[b].shape[1], Zs[b].shape[1], dev) for b in idx]
        _, _, st = ctx.oqr_batched([As[b] for b in idx], [Zs[b] for b in idx], Qs=Qt, Rs=Rt, stream=stream)
        return Qt, Rt, st.cpu().tolist(), [float("nan")] * len(idx)

    def take(idx, res, options):
        """Keeps each completed result that is the instance's first or more orthogonal than its last."""
        Qt, Rt, st, o = res
        for k, b in enumerate(idx):
            if st[k] != 0:
                continue
            if status[b] != 0 or o[k] < orth[b]:
                Qs[b].copy_(Qt[k])
                Rs[b].copy_(Rt[k])
                status[b], orth[b], used[b] = 0, o[k], options[k]
            if options[k] in (2, 3) or o[k] <= tol:
                accepted[b] = True

    tc = [b for b in range(B) if choice[b] != 3]
    if tc:
        take(tc, run_tc(tc, [BATCH_PROGRAMS[choice[b]] for b in tc]), [choice[b] for b in tc])
    fp = [b for b in range(B) if choice[b] == 3]
    if fp:
        take(fp, run_fp64(fp), [3] * len(fp))
    rest = [b for b in range(B) if not accepted[b]]
    if rest:
        take(rest, run_tc(rest, [BATCH_PROGRAMS[2]] * len(rest)), [2] * len(rest))
    rest = [b for b in range(B) if status[b] != 0]
    if rest:
        take(rest, run_fp64(rest), [3] * len(rest))
    return Qs, Rs, {"choice": choice, "used": used, "orth": orth, "status": status}


def save(P, path):
    with open(path, "w") as f:
        json.dump({"layout": "W1[64][16] b1[64] W2[64][64] b2[64] W3[4][64] b3[4]",
                   "params": [float(x) for x in P.detach().cpu().numpy()]}, f)


def load(path, device="cuda"):
    import torch
    with open(path) as f:
        return torch.tensor(json.load(f)["params"], dtype=torch.float32, device=device)
