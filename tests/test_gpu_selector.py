"""Selector (learned choice of passes and precision) on the GPU.

The network's forward and backward kernels are checked against the CPU
restatement in oracle/mlp.py (itself pinned by finite differences); the
feature kernel against its definition evaluated on the oracle's FP64 Gram; the
mixed shifted A-CholQR3 option against the CHOL-EQR oracle.  The last test
trains the network with the library's kernels on method-generated instances
and measures what it gains over always running the safe mixed option, with
every result meeting ||Q^T A Q - I||_2 <= 1e-12 after the FP64 fallback.
"""
import time

import numpy as np
import pytest

import oracle
from oracle import mlp
from paper_1401_5171_gb300 import inputs, selector

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1401_5171_gb300 import oqr
    return torch, oqr, oqr.Oqr(0)


def test_mlp_forward_matches_oracle(env):
    torch, oqr, ctx = env
    rng = np.random.default_rng(2)
    p = (rng.standard_normal(mlp.COUNT) * 0.2).astype(np.float32)
    X = rng.standard_normal((300, 16)).astype(np.float32)
    z_ref, _ = mlp.forward(p.astype(np.float64), X.astype(np.float64))
    P, Xd = torch.tensor(p, device="cuda"), torch.tensor(X, device="cuda")
    z32, c32 = ctx.oqr_mlp_forward(Xd, P, bf16=False)
    z32 = z32.cpu().numpy()
    assert np.max(np.abs(z32 - z_ref)) <= 1e-4 * (1 + np.abs(z_ref).max())
    assert np.array_equal(c32.cpu().numpy(), np.argmax(z32, axis=1))
    z16, c16 = ctx.oqr_mlp_forward(Xd, P, bf16=True)
    z16 = z16.cpu().numpy()
    assert np.max(np.abs(z16 - z_ref)) <= 0.05 * (1 + np.abs(z_ref).max())
    margin = np.sort(z_ref, axis=1)[:, -1] - np.sort(z_ref, axis=1)[:, -2]
    clear = margin > 0.1 * (1 + np.abs(z_ref).max())
    assert np.all(c16.cpu().numpy()[clear] == np.argmax(z_ref, axis=1)[clear])


def test_mlp_gradient_matches_oracle(env):
    torch, oqr, ctx = env
    rng = np.random.default_rng(3)
    p = (rng.standard_normal(mlp.COUNT) * 0.2).astype(np.float32)
    X = rng.standard_normal((257, 16)).astype(np.float32)
    y = rng.integers(0, 4, size=257).astype(np.int32)
    loss_ref, g_ref = mlp.loss_and_grad(p.astype(np.float64), X.astype(np.float64), y)
    g, loss = ctx.oqr_mlp_grad(torch.tensor(X, device="cuda"), torch.tensor(y, device="cuda"),
                               torch.tensor(p, device="cuda"))
    g = g.cpu().numpy()
    assert abs(loss.item() - loss_ref) <= 1e-5 * (1 + loss_ref)
    assert np.linalg.norm(g - g_ref) <= 1e-4 * np.linalg.norm(g_ref)
    assert np.max(np.abs(g - g_ref)) <= 1e-5 + 1e-3 * np.abs(g_ref).max()


def test_adam_step_definition(env):
    torch, oqr, ctx = env
    rng = np.random.default_rng(4)
    p = rng.standard_normal(mlp.COUNT).astype(np.float32)
    g = rng.standard_normal(mlp.COUNT).astype(np.float32)
    m = rng.standard_normal(mlp.COUNT).astype(np.float32) * 0.1
    v = np.abs(rng.standard_normal(mlp.COUNT)).astype(np.float32) * 0.1
    P, G, M, V = (torch.tensor(a, device="cuda") for a in (p, g, m, v))
    ctx.oqr_mlp_adam(P, G, M, V, lr=1e-2, t=3)
    b1, b2, eps = 0.9, 0.999, 1e-8
    m1 = b1 * m + (1 - b1) * g
    v1 = b2 * v + (1 - b2) * g * g
    p1 = p - 1e-2 * (m1 / (1 - b1 ** 3)) / (np.sqrt(v1 / (1 - b2 ** 3)) + eps)
    assert np.allclose(P.cpu().numpy(), p1, rtol=1e-5, atol=1e-6)


def features_def(m, n, G, normA, normZ2):
    d = np.diag(G)
    C = G / np.sqrt(np.outer(d, d))
    off = np.abs(C - np.diag(np.diag(C)))
    f = np.zeros(16)
    f[0], f[1], f[2] = np.log10(m) / 4, np.log10(n) / 2, n / m
    f[3], f[4] = np.log10(d.max() / d.min()) / 6, off.max()
    piv = np.diag(np.linalg.cholesky(C)) ** 2
    f[7], f[8] = -np.log10(piv.min()) / 6, np.log10(piv.max()) / 6
    f[9], f[10], f[11] = np.log10(normA) / 6, np.log10(normZ2) / 6, np.log10(d.sum() / d.max()) / 3
    return f


@pytest.mark.parametrize("seed,m,n,kz", [(1, 300, 12, 1e1), (2, 800, 40, 1e2), (3, 500, 64, 1e3)])
def test_features_match_definition(env, seed, m, n, kz):
    torch, oqr, ctx = env
    A, Z = inputs.paper_case(4, m, n, 1e4, kz, seed=seed)
    f = ctx.oqr_features(oqr.colmajor(torch.as_tensor(A).cuda()), oqr.colmajor(torch.as_tensor(Z).cuda()))
    f = f.cpu().numpy()
    ref = features_def(m, n, oracle.gram(A, Z), np.linalg.norm(A), np.linalg.norm(Z) ** 2)
    assert f[5] == 0.0 and f[6] == 0.0
    assert np.allclose(f[[0, 1, 2, 9, 10, 11]], ref[[0, 1, 2, 9, 10, 11]], atol=1e-5)
    assert np.allclose(f[[3, 4, 8]], ref[[3, 4, 8]], atol=1e-3)
    assert abs(f[7] - ref[7]) <= 0.02             # pivots of a BF16X3 matrix


def test_mixed_shifted_cholqr3_option(env):
    # kappa(A^{1/2} Z) ~ 1e9: beyond the unshifted methods, within shifted A-CholQR3
    # (all passes FP64-accurate on the tensor cores)
    torch, oqr, ctx = env
    A, Z = inputs.paper_case(4, 600, 20, 1e4, 1e9, seed=21)
    Qr, Rr = oracle.oblique_qr(A, Z)
    Ad, Zd = (oqr.colmajor(torch.as_tensor(x).cuda()) for x in (A, Z))
    Q, R, st, orth = selector.run_option(ctx, 2, Ad, Zd)
    assert st == 0
    # and the BF16X3-first shifted variant (trace-based shift) on the same instance
    Qb, Rb, (stb, infob) = ctx.oqr_cholqr2(Ad, Zd, shifted=1, prec=1, prec_mid=3, final_prec=3, check=2)
    assert stb == 0 and infob.orth_err <= 1e-12
    Q, R = Q.cpu().numpy(), R.cpu().numpy()
    assert oracle.orth_error(A, Q) <= max(1e-12, 10 * oracle.orth_error(A, Qr))
    assert oracle.repres_error(Z, Q, R) <= 1e-13
    assert np.linalg.norm(R - Rr) / np.linalg.norm(Rr) <= 1e-6


def test_selector_trains_and_gains(env):
    """Train on small and mid-size instances; evaluate on large ones, where the
    options' costs differ: time of selected-option + check + fallback against
    always running the plain FP64 A-CholQR2 (the method without the network)
    and against always running the safe shifted mixed A-CholQR3."""
    torch, oqr, ctx = env
    tr1 = selector.make_set(ctx, 700, seed=100, m_range=(64, 1024), n_range=(4, 64))
    tr2 = selector.make_set(ctx, 160, seed=101, m_range=(2048, 6144), n_range=(8, 64))
    X = torch.cat([tr1["X"], tr2["X"]])
    y = torch.cat([tr1["y"], tr2["y"]])
    P, losses = selector.train(ctx, X, y, epochs=150)
    assert losses[-1] < 0.6 * losses[0]
    count = 48
    feats, labels = [], []
    t_sel = t_safe = t_fp64 = 0.0
    fallbacks = 0
    for A, Z in selector.instances(count, seed=200, m_range=(8192, 12288), n_range=(16, 64)):
        lab, orth = selector.label_instance(ctx, A, Z)
        labels.append(lab)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Q, R, info = selector.solve(ctx, A, Z, P)
        torch.cuda.synchronize()
        t_sel += time.perf_counter() - t0
        fallbacks += info["fallback"]
        feats.append(info["choice"])
        best = np.min(orth)
        if np.isfinite(best):                     # some option completes: so must the chain
            assert info["status"] == 0
            if info["used"] in (0, 1) or best <= 1e-12:
                assert info["orth"] <= max(1e-12, 10 * best)
        for k, acc in ((2, "safe"), (3, "fp64")):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            selector.run_option(ctx, k, A, Z, check=False)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            if acc == "safe":
                t_safe += dt
            else:
                t_fp64 += dt
        del A, Z, Q, R
    acc = float(np.mean(np.array(feats) == np.array(labels)))
    print(f"\nselector: train label mix {np.bincount(y.cpu().numpy(), minlength=4)}, held-out (m 8192-12288) "
          f"accuracy {acc:.3f}, fallbacks {fallbacks}/{count}; time features+choice+selected+check "
          f"{t_sel:.3f}s vs always FP64 A-CholQR2 {t_fp64:.3f}s ({t_fp64 / t_sel:.2f}x) vs always shifted "
          f"mixed A-CholQR3 {t_safe:.3f}s ({t_safe / t_sel:.2f}x); the baselines run without a check")
    assert acc >= 0.6
    assert t_sel < t_fp64
