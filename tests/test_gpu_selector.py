"""Selector (learned choice of passes and precision) on the GPU.

The network's forward and backward kernels are checked against the CPU
restatement in oracle/mlp.py (itself pinned by finite differences); the
feature kernels against their definitions evaluated on the oracle's FP64 Gram;
the shifted A-CholQR3 option against the CHOL-EQR oracle; the selector mode of
oqr_batched (through the C ABI) against the oracle and the attainable
orthogonality.  The last test trains the network with the library's kernels on
method-generated instances and measures what it gains over the fixed policies
that meet the bar on every instance.
"""
import os
import time

import numpy as np
import pytest

import oracle
import selector_defs
from oracle import mlp
from paper_1401_5171_gb300 import inputs, selector

pytestmark = pytest.mark.gpu
U = 2.0 ** -53


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
    Q, R, (st, _) = ctx.oqr_cholqr2(Ad, Zd, shifted=1, prec=3, prec_mid=3, final_prec=3)
    assert st == 0
    # and the BF16X3-first shifted variant (trace-based shift) on the same instance
    Qb, Rb, (stb, infob) = ctx.oqr_cholqr2(Ad, Zd, shifted=1, prec=1, prec_mid=3, final_prec=3, check=2)
    assert stb == 0 and infob.orth_err <= 1e-12
    Q, R = Q.cpu().numpy(), R.cpu().numpy()
    assert oracle.orth_error(A, Q) <= max(1e-12, 10 * oracle.orth_error(A, Qr))
    assert oracle.repres_error(Z, Q, R) <= 1e-13
    assert np.linalg.norm(R - Rr) / np.linalg.norm(Rr) <= 1e-6


def _instances_host(As, Zs, idx):
    return [(As[b].cpu().numpy(), Zs[b].cpu().numpy()) for b in idx]


def test_batched_features_match_definition(env):
    """oqr_batched_features against the CPU definition (tests/selector_defs.py) evaluated on the oracle's
    FP64 Gram and Cholesky factor: instances that complete the first pass and instances that break down."""
    torch, oqr, ctx = env
    As, Zs, tab = inputs.batch_instances(24, seed=31, device="cuda", m_range=(64, 900), n_range=(1, 64),
                                         log_kappa_a=(0.0, 6.0), log_kappa_z=(0.0, 12.0))
    F = ctx.oqr_batched_features(As, Zs).cpu().numpy()
    for b, (A, Z) in enumerate(_instances_host(As, Zs, range(24))):
        m, n = Z.shape
        G0 = oracle.gram(A, Z)
        G0 = 0.5 * (G0 + G0.T)
        try:
            R1 = oracle.chol_upper(G0)
            col = 0
        except oracle.OracleBreakdown as e:
            R1, col = None, e.column
        ref = selector_defs.features(m, n, G0, R1, col)
        if (F[b, 10] == 1.0) != (R1 is None):
            continue          # at the breakdown threshold the two Grams' roundings may decide differently
        assert np.allclose(F[b, [0, 1, 2, 9, 10]], ref[[0, 1, 2, 9, 10]], atol=1e-5), b
        assert np.allclose(F[b, [3, 4]], ref[[3, 4]], atol=1e-4), b
        if R1 is not None:
            # sigma_min(R1)^2 of a Gram with kappa(G0) = kappa_sketch^2 moves by about kappa(G0) times the
            # Grams' relative difference (~1e-15): the feature, log10(kappa_sketch)/8, is held to that
            kap = 10.0 ** (8 * ref[12])
            tol = 1e-3 + min(0.1, kap * kap * 1e-15 / 8)
            assert abs(F[b, 12] - ref[12]) <= tol, (b, F[b, 12], ref[12])
            if ref[5] == 0.0:
                # the smallest pivot p of the scaled Gram moves by about 1e-15 / p relative (its rounding)
                pmin = 10.0 ** (-6 * ref[7])
                assert abs(F[b, 7] - ref[7]) <= 2e-3 + min(0.2, 1e-14 / pmin), b
                assert abs(F[b, 8] - ref[8]) <= 2e-3, b
        else:   # both broke down; where depends on the last bits of pivots near zero, so only the range is fixed
            assert 0.0 < F[b, 11] <= 1.0, b


def _bar(torch, As, Zs, Qs, st, tab):
    """Per instance: ||Q^T A Q - I||_2 (torch, FP64) and the bar max(1e-12, m u ||A||_2 ||Q||_2^2) (Thm 4.1's
    attainable level with c = 1; ||A||_2 = kappa(A), the smallest eigenvalue being 1)."""
    orth, bar = np.full(len(Zs), np.inf), np.zeros(len(Zs))
    for b in range(len(Zs)):
        m, n = Zs[b].shape
        qn = torch.linalg.matrix_norm(Qs[b], 2).item() if st[b] == 0 else 1.0
        bar[b] = max(1e-12, m * U * float(tab["kappa_A"][b]) * qn * qn)
        if st[b] == 0:
            E = Qs[b].T @ (As[b] @ Qs[b]) - torch.eye(n, dtype=torch.float64, device="cuda")
            orth[b] = torch.linalg.eigvalsh(0.5 * (E + E.T)).abs().max().item()
    return orth, bar


def test_selector_mode_through_the_c_abi(env):
    """OQR_BATCHED_SELECTOR with an untrained network (its choices are arbitrary): the checks and the
    fallback chain still give every instance a result at the bar, and R matches the oracle's."""
    torch, oqr, ctx = env
    As, Zs, tab = inputs.batch_instances(40, seed=41, device="cuda", m_range=(64, 700), n_range=(4, 64),
                                         log_kappa_a=(0.0, 6.0), log_kappa_z=(0.0, 10.0))
    P = torch.as_tensor(selector.init_params(3), device="cuda")
    Qs, Rs, st, orth, choice = selector.solve_batch(ctx, As, Zs, P)
    st = st.cpu().numpy()
    ch = choice.cpu().numpy()
    assert set(ch.tolist()) <= {0, 1, 2, 3}
    o, bar = _bar(torch, As, Zs, Qs, st, tab)
    for b in range(40):
        assert st[b] == 0, (b, st[b])
        assert o[b] <= bar[b], (b, ch[b], o[b], bar[b])
    for b in range(0, 40, 8):       # a sample against the oracle
        A, Z = As[b].cpu().numpy(), Zs[b].cpu().numpy()
        Qr, Rr = oracle.oblique_qr(A, Z)
        assert np.linalg.norm(Rs[b].cpu().numpy() - Rr) / np.linalg.norm(Rr) <= max(1e-12, 100 * U * np.linalg.cond(Rr))


def _forced(torch, k):
    """Network parameters whose choice is always option k (last layer: zero weights, bias one-hot)."""
    p = np.zeros(mlp.COUNT, dtype=np.float32)
    p[-4 + k] = 10.0
    return torch.as_tensor(p, device="cuda")


def test_selector_routes_on_the_device(env):
    """The routes decided on the device, each forced by the network on a batch whose kappa(A^{1/2} Z) reaches
    ~1e11: 'plain' (options 1 and 2) must settle one-pass against two-pass from the pass-1 Gram and send
    the instances a plain route cannot reach to the late shifted refactor (reported as the shifted
    option); 'shift' runs shifted A-CholQR3 from the probe's Gram; every result meets the bar, with the
    extra check's values (check_all) at most that bar."""
    torch, oqr, ctx = env
    As, Zs, tab = inputs.batch_instances(48, seed=43, device="cuda", m_range=(64, 1500), n_range=(4, 64),
                                         log_kappa_a=(0.0, 5.0), log_kappa_z=(0.0, 9.0))
    for k in (0, 1, 2):
        Qs, Rs, st, orth, choice = selector.solve_batch(ctx, As, Zs, _forced(torch, k), check_all=True)
        st, ch, orth = st.cpu().numpy(), choice.cpu().numpy(), orth.cpu().numpy()
        o, bar = _bar(torch, As, Zs, Qs, st, tab)
        for b in range(len(Zs)):
            assert st[b] == 0, (k, b, st[b])
            assert o[b] <= bar[b], (k, b, ch[b], o[b], bar[b])
            assert np.isnan(orth[b]) or orth[b] <= 10 * bar[b] + 1e-12, (k, b, orth[b])
        if k < 2:
            assert set(ch.tolist()) <= {0, 1, 2}
            assert (ch == 2).any(), "no instance of this batch needed the late shifted refactor"
            assert (ch < 2).any()
        else:
            assert set(ch.tolist()) == {2}


def test_selector_trains_and_beats_fixed_policies(env):
    """Train on method-generated instances (m <= 1024) with the library's kernels; then, on the selector's
    workload at the batched sizes (m up to 4096, kappa(A^{1/2} Z) to ~1e12), the selector through the C ABI
    against the fixed policies that meet the bar everywhere: always shifted A-CholQR3 on the tensor cores,
    and always A-CholQR2 on the tensor cores with the same check and fallback.  Every result of the selector
    must meet the bar; it must be faster than both."""
    torch, oqr, ctx = env
    tr = selector.make_set(ctx, 8192, seed=5, batch_size=2048)
    P, losses = selector.train(ctx, tr["X"], tr["y"], epochs=40)
    assert losses[-1] < 0.7 * losses[0]
    ho = selector.make_set(ctx, 512, seed=6, batch_size=512, m_range=(64, 4096))
    acc = float(np.mean(selector.choose(ctx, ho["X"], P).cpu().numpy() == ho["y"].cpu().numpy()))
    assert acc >= 0.7, acc
    if os.path.exists(selector.WEIGHTS):
        P = selector.load()                 # the committed network, trained on 1e5 instances
    As, Zs, tab = selector.batch(1024, seed=77, m_range=(64, 4096))

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = fn()
        torch.cuda.synchronize()
        return time.perf_counter() - t0, out

    t_sel, (Qs, Rs, st, orth, choice) = timed(lambda: selector.solve_batch(ctx, As, Zs, P))
    st = st.cpu().numpy()
    o, bar = _bar(torch, As, Zs, Qs, st, tab)
    bad = [b for b in range(len(Zs)) if not (o[b] <= bar[b])]
    assert not bad, [(b, o[b], bar[b], int(choice[b])) for b in bad[:5]]
    t_shift, _ = timed(lambda: ctx.oqr_batched(As, Zs, mode=oqr.OQR_BATCHED_SHIFTED_TC))
    # always A-CholQR2 (tensor cores): every result checked, failures to shifted A-CholQR3
    def cholqr2_checked():
        _, _, st2, o2 = ctx.oqr_batched_mixed(As, Zs, program=[2] * len(Zs), check=True)
        fail = [b for b in range(len(Zs)) if st2[b].item() != 0 or not (o2[b].item() <= 1e-12)]
        if fail:
            ctx.oqr_batched_mixed([As[b] for b in fail], [Zs[b] for b in fail], program=[3] * len(fail), check=True)
    t_c2, _ = timed(cholqr2_checked)
    mix = np.bincount(choice.cpu().numpy(), minlength=4).tolist()
    print(f"\nselector: trained loss {losses[0]:.3f} -> {losses[-1]:.3f}, held-out accuracy {acc:.3f}; on 1024 "
          f"instances: selector {t_sel:.3f}s (options used {mix}), always shifted A-CholQR3 {t_shift:.3f}s "
          f"({t_shift / t_sel:.2f}x), always A-CholQR2 + check + fallback {t_c2:.3f}s ({t_c2 / t_sel:.2f}x)")
    assert t_sel < t_shift and t_sel < t_c2
