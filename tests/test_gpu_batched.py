"""GPU parity of the batched A-CholQR2 (oqr_batched) against the CPU oracle.

Batches follow the batched workload's recipe (m, n uniform integers,
kappa(A), kappa(Z) log-uniform up to 1e6, dense SPD A).  Every instance is
compared with the oracle (CHOL-EQR, Algorithm 3) on the small batches; the
full 4096-instance batch is checked on every instance through properties
that fix (Q, R) (Q^T A Q = I, Z = QR, R upper with positive diagonal) and on a
stratified sample against the oracle.  A Cholesky breakdown is an accepted
outcome only where the oracle's kappa(R) exceeds 1e7 (the normal-equation
methods need kappa(A^{1/2} Z)^2 u < 1).
"""
import numpy as np
import pytest

import oracle
from paper_1401_5171_gb300 import autotune, inputs

pytestmark = pytest.mark.gpu
U = 2.0 ** -53


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1401_5171_gb300 import oqr
    return torch, oqr, oqr.Oqr(0)


def check_instance(A, Z, Q, R, status):
    Qr, Rr = oracle.oblique_qr(A, Z)
    kap = np.linalg.cond(Rr)
    if status != 0:
        assert kap > 1e7, f"breakdown at column {status} with kappa(R) = {kap:.2e}"
        return
    assert np.all(np.tril(R, -1) == 0) and np.all(np.diag(R) > 0)
    assert np.linalg.norm(R - Rr) / np.linalg.norm(Rr) <= max(1e-12, 50 * U * kap)
    floor = 100 * U * np.linalg.eigvalsh(A).max() * np.linalg.norm(Qr, 2) ** 2
    assert oracle.orth_error(A, Q) <= max(1e-12, 10 * oracle.orth_error(A, Qr), floor)


def test_batched_small_parity(env):
    torch, oqr, ctx = env
    As, Zs, tab = inputs.batch_instances(40, seed=3, device="cuda", m_range=(64, 700), n_range=(4, 64))
    Qs, Rs, st = ctx.oqr_batched(As, Zs)
    torch.cuda.synchronize()
    st = st.cpu().numpy()
    for b in range(len(Zs)):
        check_instance(As[b].cpu().numpy(), Zs[b].cpu().numpy(), Qs[b].cpu().numpy(), Rs[b].cpu().numpy(), st[b])


def test_batched_breakdown_is_isolated(env):
    torch, oqr, ctx = env
    As, Zs, _ = inputs.batch_instances(6, seed=5, device="cuda", m_range=(64, 300), n_range=(4, 40),
                                       log_kappa_z=(0.0, 2.0))
    bad = torch.eye(100, dtype=torch.float64, device="cuda")
    bad[7, 7] = -1.0                             # indefinite: breaks at column 8 for Z = I[:, :10]
    As.insert(2, oqr.colmajor(bad))
    Zs.insert(2, oqr.colmajor(torch.eye(100, 10, dtype=torch.float64, device="cuda")))
    Qs, Rs, st = ctx.oqr_batched(As, Zs)
    torch.cuda.synchronize()
    st = st.cpu().numpy()
    assert st[2] == 8
    for b in range(len(Zs)):
        if b != 2:
            check_instance(As[b].cpu().numpy(), Zs[b].cpu().numpy(), Qs[b].cpu().numpy(), Rs[b].cpu().numpy(), st[b])


def test_batched_plans_agree(env):
    # different work plans change only the rounding order of the Gram partial sums
    torch, oqr, ctx = env
    As, Zs, _ = inputs.batch_instances(12, seed=9, device="cuda", m_range=(500, 1500), n_range=(4, 64),
                                       log_kappa_z=(0.0, 3.0))
    ms = [z.shape[0] for z in Zs]
    outs = []
    for t in (64, 4096):
        plan = [autotune.splits_for(m, t) for m in ms]
        Qs, Rs, st = ctx.oqr_batched(As, Zs, splits=plan)
        torch.cuda.synchronize()
        assert st.abs().sum().item() == 0
        outs.append([r.cpu().numpy() for r in Rs])
    for R1, R2 in zip(*outs):
        assert np.linalg.norm(R1 - R2) / np.linalg.norm(R1) < 1e-12


def test_batched_graph_replay_same_result(env):
    torch, oqr, ctx = env
    As, Zs, _ = inputs.batch_instances(10, seed=13, device="cuda", m_range=(64, 400), n_range=(4, 64),
                                       log_kappa_z=(0.0, 2.0))
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        _, R1, st1 = ctx.oqr_batched(As, Zs, stream=s)
        _, R2, st2 = ctx.oqr_batched(As, Zs, stream=s)     # replays the cached graph
    torch.cuda.synchronize()
    for a, b in zip(R1, R2):
        assert torch.equal(a, b)


def check_full_batch(torch, As, Zs, Qs, Rs, st, tab):
    """Properties that fix (Q, R) on every instance; returns the number of completed instances and
    each instance's ||Q^T A Q - I||_2 (-1 where it broke down)."""
    ok = 0
    orths = np.full(len(Zs), -1.0)
    for b in range(len(Zs)):
        A, Z, Q, R = As[b], Zs[b], Qs[b], Rs[b]
        if st[b] != 0:
            # breakdown only for kappa(A^{1/2} Z) beyond the method's reach
            G = Z.T @ (A @ Z)
            ev = torch.linalg.eigvalsh(0.5 * (G + G.T))
            assert (ev.max() / ev.min().clamp_min(1e-300)).item() > 1e14
            continue
        ok += 1
        n = Z.shape[1]
        E = Q.T @ (A @ Q) - torch.eye(n, dtype=torch.float64, device="cuda")
        orth = torch.linalg.eigvalsh(0.5 * (E + E.T)).abs().max().item()
        orths[b] = orth
        nA = float(tab["kappa_A"][b])                  # ||A||_2 = kappa(A) (smallest eigenvalue 1)
        qn = torch.linalg.matrix_norm(Q, 2).item()
        assert orth <= max(1e-12, 1e3 * Z.shape[0] * U * nA * qn * qn)
        rep = (torch.linalg.matrix_norm(Z - Q @ R, 2) / torch.linalg.matrix_norm(Z, 2)).item()
        assert rep <= 1e-13
        assert torch.all(torch.tril(R, -1) == 0) and torch.all(torch.diagonal(R) > 0)
    assert ok >= 0.9 * len(Zs)
    return ok, orths


def check_worst_against_oracle(As, Zs, orths):
    """The batch's least orthogonal instance against the oracle's own orthogonality on it.

    Thm 4.1 puts the attainable floor at c m u ||A|| ||Q||^2 (CHOL-EQR reaches it); an instance
    above 1e-12 must be within 10x of the oracle there, i.e. at the floor, not an emulation loss."""
    b = int(np.argmax(orths))
    A, Z = As[b].cpu().numpy(), Zs[b].cpu().numpy()
    Qr, _ = oracle.oblique_qr(A, Z)
    orth_ref = oracle.orth_error(A, Qr)
    assert orths[b] <= max(1e-12, 10 * orth_ref), (b, A.shape[0], Z.shape[1], orths[b], orth_ref)
    return b, orths[b], orth_ref


def test_config3_full_batch(env):
    """4096 instances, m in [64, 4096], n in [4, 64], kappa(A), kappa(Z) log-uniform in [1, 1e6]; the FP64
    path, then the tensor-core path (every pass FP64-accurate; about 20 waves of packed instances)."""
    torch, oqr, ctx = env
    As, Zs, tab = inputs.batch_instances(4096, seed=2024, device="cuda")
    plan, table, _ = autotune.tune(ctx, As[:512], Zs[:512], reps=1)
    plan = autotune.plan_from_table([z.shape[0] for z in Zs], table)
    Qs, Rs, st = ctx.oqr_batched(As, Zs, splits=plan)
    torch.cuda.synchronize()
    st = st.cpu().numpy()
    _, orth64 = check_full_batch(torch, As, Zs, Qs, Rs, st, tab)
    worst64 = check_worst_against_oracle(As, Zs, orth64)
    # stratified oracle sample: one instance per m-quartile with m <= 2500
    ms = np.array([z.shape[0] for z in Zs])
    for lo, hi in ((64, 700), (700, 1400), (1400, 2000), (2000, 2500)):
        cand = [b for b in range(len(Zs)) if lo <= ms[b] < hi and st[b] == 0]
        b = cand[0]
        check_instance(As[b].cpu().numpy(), Zs[b].cpu().numpy(), Qs[b].cpu().numpy(), Rs[b].cpu().numpy(), st[b])
    # the tensor-core path on the same batch: same properties, and R agrees with the FP64 path's
    torch.cuda.empty_cache()
    Qm, Rm, stm = ctx.oqr_batched(As, Zs, Qs=Qs, mode=1)
    torch.cuda.synchronize()
    stm = stm.cpu().numpy()
    _, orthm = check_full_batch(torch, As, Zs, Qm, Rm, stm, tab)
    worstm = check_worst_against_oracle(As, Zs, orthm)
    print(f"config-3 batch worst instances (index, GPU orth, oracle orth): FP64 {worst64}, tensor cores {worstm}")
    for b in range(len(Zs)):
        if st[b] == 0 and stm[b] == 0:
            kap = torch.linalg.cond(Rs[b]).item()
            assert (torch.linalg.norm(Rm[b] - Rs[b]) / torch.linalg.norm(Rs[b])).item() <= max(1e-12, 100 * U * kap)


# ---- the tensor-core form (oqr_batched_mixed; oqr_batched modes 1 and 2) -------------------------

def test_batched_mixed_parity(env):
    """Every pass FP64-accurate on the tensor cores (mode 1): the FP64 path's tolerances."""
    torch, oqr, ctx = env
    As, Zs, _ = inputs.batch_instances(40, seed=3, device="cuda", m_range=(64, 700), n_range=(4, 64))
    Qs, Rs, st = ctx.oqr_batched(As, Zs, mode=1)
    torch.cuda.synchronize()
    st = st.cpu().numpy()
    for b in range(len(Zs)):
        check_instance(As[b].cpu().numpy(), Zs[b].cpu().numpy(), Qs[b].cpu().numpy(), Rs[b].cpu().numpy(), st[b])


def test_batched_mixed_tc2_first_pass(env):
    """TC2 first pass (mode 2) on instances within its reach (kappa(A^{1/2} Z) <= 1e2), ragged m and n,
    m spanning one to several 256-column chunks and 128-row tiles."""
    torch, oqr, ctx = env
    As, Zs, _ = inputs.batch_instances(24, seed=11, device="cuda", m_range=(64, 1300), n_range=(1, 64),
                                       log_kappa_a=(0.0, 2.0), log_kappa_z=(0.0, 1.0))
    Qs, Rs, st = ctx.oqr_batched(As, Zs, mode=2)
    torch.cuda.synchronize()
    assert st.abs().sum().item() == 0
    for b in range(len(Zs)):
        check_instance(As[b].cpu().numpy(), Zs[b].cpu().numpy(), Qs[b].cpu().numpy(), Rs[b].cpu().numpy(), 0)


def test_batched_mixed_instances_independent(env):
    """An instance's (Q, R) are bit-identical whether it runs alone or packed with others, with the four
    programs (1 to 3 passes, TC2 or FP64_TC first, shifted first pass) mixed in one wave."""
    torch, oqr, ctx = env
    As, Zs, _ = inputs.batch_instances(9, seed=17, device="cuda", m_range=(64, 900), n_range=(1, 64),
                                       log_kappa_a=(0.0, 2.0), log_kappa_z=(0.0, 1.0))
    progs = (oqr.OQR_BATCH_CHOLQR2_TC, oqr.OQR_BATCH_CHOLQR2_TC2, oqr.OQR_BATCH_SCHOLQR3_TC, oqr.OQR_BATCH_CHOLQR_TC)
    fp = [progs[b % 4] for b in range(len(Zs))]
    Qs, Rs, st = ctx.oqr_batched_mixed(As, Zs, program=fp)
    torch.cuda.synchronize()
    assert st.abs().sum().item() == 0
    for b in (0, 1, 2, 3, 4, 8):
        Q1, R1, s1 = ctx.oqr_batched_mixed([As[b]], [Zs[b]], program=[fp[b]])
        torch.cuda.synchronize()
        assert s1.item() == 0
        assert torch.equal(Q1[0], Qs[b]) and torch.equal(R1[0], Rs[b])


def test_batched_mixed_breakdown_is_isolated(env):
    torch, oqr, ctx = env
    As, Zs, _ = inputs.batch_instances(6, seed=5, device="cuda", m_range=(64, 300), n_range=(4, 40),
                                       log_kappa_z=(0.0, 2.0))
    bad = torch.eye(100, dtype=torch.float64, device="cuda")
    bad[7, 7] = -1.0                             # indefinite: breaks at column 8 for Z = I[:, :10]
    As.insert(2, oqr.colmajor(bad))
    Zs.insert(2, oqr.colmajor(torch.eye(100, 10, dtype=torch.float64, device="cuda")))
    Qs, Rs, st = ctx.oqr_batched(As, Zs, mode=1)
    torch.cuda.synchronize()
    st = st.cpu().numpy()
    assert st[2] == 8
    for b in range(len(Zs)):
        if b != 2:
            check_instance(As[b].cpu().numpy(), Zs[b].cpu().numpy(), Qs[b].cpu().numpy(), Rs[b].cpu().numpy(), st[b])


def test_batched_mixed_graph_replay_same_result(env):
    torch, oqr, ctx = env
    As, Zs, _ = inputs.batch_instances(10, seed=13, device="cuda", m_range=(64, 400), n_range=(4, 64),
                                       log_kappa_z=(0.0, 2.0))
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        _, R1, st1 = ctx.oqr_batched(As, Zs, mode=1, stream=s)
        _, R2, st2 = ctx.oqr_batched(As, Zs, mode=1, stream=s)     # replays the cached graph
    torch.cuda.synchronize()
    assert st1.abs().sum().item() == 0 and torch.equal(st1, st2)
    for a, b in zip(R1, R2):
        assert torch.equal(a, b)


def test_batched_mixed_rejects_bad_program(env):
    torch, oqr, ctx = env
    As, Zs, _ = inputs.batch_instances(2, seed=1, device="cuda", m_range=(64, 128), n_range=(4, 8))
    with pytest.raises(oqr.OqrError):
        ctx.oqr_batched_mixed(As, Zs, program=[oqr.OQR_BATCH_CHOLQR2_TC, 4])


def test_batched_one_pass_matches_oracle(env):
    """One FP64_TC pass (Algorithm 1): R within the one-pass bound, T2.1's kappa^2 u growth of the
    orthogonality (reading: kappa(A^{1/2} Z) <= 1e3)."""
    torch, oqr, ctx = env
    As, Zs, _ = inputs.batch_instances(12, seed=21, device="cuda", m_range=(64, 900), n_range=(1, 64),
                                       log_kappa_a=(0.0, 2.0), log_kappa_z=(0.0, 1.0))
    Qs, Rs, st = ctx.oqr_batched_mixed(As, Zs, program=[oqr.OQR_BATCH_CHOLQR_TC] * len(Zs))
    torch.cuda.synchronize()
    assert st.abs().sum().item() == 0
    for b in range(len(Zs)):
        A, Z, Q, R = (x.cpu().numpy() for x in (As[b], Zs[b], Qs[b], Rs[b]))
        Qr, Rr = oracle.oblique_qr(A, Z)
        kap = np.linalg.cond(Rr)
        assert np.all(np.tril(R, -1) == 0) and np.all(np.diag(R) > 0)
        assert np.linalg.norm(R - Rr) / np.linalg.norm(Rr) <= max(1e-13, 50 * U * kap * kap)
        assert oracle.orth_error(A, Q) <= max(1e-13, 100 * U * kap * kap * np.linalg.eigvalsh(A).max())


def test_batched_shifted_reaches_ill_conditioned(env):
    """Shifted A-CholQR3 on the tensor cores (mode 3) completes where A-CholQR2 breaks down:
    kappa(A^{1/2} Z) up to ~1e11, orthogonality at the oracle's level, Z = QR."""
    torch, oqr, ctx = env
    As, Zs, tab = inputs.batch_instances(10, seed=31, device="cuda", m_range=(200, 1200), n_range=(8, 64),
                                         log_kappa_a=(2.0, 4.0), log_kappa_z=(8.0, 9.0))
    _, _, st2 = ctx.oqr_batched(As, Zs, mode=1)
    Qs, Rs, st = ctx.oqr_batched(As, Zs, mode=3)
    torch.cuda.synchronize()
    assert st2.ne(0).sum().item() > 0          # beyond A-CholQR2's reach on some instances
    assert st.abs().sum().item() == 0
    for b in range(len(Zs)):
        A, Z, Q, R = (x.cpu().numpy() for x in (As[b], Zs[b], Qs[b], Rs[b]))
        Qr, _ = oracle.oblique_qr(A, Z)
        floor = 100 * U * np.linalg.eigvalsh(A).max() * np.linalg.norm(Qr, 2) ** 2
        assert oracle.orth_error(A, Q) <= max(1e-12, 10 * oracle.orth_error(A, Qr), floor)
        assert np.linalg.norm(Z - Q @ R, 2) / np.linalg.norm(Z, 2) <= 1e-13
        assert np.all(np.tril(R, -1) == 0) and np.all(np.diag(R) > 0)


def test_batched_check_estimates_orthogonality(env):
    """check=True: orth[b] estimates ||Q_b^T A_b Q_b - I||_2 from an FP64-accurate Gram of the final Q
    (power iteration, a lower bound); +inf after a breakdown."""
    torch, oqr, ctx = env
    As, Zs, _ = inputs.batch_instances(10, seed=41, device="cuda", m_range=(64, 700), n_range=(2, 64),
                                       log_kappa_a=(0.0, 2.0), log_kappa_z=(3.0, 4.0))
    bad = torch.eye(100, dtype=torch.float64, device="cuda")
    bad[7, 7] = -1.0
    As.append(oqr.colmajor(bad))
    Zs.append(oqr.colmajor(torch.eye(100, 10, dtype=torch.float64, device="cuda")))
    progs = [oqr.OQR_BATCH_CHOLQR_TC, oqr.OQR_BATCH_CHOLQR2_TC] * 5 + [oqr.OQR_BATCH_CHOLQR2_TC]
    Qs, Rs, st, orth = ctx.oqr_batched_mixed(As, Zs, program=progs, check=True)
    torch.cuda.synchronize()
    st, orth = st.cpu().numpy(), orth.cpu().numpy()
    assert st[-1] == 8 and np.isinf(orth[-1])
    for b in range(len(Zs) - 1):
        assert st[b] == 0
        A = As[b].cpu().numpy()
        ref = oracle.orth_error(A, Qs[b].cpu().numpy())
        # the check's own Gram rounds at about sqrt(m) u ||A|| ||Q||^2 (here ||Q||_2 <= 1: smallest eigenvalue 1)
        slack = 2 * np.sqrt(A.shape[0]) * U * np.linalg.eigvalsh(A).max()
        assert orth[b] <= 1.05 * ref + slack
        assert orth[b] >= 0.2 * ref - slack
        if b % 2 == 0:                     # one pass: kappa^2 u, well above the rounding level
            assert ref > 10 * slack and 0.9 * ref <= orth[b] <= 1.05 * ref


def test_batched_check_graph_replay_new_outputs(env):
    """A replay of the cached graph writes this call's status and orth arrays, not the first call's."""
    torch, oqr, ctx = env
    As, Zs, _ = inputs.batch_instances(5, seed=61, device="cuda", m_range=(64, 300), n_range=(4, 32),
                                       log_kappa_a=(0.0, 2.0), log_kappa_z=(2.0, 3.0))
    s = torch.cuda.Stream()
    progs = [oqr.OQR_BATCH_CHOLQR_TC] * len(Zs)
    with torch.cuda.stream(s):
        _, R1, st1, o1 = ctx.oqr_batched_mixed(As, Zs, program=progs, stream=s, check=True)
        # the same status array, a new orth array (the binding allocates one per call; o1 stays alive)
        _, R2, st2, o2 = ctx.oqr_batched_mixed(As, Zs, program=progs, stream=s, check=True, status=st1)
    torch.cuda.synchronize()
    assert o1.data_ptr() != o2.data_ptr()
    assert st1.abs().sum().item() == 0
    assert torch.equal(o1, o2) and bool(torch.all(o2 > 0))
    for a, b in zip(R1, R2):
        assert torch.equal(a, b)


def test_batched_waves_do_not_change_results(env):
    """One wave for the whole batch, or one instance per wave (a 1 MiB plane budget): (Q, R, status,
    orth) bit-identical, with every program in the batch."""
    torch, oqr, ctx = env
    As, Zs, _ = inputs.batch_instances(12, seed=81, device="cuda", m_range=(64, 1100), n_range=(1, 64),
                                       log_kappa_a=(0.0, 2.0), log_kappa_z=(0.0, 2.0))
    progs = [(oqr.OQR_BATCH_CHOLQR_TC, oqr.OQR_BATCH_CHOLQR2_TC2, oqr.OQR_BATCH_CHOLQR2_TC,
              oqr.OQR_BATCH_SCHOLQR3_TC)[b % 4] for b in range(len(Zs))]
    Q1, R1, s1, o1 = ctx.oqr_batched_mixed(As, Zs, program=progs, check=True)
    torch.cuda.synchronize()
    try:
        ctx.set_batch_budget(1 << 20)
        Q2, R2, s2, o2 = ctx.oqr_batched_mixed(As, Zs, program=progs, check=True)
        torch.cuda.synchronize()
    finally:
        ctx.set_batch_budget(0)
    assert s1.abs().sum().item() == 0 and torch.equal(s1, s2) and torch.equal(o1, o2)
    for b in range(len(Zs)):
        assert torch.equal(Q1[b], Q2[b]) and torch.equal(R1[b], R2[b])


def test_batched_mixed_in_place(env):
    """Q aliasing Z (the factorization overwrites Z): bit-identical to the separate-output run."""
    torch, oqr, ctx = env
    As, Zs, _ = inputs.batch_instances(6, seed=91, device="cuda", m_range=(64, 600), n_range=(2, 48),
                                       log_kappa_a=(0.0, 2.0), log_kappa_z=(0.0, 2.0))
    progs = [oqr.OQR_BATCH_CHOLQR2_TC2, oqr.OQR_BATCH_SCHOLQR3_TC, oqr.OQR_BATCH_CHOLQR_TC] * 2
    Q1, R1, s1 = ctx.oqr_batched_mixed(As, Zs, program=progs)
    Zc = [oqr.colmajor(z.clone()) for z in Zs]
    Q2, R2, s2 = ctx.oqr_batched_mixed(As, Zc, program=progs, Qs=Zc)
    torch.cuda.synchronize()
    assert s1.abs().sum().item() == 0 and torch.equal(s1, s2)
    for b in range(len(Zs)):
        assert Q2[b].data_ptr() == Zc[b].data_ptr()
        assert torch.equal(Q1[b], Q2[b]) and torch.equal(R1[b], R2[b])


def test_wave_budget_autotuner(env):
    """tune_waves times every budget and leaves the fastest set; the results do not depend on it."""
    torch, oqr, ctx = env
    As, Zs, _ = inputs.batch_instances(24, seed=101, device="cuda", m_range=(64, 2000), n_range=(4, 64),
                                       log_kappa_a=(0.0, 2.0), log_kappa_z=(0.0, 2.0))
    Q0, R0, s0 = ctx.oqr_batched_mixed(As, Zs)
    torch.cuda.synchronize()
    try:
        best, timings = autotune.tune_waves(ctx, As, Zs, reps=1, budgets=(1 << 24, 1 << 27, 16 << 30))
        assert best in timings and len(timings) == 3 and all(t > 0 for t in timings.values())
        Q1, R1, s1 = ctx.oqr_batched_mixed(As, Zs)
        torch.cuda.synchronize()
    finally:
        ctx.set_batch_budget(0)
    assert torch.equal(s0, s1)
    for b in range(len(Zs)):
        assert torch.equal(Q0[b], Q1[b]) and torch.equal(R0[b], R1[b])
