"""Host logic of the batched selector (selector.solve_batch) with a scripted
context on the CPU: which program runs for which choice, which results are
accepted, and what the fallback chain keeps.  No GPU: the fake context returns
scripted statuses and orthogonalities and marks every result with the program
that produced it."""
import math

import pytest

torch = pytest.importorskip("torch")

from paper_1401_5171_gb300 import selector  # noqa: E402

FP64 = "fp64"


class FakeCtx:
    """outcome[b][program] = (status, orth); program is an OQR_BATCH_* value or FP64."""

    def __init__(self, choices, outcome):
        self.choices = choices
        self.outcome = outcome
        self.calls = []

    def oqr_features(self, A, Z, out=None, stream=None):
        out.zero_()

    def oqr_mlp_forward(self, X, P, bf16=True, want_logits=False):
        return None, torch.tensor(self.choices, dtype=torch.int32)

    def _run(self, idx, programs, Qs, Rs):
        st, orth = [], []
        for k, b in enumerate(idx):
            s, o = self.outcome[b][programs[k]]
            Qs[k].fill_(mark(programs[k]))                # marks which program produced the result
            st.append(s)
            orth.append(o)
        return torch.tensor(st, dtype=torch.int32), torch.tensor(orth, dtype=torch.float64)

    def oqr_batched_mixed(self, As, Zs, program=None, Qs=None, Rs=None, stream=None, status=None, check=False):
        idx = [self.index[id(z)] for z in Zs]
        self.calls.append(("tc", idx, list(program)))
        st, orth = self._run(idx, list(program), Qs, Rs)
        return Qs, Rs, st, orth

    def oqr_batched(self, As, Zs, Qs=None, Rs=None, splits=None, stream=None, status=None, mode=0):
        idx = [self.index[id(z)] for z in Zs]
        self.calls.append(("fp64", idx, [FP64] * len(idx)))
        st, _ = self._run(idx, [FP64] * len(idx), Qs, Rs)
        return Qs, Rs, st


MARKS = {0: 10.0, 1: 11.0, 2: 12.0, 3: 13.0, FP64: 14.0}


def mark(p):
    return MARKS[p]


def run(choices, outcome):
    n = len(choices)
    As = [torch.zeros(8, 8, dtype=torch.float64) for _ in range(n)]
    Zs = [torch.zeros(8, 2, dtype=torch.float64) for _ in range(n)]
    ctx = FakeCtx(choices, outcome)
    ctx.index = {id(z): b for b, z in enumerate(Zs)}
    Qs, Rs, info = selector.solve_batch(ctx, As, Zs, P=None, tol=1e-12)
    return ctx, Qs, info


CHOL, TC2, CHOL2, SHIFT = 0, 1, 2, 3      # OQR_BATCH_* programs


def test_choices_map_to_programs_and_pass_checks():
    ok = (0, 1e-14)
    outcome = [{CHOL: ok}, {TC2: ok}, {SHIFT: ok}, {FP64: ok}]
    ctx, Qs, info = run([0, 1, 2, 3], outcome)
    assert ctx.calls[0] == ("tc", [0, 1, 2], [CHOL, TC2, SHIFT])
    assert ctx.calls[1] == ("fp64", [3], [FP64])
    assert len(ctx.calls) == 2                       # everything accepted: no fallback
    assert info["used"] == [0, 1, 2, 3] and info["status"] == [0, 0, 0, 0]
    assert [Qs[b][0, 0].item() for b in range(4)] == [mark(CHOL), mark(TC2), mark(SHIFT), mark(FP64)]


def test_failed_check_falls_back_and_keeps_the_more_orthogonal():
    outcome = [
        {CHOL: (0, 1e-9), SHIFT: (0, 1e-14)},        # option 0 misses tol: the shifted result is kept
        {TC2: (0, 1e-13)},                           # option 1 meets tol
        {TC2: (0, 1e-8), SHIFT: (0, 1e-7)},          # the fallback is worse: option 1's result stays
    ]
    ctx, Qs, info = run([0, 1, 1], outcome)
    assert ctx.calls[1] == ("tc", [0, 2], [SHIFT, SHIFT])
    assert info["used"] == [2, 1, 1]
    assert Qs[0][0, 0].item() == mark(SHIFT) and Qs[2][0, 0].item() == mark(TC2)
    assert info["orth"][0] == 1e-14 and info["orth"][2] == 1e-8


def test_breakdowns_go_down_the_whole_chain():
    outcome = [
        {TC2: (5, math.inf), SHIFT: (3, math.inf), FP64: (0, math.nan)},
        {SHIFT: (0, 1e-13)},                         # option 2 accepted once it completes
    ]
    ctx, Qs, info = run([1, 2], outcome)
    assert [c[0] for c in ctx.calls] == ["tc", "tc", "fp64"]
    assert ctx.calls[1] == ("tc", [0], [SHIFT]) and ctx.calls[2] == ("fp64", [0], [FP64])
    assert info["status"] == [0, 0] and info["used"] == [3, 2]
    assert Qs[0][0, 0].item() == mark(FP64)


def test_nothing_completes():
    outcome = [{CHOL: (2, math.inf), SHIFT: (2, math.inf), FP64: (2, math.nan)}]
    ctx, Qs, info = run([0], outcome)
    assert info["status"] == [1] and info["used"] == [None]
