"""Autotuners for the batched paths' work plans.

FP64 path:
oqr_batched cuts each instance's Gram (A_b's lower triangle, in k-steps of 16
over 64-row blocks) into `splits` ranges, one CTA each.  Too few ranges leave
SMs idle on a skewed batch; too many add partial sums and epilogues.  The tuner
groups the instances into m-buckets, times each bucket's sub-batch on the
device for a family of target k-steps per CTA, and keeps the fastest target per
bucket.  The resulting plan (splits per instance) and the table
{bucket: target} are returned; the table can be saved as JSON and reused for
batches with the same size mix.

Tensor-core path (oqr_batched_mixed): the instances run in waves whose slice
planes fit a byte budget.  A small budget gives more waves, each with fewer
work items for the persistent product kernels and a longer tail; a large one
holds more workspace.  tune_waves times a family of budgets on a sample batch
and returns the fastest (set it with Oqr.set_batch_budget); the results do not
depend on it.
"""
from __future__ import annotations

import json
import math

BUCKETS = ((1, 512), (513, 1024), (1025, 2048), (2049, 4096))
TARGETS = (64, 128, 256, 512, 1024, 2048)


def gram_steps(m: int) -> int:
    """k-steps of 16 over the 64-row blocks of an m x m lower triangle (as the kernel walks them)."""
    nb = -(-m // 64)
    return 2 * (nb - 1) * nb + -(-min(nb * 64, m) // 16)


def splits_for(m: int, target: int) -> int:
    return max(1, min(64, -(-gram_steps(m) // target)))


def plan_from_table(ms, table) -> list:
    out = []
    for m in ms:
        t = 256
        for (lo, hi), tgt in table.items():
            if lo <= m <= hi:
                t = tgt
        out.append(splits_for(m, t))
    return out


def tune(ctx, As, Zs, reps: int = 2, targets=TARGETS, buckets=BUCKETS, stream=None):
    """Times every (bucket, target) pair on the device; returns (plan, table, timings)."""
    import torch
    ms = [z.shape[0] for z in Zs]
    table, timings = {}, {}
    for (lo, hi) in buckets:
        sel = [b for b, m in enumerate(ms) if lo <= m <= hi]
        if not sel:
            continue
        sA, sZ = [As[b] for b in sel], [Zs[b] for b in sel]
        from .oqr import empty_colmajor
        Qs = [empty_colmajor(z.shape[0], z.shape[1], z.device) for z in sZ]
        Rs = [empty_colmajor(z.shape[1], z.shape[1], z.device) for z in sZ]
        best = None
        for t in targets:
            plan = [splits_for(ms[b], t) for b in sel]
            ctx.oqr_batched(sA, sZ, Qs, Rs, splits=plan, stream=stream)   # capture / warm
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                ctx.oqr_batched(sA, sZ, Qs, Rs, splits=plan, stream=stream)
            e1.record()
            torch.cuda.synchronize()
            ms_t = e0.elapsed_time(e1) / reps
            timings[f"{lo}-{hi}:{t}"] = ms_t
            if best is None or ms_t < best[1]:
                best = (t, ms_t)
        table[(lo, hi)] = best[0]
    return plan_from_table(ms, table), table, timings


def save_table(table, path):
    with open(path, "w") as f:
        json.dump({f"{lo}-{hi}": t for (lo, hi), t in table.items()}, f, indent=1)


def load_table(path):
    with open(path) as f:
        raw = json.load(f)
    return {tuple(int(x) for x in k.split("-")): v for k, v in raw.items()}


WAVE_BUDGETS = (2 << 30, 4 << 30, 8 << 30, 16 << 30, 32 << 30)


def tune_waves(ctx, As, Zs, program=None, reps: int = 2, budgets=WAVE_BUDGETS, stream=None):
    """Times oqr_batched_mixed on (As, Zs) for every plane budget; returns (best budget, {budget: ms}).
    The context's budget is left at the best one."""
    import torch
    from .oqr import empty_colmajor
    Qs = [empty_colmajor(z.shape[0], z.shape[1], z.device) for z in Zs]
    Rs = [empty_colmajor(z.shape[1], z.shape[1], z.device) for z in Zs]
    timings = {}
    for b in budgets:
        ctx.set_batch_budget(b)
        ctx.oqr_batched_mixed(As, Zs, program=program, Qs=Qs, Rs=Rs, stream=stream)   # capture / warm
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            ctx.oqr_batched_mixed(As, Zs, program=program, Qs=Qs, Rs=Rs, stream=stream)
        e1.record()
        torch.cuda.synchronize()
        timings[b] = e0.elapsed_time(e1) / reps
    best = min(timings, key=timings.get)
    ctx.set_batch_budget(best)
    return best, timings
