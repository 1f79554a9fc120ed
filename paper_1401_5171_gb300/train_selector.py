"""Trains the selector's network on method-generated instances and writes selector_weights.json.

    python -m paper_1401_5171_gb300.train_selector [--count 100000] [--epochs 60] [--out PATH]

The training set is the selector's workload at small sizes (m uniform in [64, 1024], n in [4, 64],
kappa(A) log-uniform to 1e6, kappa(Z) log-uniform to 1e12): features from the first FP64-accurate pass
(oqr_batched_features), labels from the three tensor-core options run with their check (the cheapest that
reaches ||Q^T A Q - I||_2 <= 1e-12).  Training and inference use the library's MLP kernels.  A held-out
set at the batched workload's sizes (m up to 4096) measures the accuracy.  Runs on one GPU.
"""
from __future__ import annotations

import argparse
import json
import sys
import time


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--count", type=int, default=100000)
    p.add_argument("--heldout", type=int, default=2048)
    p.add_argument("--epochs", type=int, default=60)
    p.add_argument("--seed", type=int, default=7)
    p.add_argument("--out", default=None)
    a = p.parse_args(argv)
    import numpy as np
    import torch

    from . import build, oqr, selector
    build.build()
    ctx = oqr.Oqr(0)
    t0 = time.time()
    tr = selector.make_set(ctx, a.count, seed=a.seed, batch_size=2048)
    t1 = time.time()
    P, losses = selector.train(ctx, tr["X"], tr["y"], epochs=a.epochs, seed=a.seed)
    t2 = time.time()
    ho = selector.make_set(ctx, a.heldout, seed=a.seed + 1, batch_size=512, m_range=(64, 4096))
    pred = selector.choose(ctx, ho["X"], P).cpu().numpy()
    lab = ho["y"].cpu().numpy()
    mix = np.bincount(tr["y"].cpu().numpy(), minlength=selector.CLASSES).tolist()
    meta = {"train_count": a.count, "train_sizes": "m 64..1024, n 4..64", "kappa_A": "log-uniform 1..1e6",
            "kappa_Z": "log-uniform 1..1e12", "epochs": a.epochs, "label_mix": mix,
            "loss_first": losses[0], "loss_last": losses[-1],
            "heldout_count": a.heldout, "heldout_sizes": "m 64..4096, n 4..64",
            "heldout_accuracy": float(np.mean(pred == lab)),
            "heldout_unsafe_rate": float(np.mean(pred < lab)),   # chose a cheaper option than the label
            "seconds": {"labels": t1 - t0, "train": t2 - t1}}
    selector.save(P, a.out or selector.WEIGHTS, meta)
    print(json.dumps(meta), flush=True)
    ctx.close()


if __name__ == "__main__":
    sys.exit(main())
