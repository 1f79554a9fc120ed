"""The N > 1 path of bench.py on CPU ranks (gloo, world size 2): every rank
factors its own instance (replicas, no data-path collective), the job's time
is the maximum over ranks, and the value is the units of all ranks over that
time.  Each rank factors its (small) instance with the oracle, so the test
also checks that the ranks' instances are distinct and independent."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    from paper_1401_5171_gb300 import inputs
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sa, sz = bench.instance_seeds(rank)
        A, _ = inputs.dense_spd(64, 1e2, seed=sa)
        Z = inputs.tall_z(64, 8, 1e1, seed=sz)
        A, Z = A.numpy(), Z.numpy()
        _, R = oracle.oblique_qr(A, Z)
        ms = 10.0 * (rank + 1)                      # this rank's time
        job = bench.max_over_ranks(ms, world, dist, "cpu")
        rate = bench.whole_job_rate(world, 3, job)
        np.save(os.path.join(out, f"r{rank}.npy"), np.concatenate([[job, rate], R.ravel()]))
    finally:
        dist.destroy_process_group()


def test_two_ranks_replicas(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    port = 29500 + (os.getpid() % 2000)
    mp.start_processes(_rank, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    r0, r1 = (np.load(tmp_path / f"r{k}.npy") for k in (0, 1))
    assert r0[0] == r1[0] == 20.0                   # max over ranks
    assert r0[1] == pytest.approx(2 * 3 / 0.020)    # all ranks' units over the job's time
    assert not np.allclose(r0[2:], r1[2:])          # distinct instances per rank


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.whole_job_rate(1, 5, 250.0) == pytest.approx(20.0)
    assert bench.instance_seeds(0) != bench.instance_seeds(1)
