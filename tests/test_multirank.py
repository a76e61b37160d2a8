"""The multi-rank bench path on CPU (world size 2, gloo): every rank builds its own
independent workload (weak scaling, no collective on the data path), the job's time
is the slowest rank's, and the reported value counts every rank's points."""
import os
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, ws, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        assert bench._dist() == (ws, rank, rank)
        spec = bench.Spec("vmf_s2_50k", rank)
        # independent clouds per rank: gather a checksum of every rank's points
        cs = torch.tensor([float(np.asarray(spec.x, dtype=np.float64).sum())], dtype=torch.float64)
        allcs = [torch.zeros_like(cs) for _ in range(ws)]
        dist.all_gather(allcs, cs)
        # the slowest rank's time, and the whole-job throughput built on it
        t = bench.max_over_ranks(1.0 + rank, ws, torch.device("cpu"))
        v = bench.job_throughput(spec.n, 10, ws, t)
        out[rank] = (float(allcs[0]), float(allcs[1]), t, v, spec.n)
    finally:
        dist.destroy_process_group()


def test_two_ranks_weak_scaling():
    port = 29500 + (os.getpid() % 2000)
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        r0, r1 = out[0], out[1]
    assert r0[0] != r0[1]                       # the ranks' clouds differ
    assert r0[:2] == r1[:2]                     # and both ranks saw the same gather
    assert r0[2] == r1[2] == 2.0                # max over ranks of 1.0 and 2.0
    n = r0[4]
    assert r0[3] == pytest.approx(n * 10 * 2 / 2.0)
