"""The multi-GPU path of bench.py, run as two gloo ranks on the CPU: every
rank draws its own independent workload (weak scaling, nothing exchanged on
the data path), the job time is the slowest rank's, and the whole-job value
counts the voxels of all ranks."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, ws, port, out):
    import numpy as np
    import torch
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        env = bench.dist_env()
        host = bench.make_workload(rank, frames=1)
        digest = np.frombuffer(host[0, 0, 0].tobytes(), dtype=np.uint64)[:64].copy()
        ms = bench.max_over_ranks(10.0 * (rank + 1), "cpu", ws)
        seeds = [None] * ws
        dist.all_gather_object(seeds, bench.rank_seed(rank))
        digests = [None] * ws
        dist.all_gather_object(digests, digest.tolist())
        out.put((rank, env, ms, seeds, digests))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ws = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    results = [q.get(timeout=300) for _ in range(ws)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, env, ms, seeds, digests in results:
        assert env == (ws, rank, rank)
        assert ms == 10.0 * ws                      # slowest rank's time
        assert len(set(seeds)) == ws                # independent workloads
        assert digests[0] != digests[1]
    import bench
    assert bench.job_gvox_per_s(2e9, 1000.0, ws) == pytest.approx(4.0)
