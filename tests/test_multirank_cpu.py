"""The N > 1 path of bench.py on CPU ranks (gloo, world size 2): every rank solves its own
independent sources, timings are reduced with MAX, and the reference arm runs on rank 0 only."""
import io
import os
import socket
import contextlib

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def worker(rank, world, port, results):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_0907_3261_gb300 import inputs as I
    # max over ranks of a per-rank timing
    t = bench.max_over_ranks(0.5 + rank, dist, "cpu")
    # independent sources per rank
    B = I.z4_noise((2, 2, 2, 2), 3, seed=bench.source_seed(rank))
    import torch
    mine = torch.from_numpy(B.view(np.float64).copy())
    gathered = [torch.zeros_like(mine) for _ in range(world)]
    dist.all_gather(gathered, mine)
    differ = not torch.equal(gathered[0], gathered[1])
    # the reference arm works on rank 0 only: the other ranks return at once, printing nothing
    out = io.StringIO()
    rc = None
    if rank != 0:
        class A:
            steps, warmup, gpus = 1, 3, world
        with contextlib.redirect_stdout(out):
            rc = bench.reference_arm(A)
    results[rank] = (t, differ, rc, out.getvalue())
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    port = free_port()
    with mp.Manager() as m:
        results = m.dict()
        mp.spawn(worker, args=(2, port, results), nprocs=2, join=True)
        res = dict(results)
    assert res[0][0] == res[1][0] == 1.5
    assert res[0][1] and res[1][1]
    assert res[1][2] == 0 and res[1][3] == ""


def test_single_process_needs_no_group():
    import bench
    assert bench.max_over_ranks(2.5) == 2.5
    assert bench.source_seed(0) != bench.source_seed(1)
