"""Domain-decomposed solve on the CUDA library (needs a GB300): ranks are processes sharing the one
GPU, each holding a t-slab with one halo slice on each side (wd_set_domain), with halos and rank
sums exchanged on the host over gloo -- no kernel ever waits on another rank's.

The stencils see exact neighbour values on every interior site, so the products with A and the
Jacobi sweeps reproduce the single-domain library bit for bit there; the solve differs from the
single-domain one only by the summation order of its reductions."""
import os
import socket

import numpy as np
import pytest

from oracle import operator as O
from oracle import solver as S
from paper_0907_3261_gb300 import domain as D
from paper_0907_3261_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def case_inputs(dims, L):
    return (I.random_links(dims, 0.2, seed=0), I.z4_noise(dims, L, seed=1),
            I.gaussian_block(dims, L, seed=2))


def worker(rank, world, port, case, results):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    import paper_0907_3261_gb300 as wd
    dims, L, kappa, csw, j = case
    U, B, P = case_inputs(dims, L)
    Ss = D.slice_sites(dims)
    t0, t1 = D.slab_range(dims[3], rank, world)
    mine = slice(t0 * Ss, t1 * Ss)
    ds = D.DomainSolver(wd, U[mine], dims, kappa, csw, dist, rank, world)
    Y = ds.interior(wd.wd_apply(ds.ctx, ds.extend(P[mine]))).cpu().numpy()
    G = ds.interior(wd.jacobi_precond(ds.ctx, ds.extend(P[mine]), 5)).cpu().numpy()
    X, info = ds.solve(B[mine], j=j, tol=1e-12)
    results[rank] = (t0, t1, Y, G, X.cpu().numpy(),
                     {k: info[k] for k in ("status", "iters", "max_true_resid")})
    ds.close()
    dist.barrier()
    dist.destroy_process_group()


def run(case, world):
    import torch.multiprocessing as mp
    import __graft_entry__
    __graft_entry__.build()
    port = free_port()
    # the manager's server process is started with spawn too: this process has a CUDA context
    with mp.get_context("spawn").Manager() as m:
        results = m.dict()
        mp.spawn(worker, args=(world, port, case, results), nprocs=world, join=True)
        return dict(results)


def single_domain(case):
    import paper_0907_3261_gb300 as wd
    dims, L, kappa, csw, j = case
    U, B, P = case_inputs(dims, L)
    ctx = wd.wd_create(torch.from_numpy(U).cuda(), dims, kappa, csw)
    Y = wd.wd_apply(ctx, torch.from_numpy(P).cuda()).cpu().numpy()
    G = wd.jacobi_precond(ctx, torch.from_numpy(P).cuda(), 5).cpu().numpy()
    X, info = wd.bbicggr_solve(ctx, torch.from_numpy(B).cuda(), j=j, tol=1e-12)
    X = X.cpu().numpy()
    wd.wd_destroy(ctx)
    return Y, G, X, info


def gather(res, world, idx):
    return np.concatenate([res[r][idx] for r in range(world)])


@pytest.mark.parametrize("world", [2, 3])
def test_domain_solve_8x8x8x16_L12(world):
    """8^3 x 16, L = 12, j = 12: 2 ranks (8 slices each) or 3 (6, 5, 5)."""
    case = ((8, 8, 8, 16), 12, 0.125, 1.0, 12)
    res = run(case, world)
    Y1, G1, X1, info1 = single_domain(case)
    covered = [(res[r][0], res[r][1]) for r in range(world)]
    assert covered[0][0] == 0 and covered[-1][1] == 16
    assert all(covered[r][1] == covered[r + 1][0] for r in range(world - 1))
    assert np.array_equal(gather(res, world, 2), Y1)        # A X: bit for bit
    assert np.array_equal(gather(res, world, 3), G1)        # five Jacobi sweeps: bit for bit
    X = gather(res, world, 4)
    for r in range(world):
        assert res[r][5] == res[0][5]                       # every rank decided the same
    info = res[0][5]
    assert info["status"] == 0 and abs(info["iters"] - info1["iters"]) <= 1
    dims, L, kappa, csw, j = case
    U, B, _ = case_inputs(dims, L)
    op = O.WilsonClover(U, dims, kappa, csw)
    assert S.true_residual(op, B, X).max() <= 1e-12
    assert np.linalg.norm(X - X1) / np.linalg.norm(X1) <= 1e-10


def test_domain_solve_matches_the_oracle_4x4x4x8():
    case = ((4, 4, 4, 8), 4, 0.12, 1.0, 4)
    res = run(case, 2)
    X = gather(res, 2, 4)
    dims, L, kappa, csw, j = case
    U, B, _ = case_inputs(dims, L)
    op = O.WilsonClover(U, dims, kappa, csw)
    ref = S.solve(op, B, j=j, tol=1e-12)
    assert res[0][5]["status"] == 0
    assert S.true_residual(op, B, X).max() <= 1e-12
    assert np.linalg.norm(X - ref.X) / np.linalg.norm(ref.X) <= 1e-9


def test_domain_rejects_what_it_cannot_do():
    import paper_0907_3261_gb300 as wd
    import __graft_entry__
    __graft_entry__.build()
    dims = (4, 4, 4, 8)
    U, B, _ = case_inputs(dims, 2)
    ds = D.DomainSolver(wd, U, dims, 0.12, 1.0)           # one rank: the slab wraps onto itself
    with pytest.raises(wd.WDError):                        # low-precision sweeps have no exchange
        wd.bbicggr_solve(ds.ctx, ds.extend(B), j=4, precision=4)
    with pytest.raises(wd.WDError):
        wd.jacobi_precond(ds.ctx, ds.extend(B), 3, precision=1)
    X, info = ds.solve(B, j=4)
    op = O.WilsonClover(U, dims, 0.12, 1.0)
    assert info["status"] == 0 and S.true_residual(op, B, X.cpu().numpy()).max() <= 1e-12
    ds.close()
    thin = wd.wd_create(torch.from_numpy(U[:2 * 64]).cuda(), (4, 4, 4, 2), 0.12, 1.0)
    with pytest.raises(wd.WDError):                        # no interior slice
        wd.wd_set_domain(thin, D.exchange_callback(), D.allreduce_callback())
    wd.wd_destroy(thin)
