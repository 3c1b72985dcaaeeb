"""Domain decomposition across CPU ranks (gloo): slabs along t, one-slice halo exchange and the
Gram allreduce reproduce the global operator and the global Gram products of the oracle."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_0907_3261_gb300 import domain as D


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


DIMS = (3, 4, 2, 8)
KAPPA, CSW = 0.125, 1.3


def global_fields():
    from paper_0907_3261_gb300 import inputs as I
    U = I.random_links(DIMS, 0.5, seed=3)
    psi = I.gaussian_block(DIMS, 3, seed=4)
    Rt = I.gaussian_block(DIMS, 3, seed=5)
    return U, psi, Rt


def worker(rank, world, port, results):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import operator as O
    U, psi, Rt = global_fields()
    S = D.slice_sites(DIMS)
    t0, t1 = D.slab_range(DIMS[3], rank, world)
    sl = slice(t0 * S, t1 * S)
    U_ext = D.extend_with_halo(torch.from_numpy(U[sl].copy()), DIMS, dist, rank, world).numpy()
    p_ext = D.extend_with_halo(torch.from_numpy(psi[sl].copy()), DIMS, dist, rank, world).numpy()
    ext_dims = (DIMS[0], DIMS[1], DIMS[2], t1 - t0 + 2)
    # the periodic operator on the extended slab is exact on the interior slices: their hops and
    # clover leaves reach at most one slice out, into the halo
    Y = O.WilsonClover(U_ext, ext_dims, KAPPA, CSW).apply(p_ext)[S:-S]
    gram = torch.from_numpy(Rt[sl].reshape(-1, 3).conj().T @ psi[sl].reshape(-1, 3))
    D.allreduce_sum(gram, dist)
    results[rank] = (t0, t1, Y, gram.numpy())
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_slab_halo_exchange_and_gram_allreduce(world):
    from oracle import operator as O
    port = free_port()
    with mp.Manager() as m:
        results = m.dict()
        mp.spawn(worker, args=(world, port, results), nprocs=world, join=True)
        res = dict(results)
    U, psi, Rt = global_fields()
    Y_ref = O.WilsonClover(U, DIMS, KAPPA, CSW).apply(psi)
    S = D.slice_sites(DIMS)
    covered = 0
    for r in range(world):
        t0, t1, Y, gram = res[r]
        assert np.abs(Y - Y_ref[t0 * S:t1 * S]).max() <= 1e-14 * np.abs(Y_ref).max()
        assert np.allclose(gram, Rt.reshape(-1, 3).conj().T @ psi.reshape(-1, 3), rtol=1e-13, atol=1e-13)
        covered += t1 - t0
    assert covered == DIMS[3]


def test_single_rank_wraps_periodically():
    from oracle import operator as O
    U, psi, _ = global_fields()
    S = D.slice_sites(DIMS)
    ext = D.extend_with_halo(torch.from_numpy(psi), DIMS).numpy()
    assert np.array_equal(ext[:S], psi[-S:]) and np.array_equal(ext[-S:], psi[:S])
    assert D.slab_range(8, 0, 3) == (0, 3) and D.slab_range(8, 2, 3) == (6, 8)
    with pytest.raises(ValueError):
        D.slab_range(2, 0, 3)


def callback_worker(rank, world, port, results):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ex = D.exchange_callback(dist, rank, world)
    ar = D.allreduce_callback(dist)
    n = 40
    send_lo = np.full(n, 10 * rank + 1, dtype=np.uint8)
    send_hi = np.full(n, 10 * rank + 2, dtype=np.uint8)
    recv_lo, recv_hi = np.zeros(n, np.uint8), np.zeros(n, np.uint8)
    for _ in range(2):               # two exchanges in a row reuse the same tags
        ex(send_lo, send_hi, recv_lo, recv_hi)
    buf = np.array([float(rank), 1.0, 0.5 * rank])
    ar(buf)
    results[rank] = (recv_lo.copy(), recv_hi.copy(), buf)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_domain_callbacks_exchange_halos_and_sum(world):
    """The callbacks wd_set_domain calls: each rank receives the previous rank's last interior
    slice as its lower halo and the next rank's first as its upper halo (periodic), and the sum
    over ranks is the same on every rank."""
    port = free_port()
    with mp.Manager() as m:
        results = m.dict()
        mp.spawn(callback_worker, args=(world, port, results), nprocs=world, join=True)
        res = dict(results)
    for r in range(world):
        recv_lo, recv_hi, buf = res[r]
        prev, nxt = (r - 1) % world, (r + 1) % world
        assert (recv_lo == 10 * prev + 2).all() and (recv_hi == 10 * nxt + 1).all()
        assert np.array_equal(buf, res[0][2])
        assert buf[0] == sum(range(world)) and buf[1] == world


def test_single_rank_callbacks_wrap():
    ex, ar = D.exchange_callback(), D.allreduce_callback()
    lo, hi = np.arange(5, dtype=np.uint8), np.arange(5, 10, dtype=np.uint8)
    rl, rh = np.zeros(5, np.uint8), np.zeros(5, np.uint8)
    ex(lo, hi, rl, rh)
    assert np.array_equal(rl, hi) and np.array_equal(rh, lo)
    b = np.array([1.5, 2.0])
    ar(b)
    assert np.array_equal(b, [1.5, 2.0])
