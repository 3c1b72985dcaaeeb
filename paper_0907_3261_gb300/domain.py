"""Lattice domain decomposition across ranks: the host-side exchanges of a multi-GPU solve.

Block BiCGGR shards by lattice domain, not by right-hand side: the L x L Gram matrices couple all
L columns, so every rank holds all L columns of its part of the lattice.  The lattice is cut into
slabs along t, rank r owning the time slices [t0, t1) of ``slab_range``.  Because the site index is
x + Lx(y + Ly(z + Lz t)), a slab is a contiguous range of sites, and one time slice of any field
([V][...] layout) is a contiguous block of Lx*Ly*Lz sites.

Per stencil application a rank needs one neighbouring time slice on each side: the spinor halo
for the hopping term, and once per configuration the link halo for the clover leaves, which reach
one slice forward and back.  ``extend_with_halo`` exchanges them with the two neighbouring ranks
(torch.distributed point-to-point, on whatever device the tensors live: NCCL between GPUs, gloo
between CPU processes; a single rank wraps periodically by itself).  Per outer iteration the Gram
products R~_0^H V, R~_0^H R, the traces Tr[W^H R], Tr[W^H W] and the column norms are sums over all
sites; ``allreduce_sum`` completes them.  These two operations are the whole communication of a
domain-decomposed solve.  They are not wired to the CUDA solver in this library (every GPU
process here owns one GPU and the full lattice); they carry the exchange logic that a multi-GPU
solver needs and are tested with CPU ranks.
"""
from __future__ import annotations


def slab_range(Lt: int, rank: int, world: int):
    """Time slices [t0, t1) of ``rank``: an even split, the first Lt % world ranks one slice more."""
    if world < 1 or not 0 <= rank < world or Lt < world:
        raise ValueError("need 0 <= rank < world <= Lt")
    base, extra = divmod(Lt, world)
    t0 = rank * base + min(rank, extra)
    return t0, t0 + base + (1 if rank < extra else 0)


def slice_sites(dims) -> int:
    """Sites in one time slice, Lx*Ly*Lz."""
    return int(dims[0]) * int(dims[1]) * int(dims[2])


def extend_with_halo(local, dims, dist=None, rank: int = 0, world: int = 1):
    """[T_local * S, ...] -> [(T_local + 2) * S, ...]: the slab with the last time slice of the
    previous rank in front and the first time slice of the next rank behind (periodic in t)."""
    import torch
    S = slice_sites(dims)
    first, last = local[:S], local[-S:]
    if dist is None or world == 1:
        return torch.cat([last, local, first], dim=0)
    prev, nxt = (rank - 1) % world, (rank + 1) % world
    from_prev = torch.empty_like(last)
    from_next = torch.empty_like(first)
    ops = [dist.P2POp(dist.isend, last.contiguous(), nxt),
           dist.P2POp(dist.isend, first.contiguous(), prev),
           dist.P2POp(dist.irecv, from_prev, prev),
           dist.P2POp(dist.irecv, from_next, nxt)]
    for req in dist.batch_isend_irecv(ops):
        req.wait()
    return torch.cat([from_prev, local, from_next], dim=0)


def allreduce_sum(t, dist=None):
    """Sum of ``t`` over all ranks (in place; returns it)."""
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t
