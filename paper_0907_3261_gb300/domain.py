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
domain-decomposed solve.  ``DomainSolver`` wires them to the CUDA solver: each rank's library
context holds its slab plus one halo slice on each side, and the library calls back into
``exchange_callback`` before every stencil application and ``allreduce_callback`` after every Gram
product, trace and norm (wd_set_domain).  The callbacks stage through host memory and move numpy
buffers with torch.distributed point-to-point (gloo between processes; a single rank wraps onto
itself), so several ranks may share one GPU, each in its own process, with no kernel waiting on
another.
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


# tags of the two directions of a halo exchange: upward (a rank's last interior slice to the next
# rank) and downward (its first interior slice to the previous rank)
TAG_UP, TAG_DOWN = 11, 12


def exchange_callback(dist=None, rank: int = 0, world: int = 1):
    """The halo exchange of wd_set_domain over torch.distributed point-to-point on host buffers."""
    import torch

    def exchange(send_lo, send_hi, recv_lo, recv_hi):
        if dist is None or world == 1:
            recv_lo[:] = send_hi
            recv_hi[:] = send_lo
            return
        prev, nxt = (rank - 1) % world, (rank + 1) % world
        t = [torch.from_numpy(a) for a in (send_lo, send_hi, recv_lo, recv_hi)]
        reqs = [dist.isend(t[1], nxt, tag=TAG_UP), dist.isend(t[0], prev, tag=TAG_DOWN),
                dist.irecv(t[2], prev, tag=TAG_UP), dist.irecv(t[3], nxt, tag=TAG_DOWN)]
        for r in reqs:
            r.wait()
    return exchange


def allreduce_callback(dist=None):
    """The sum over ranks of wd_set_domain (in place on a float64 host buffer)."""
    import torch

    def allreduce(buf):
        if dist is not None:
            dist.all_reduce(torch.from_numpy(buf), op=dist.ReduceOp.SUM)
    return allreduce


class DomainSolver:
    """One rank's part of a domain-decomposed block BiCGGR solve on the CUDA library.

    ``links_local``: this rank's slab of links ([T*S][4][3][3], time slices slab_range(...)), host
    numpy.  The links of the extended slab come from the neighbouring ranks; the library context
    is built on the extended slab and given the domain's callbacks.  ``solve`` takes and returns
    the rank's slab of B and X."""

    def __init__(self, wd, links_local, dims, kappa: float, csw: float, dist=None, rank: int = 0,
                 world: int = 1, device=None):
        import numpy as np
        import torch
        self.wd, self.dims, self.dist, self.rank, self.world = wd, tuple(dims), dist, rank, world
        self.S = slice_sites(dims)
        self.t0, self.t1 = slab_range(dims[3], rank, world)
        ext = extend_with_halo(torch.from_numpy(np.ascontiguousarray(links_local)), dims, dist,
                               rank, world)
        self.ext_dims = (dims[0], dims[1], dims[2], self.t1 - self.t0 + 2)
        self.device = device or torch.device("cuda", torch.cuda.current_device())
        self.ctx = wd.wd_create(ext.to(self.device), self.ext_dims, kappa, csw)
        wd.wd_set_domain(self.ctx, exchange_callback(dist, rank, world), allreduce_callback(dist))

    def extend(self, block_local):
        """A block of the slab embedded in the extended slab (halo slices zero), on the device."""
        import torch
        b = torch.as_tensor(block_local)
        out = torch.zeros((b.shape[0] + 2 * self.S,) + tuple(b.shape[1:]), dtype=b.dtype)
        out[self.S:-self.S] = b.cpu()
        return out.to(self.device)

    def interior(self, block_ext):
        return block_ext[self.S:-self.S]

    def solve(self, B_local, j: int = 12, tol: float = 1e-12, **kw):
        """X of this rank's slab and the info dict (identical on every rank)."""
        B = self.extend(B_local)
        X, info = self.wd.bbicggr_solve(self.ctx, B, j=j, tol=tol, precision=0, **kw)
        return self.interior(X), info

    def close(self):
        self.wd.wd_set_domain(self.ctx, None, None)
        self.wd.wd_destroy(self.ctx)
