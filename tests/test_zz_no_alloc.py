"""jacobi_precond_noalloc, the allocation-free Jacobi preconditioner, against jacobi_precond.

For callers that cannot let the library call cudaMalloc (a caching allocator that owns the free
device memory, or a loop that cannot pay for allocation and the synchronisation cudaFree implies),
jacobi_precond_noalloc computes the same G = M R with its scratch block in a static device array.
Both entry points launch the same FP64 kernels on the same inputs in the same order, so their
results are compared bit for bit.  The allocation-free calls come first on a fresh context, before
jacobi_precond has allocated the context's workspace.
This file is collected last so that a run stopping at the first failure has run every other test.
"""
import numpy as np
import pytest

from paper_0907_3261_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_0907_3261_gb300 as pkg
    return pkg


@pytest.mark.parametrize("js", [(5, 4), (4, 5), (0, 1)])
def test_noalloc_first_on_a_fresh_context_two_calls_in_a_row(wd, js):
    dims, L = (8, 8, 8, 16), 12
    links = torch.from_numpy(I.random_links(dims, 0.2, seed=0)).cuda()
    ctx = wd.wd_create(links, dims, 0.13, 1.0)
    Rs = [torch.from_numpy(I.gaussian_block(dims, L, seed=s)).cuda() for s in (11, 12)]
    got = []
    for R, j in zip(Rs, js):                  # two allocation-free calls in a row, nothing else
        G = torch.full_like(R, float("nan"))
        wd.jacobi_precond_noalloc(ctx, R, G, j)
        got.append(G)
    torch.cuda.synchronize()
    for R, j, G in zip(Rs, js, got):
        want = wd.jacobi_precond(ctx, R, j)
        torch.cuda.synchronize()
        assert torch.equal(G, want), j
    wd.wd_destroy(ctx)


def test_noalloc_after_jacobi_precond_matches_bit_for_bit(wd):
    dims, L, j = (4, 4, 4, 8), 5, 7
    links = torch.from_numpy(I.random_links(dims, 0.3, seed=1)).cuda()
    ctx = wd.wd_create(links, dims, 0.125, 1.0)
    R = torch.from_numpy(I.z4_noise(dims, L, seed=2)).cuda()
    want = wd.jacobi_precond(ctx, R, j)
    for _ in range(2):
        G = torch.full_like(R, float("nan"))
        wd.jacobi_precond_noalloc(ctx, R, G, j)
        torch.cuda.synchronize()
        assert torch.equal(G, want)
    wd.wd_destroy(ctx)


def test_noalloc_rejects_what_it_cannot_hold(wd):
    dims = (16, 16, 16, 16)              # 12 * V * L = 9.4e6 complex numbers > 2^21
    links = torch.from_numpy(I.random_links(dims, 0.2, seed=0)).cuda()
    ctx = wd.wd_create(links, dims, 0.12, 1.0)
    R = torch.zeros((int(np.prod(dims)), 4, 3, 12), dtype=torch.complex128, device="cuda")
    with pytest.raises(wd.WDError):
        wd.jacobi_precond_noalloc(ctx, R, torch.empty_like(R), 3)
    Rh = np.zeros((int(np.prod(dims)), 4, 3, 1), dtype=np.complex128)
    with pytest.raises(wd.WDError):                  # host buffers would need staging
        wd.jacobi_precond_noalloc(ctx, Rh, np.empty_like(Rh), 3)
    wd.wd_destroy(ctx)
