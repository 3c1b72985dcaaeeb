"""jacobi_precond_noalloc, the allocation-free Jacobi preconditioner, against jacobi_precond.

For callers that cannot let the library call cudaMalloc (a caching allocator that owns the free
device memory, or a loop that cannot pay for allocation and the synchronisation cudaFree implies),
jacobi_precond_noalloc computes the same G = M R with its scratch block in a static device array.
This file is collected last so that a run stopping at the first failure has run every other test.
"""
import numpy as np
import pytest

from paper_0907_3261_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12   # the relative tolerance of the Jacobi parity tests


@pytest.fixture(scope="module")
def wd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_0907_3261_gb300 as pkg
    return pkg


def rel(a, b):
    a = a.cpu().numpy()
    b = b.cpu().numpy()
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("j", [5, 4, 0])
def test_noalloc_matches_jacobi_precond_two_calls_in_a_row(wd, j):
    dims, L = (8, 8, 8, 16), 12
    links = torch.from_numpy(I.random_links(dims, 0.2, seed=0)).cuda()
    ctx = wd.wd_create(links, dims, 0.13, 1.0)
    for call, seed in enumerate((11, 12)):
        R = torch.from_numpy(I.gaussian_block(dims, L, seed=seed)).cuda()
        want = wd.jacobi_precond(ctx, R, j)
        got = torch.full_like(R, float("nan"))
        wd.jacobi_precond_noalloc(ctx, R, got, j)
        torch.cuda.synchronize()
        assert rel(got, want) <= TOL, (call, j)
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
