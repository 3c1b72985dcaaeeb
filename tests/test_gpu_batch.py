"""Batched solves in one CUDA graph with device-side iteration control (needs a GB300)."""
import numpy as np
import pytest

from oracle import operator as O
from oracle import solver as S
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


CASES = [((4, 4, 4, 4), 4, 0.115, 4, 0), ((3, 4, 5, 6), 3, 0.12, 2, 0),
         ((8, 8, 8, 16), 12, 0.13, 12, 1), ((4, 4, 4, 8), 1, 0.12, 3, 1), ((2, 2, 2, 2), 12, 0.115, 0, 0),
         ((4, 4, 4, 8), 6, 0.115, 4, 3), ((4, 4, 4, 4), 5, 0.12, 6, 4)]


def test_batch_matches_host_controlled_solves(wd):
    jobs, refs, ops = [], [], []
    for n, (dims, L, kappa, j, prec) in enumerate(CASES):
        links = I.random_links(dims, 0.3, seed=n)
        ctx = wd.wd_create(dev(links), dims, kappa, 1.0)
        B = dev(I.z4_noise(dims, L, seed=10 + n))
        Xr, ir = wd.bbicggr_solve(ctx, B, j=j, tol=1e-12, precision=prec, history=500)
        refs.append((host(Xr), ir))
        ops.append((O.WilsonClover(links, dims, kappa, 1.0), host(B)))
        jobs.append(dict(ctx=ctx, B=B, X=torch.zeros_like(B), j=j, precision=prec, history=500))
    infos = wd.bbicggr_solve_batch(jobs)
    for jb, info, (Xr, ir), (op, Bh) in zip(jobs, infos, refs, ops):
        assert info["status"] == wd.WD_OK
        assert info["iters"] == ir["iters"]
        X = host(jb["X"])
        assert np.linalg.norm(X - Xr) <= 1e-13 * np.linalg.norm(Xr)
        assert S.true_residual(op, Bh, X).max() <= 1e-12
        assert np.allclose(info["history"], ir["history"], rtol=1e-12, atol=0)
        assert info["mvm_paper"] == ir["mvm_paper"]


def test_batch_statuses(wd):
    dims = (2, 2, 2, 4)
    links = dev(I.random_links(dims, 0.3, seed=0))
    B = I.z4_noise(dims, 2, seed=1)
    c1 = wd.wd_create(links, dims, 0.115, 1.0)
    c2 = wd.wd_create(links, dims, 0.115, 1.0)
    B2 = B.copy()
    B2[..., 1] = B2[..., 0]                    # singular R~_0^H V_0
    jobs = [dict(ctx=c1, B=dev(B), X=torch.zeros_like(dev(B)), j=1, maxit=2),
            dict(ctx=c2, B=dev(B2), X=torch.zeros_like(dev(B2)), j=1)]
    infos = wd.bbicggr_solve_batch(jobs)
    assert infos[0]["status"] == wd.WD_NOT_CONVERGED and infos[0]["iters"] == 2
    assert infos[1]["status"] == wd.WD_BREAKDOWN and infos[1]["iters"] == 0
    with pytest.raises(wd.WDError):
        wd.bbicggr_solve_batch([jobs[0], dict(jobs[0])])     # two jobs on one context
