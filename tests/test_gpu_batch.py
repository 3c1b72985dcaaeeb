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


def run_pair(wd, dims, L, kappa, j, seed, **kw):
    """A job and the same solve under host control on the job's context, so that both use the
    tiles its autotuner picked: (job, host info, host X)."""
    links = dev(I.random_links(dims, 0.2, seed=seed))
    B = dev(I.z4_noise(dims, L, seed=50 + seed))
    ctx = wd.wd_create(links, dims, kappa, 1.0)
    Xr, ir = wd.bbicggr_solve(ctx, B, j=j, history=2000, **kw)
    job = dict(ctx=ctx, B=B, X=torch.zeros_like(B), j=j, history=2000, **kw)
    return job, ir, host(Xr)


def test_batch_falls_back_and_restarts_like_the_host_controlled_solve(wd):
    """The pass loop of the graph makes the decisions of bbicggr_solve on the device: a stalled
    low-precision run starts over from X_0 with the FP64 preconditioner, a network that cannot
    serve as M falls back the same way, and a true residual above tol restarts from X."""
    cases = [
        # FP32 sweeps near the critical kappa with a short stall window: falls back
        dict(dims=(6, 6, 6, 6), L=4, kappa=0.134, j=4, seed=0,
             kw=dict(precision=1, stall_window=2, maxit=2000)),
        # a network with large random weights as M: stalls or diverges, then FP64 Jacobi
        dict(dims=(4, 4, 4, 4), L=3, kappa=0.12, j=3, seed=1,
             kw=dict(stall_window=4, maxit=400, net="random")),
        # a tolerance below what the recursion can certify: true-residual restarts
        dict(dims=(4, 4, 4, 4), L=2, kappa=0.115, j=2, seed=2,
             kw=dict(tol=1e-17, maxit=300, max_restarts=2)),
        # the double-float preconditioner, no fallback needed
        dict(dims=(6, 6, 6, 6), L=4, kappa=0.134, j=4, seed=0, kw=dict(precision=5, maxit=2000)),
    ]
    jobs, refs = [], []
    for cs in cases:
        kw = dict(cs["kw"])
        if kw.get("net") == "random":
            kw["net"] = wd.wd_net_create(4, 4, I.network_weights(4, 4, seed=11, noise=0.5))
        job, ir, Xr = run_pair(wd, cs["dims"], cs["L"], cs["kappa"], cs["j"], cs["seed"], **kw)
        jobs.append(job)
        refs.append((ir, Xr))
    infos = wd.bbicggr_solve_batch(jobs)
    assert any(ir["fallbacks"] for ir, _ in refs) and any(ir["restarts"] for ir, _ in refs)
    for jb, info, (ir, Xr) in zip(jobs, infos, refs):
        for key in ("status", "iters", "restarts", "fallbacks", "mvm_paper"):
            assert info[key] == ir[key], (key, info[key], ir[key])
        X = host(jb["X"])
        assert np.linalg.norm(X - Xr) <= 1e-13 * np.linalg.norm(Xr)
        assert len(info["history"]) == len(ir["history"])
        assert np.allclose(info["history"], ir["history"], rtol=1e-12, atol=0)
        assert np.allclose(info["true_resid"], ir["true_resid"], rtol=1e-10, atol=0)


def test_batch_jobs_share_one_network(wd):
    """Several jobs of one graph run the same network at the same time on different lattices and
    L: each context has its own activations, so every job reproduces its host-controlled solve."""
    net = wd.wd_net_create(4, 4, I.network_weights(4, 4, seed=7, noise=0.01))
    jobs, refs = [], []
    for n, (dims, L) in enumerate([((4, 4, 4, 4), 1), ((4, 4, 4, 4), 3), ((4, 4, 4, 8), 2)]):
        job, ir, Xr = run_pair(wd, dims, L, 0.115, 4, 20 + n, net=net, maxit=500)
        jobs.append(job)
        refs.append((ir, Xr))
    infos = wd.bbicggr_solve_batch(jobs)
    for jb, info, (ir, Xr) in zip(jobs, infos, refs):
        assert info["status"] == ir["status"] == wd.WD_OK
        for key in ("iters", "fallbacks", "mvm_paper"):
            assert info[key] == ir[key], (key, info[key], ir[key])
        assert np.linalg.norm(host(jb["X"]) - Xr) <= 1e-13 * np.linalg.norm(Xr)
