"""Learned preconditioner network on the GPU vs the FP64 oracle (needs a GB300)."""
import numpy as np
import pytest

from oracle import network as N
from oracle import operator as O
from oracle import solver as S
from paper_0907_3261_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# FP32 activations and complex64 weights: each layer sums 9 x C_in x 4 products per output
# component, so a 4-layer network carries ~4 x 150 roundings of 2^-24 relative (~4e-5 worst case).
NET_TOL = 1e-4
GRAD_TOL = 1e-3      # gradients are differences of FP32 activations summed over the lattice


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


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


def case(dims=(3, 4, 5, 6), L=3, layers=4, hidden=4, noise=0.3):
    U = I.random_links(dims, 0.4, seed=1)
    W = I.network_weights(layers, hidden, seed=2, noise=noise)
    # complex64 weights on the GPU: give the oracle the same rounded weights
    W = [w.astype(np.complex64).astype(np.complex128) for w in W]
    R = I.gaussian_block(dims, L, seed=3)
    E = I.gaussian_block(dims, L, seed=4)
    return dims, U, W, R, E


@pytest.mark.parametrize("layers,hidden", [(4, 4), (3, 2), (1, 1)])
def test_net_forward_matches_oracle(wd, layers, hidden):
    dims, U, W, R, _ = case(layers=layers, hidden=hidden)
    ctx = wd.wd_create(dev(U), dims, 0.13, 1.0)
    net = wd.wd_net_create(layers, hidden, W)
    G = host(wd.wd_net_apply(ctx, net, dev(R)))
    Y = N.forward(U, O.Lattice(dims), W, R)[0]
    assert rel(G, Y) <= NET_TOL
    assert all(np.array_equal(a, b) for a, b in zip(wd.wd_net_get_weights(net), W))


def test_net_full_size_columns_element_wise(wd):
    """The bench lattice in the launch shape bench.py --workload net16 times (16^3 x 32, L = 12,
    4 layers, 4 hidden channels): columns 0 and 11 of the GPU's N(R) against the oracle run on
    each column alone, element by element relative to the column's largest entry."""
    dims, L = (16, 16, 16, 32), 12
    U = I.random_links(dims, 0.2, seed=0)
    W = [w.astype(np.complex64).astype(np.complex128)
         for w in I.network_weights(4, 4, seed=0, noise=0.1)]
    R = I.z4_noise(dims, L, seed=1)
    ctx = wd.wd_create(dev(U), dims, 0.134, 1.0)
    net = wd.wd_net_create(4, 4, W)
    G = host(wd.wd_net_apply(ctx, net, dev(R)))
    lat = O.Lattice(dims)
    for r in (0, L - 1):
        Y = N.forward(U, lat, W, np.ascontiguousarray(R[..., r:r + 1]))[0][..., 0]
        assert np.abs(G[..., r] - Y).max() <= NET_TOL * np.abs(Y).max()


@pytest.mark.parametrize("layers,hidden", [(4, 4), (3, 2)])
def test_net_forward_bf16_activations(wd, layers, hidden):
    """BF16-stored activations (inference): the input and every layer's output are rounded to
    BF16 once (relative 2^-8 per component).  With the near-identity weights the training starts
    from, each layer has norm ~1, so the layers + 1 roundings add up to at most (layers + 1) 2^-8."""
    dims, U, _, R, _ = case(layers=layers, hidden=hidden)
    W = [w.astype(np.complex64).astype(np.complex128)
         for w in I.network_weights(layers, hidden, seed=2, noise=0.01)]
    ctx = wd.wd_create(dev(U), dims, 0.13, 1.0)
    net = wd.wd_net_create(layers, hidden, W)
    Y = N.forward(U, O.Lattice(dims), W, R)[0]
    G16 = host(wd.wd_net_apply(ctx, net, dev(R), bf16=True))
    G32 = host(wd.wd_net_apply(ctx, net, dev(R)))
    err = rel(G16, Y)
    assert err <= (layers + 1) * 2.0 ** -8
    assert err > 10 * rel(G32, Y)            # the activations really are BF16


def test_net_bf16_preconditioned_solve(wd):
    """precision 3 with a network: BF16 activations inside block BiCGGR still reach the FP64
    answer (through the FP64-Jacobi fallback if the network stalls the method)."""
    dims, L = (4, 4, 4, 4), 4
    U = I.random_links(dims, 0.3, seed=0)
    op = O.WilsonClover(U, dims, 0.115, 1.0)
    B = I.z4_noise(dims, L, seed=1)
    ctx = wd.wd_create(dev(U), dims, 0.115, 1.0)
    net = wd.wd_net_create(4, 4, I.network_weights(4, 4, seed=7, noise=0.01))
    X, info = wd.bbicggr_solve(ctx, dev(B), j=4, tol=1e-12, net=net, precision=3)
    assert info["status"] == wd.WD_OK and info["fallbacks"] in (0, 1)
    assert S.true_residual(op, B, host(X)).max() <= 1e-12
    assert rel(host(X), S.solve(op, B, j=4, tol=1e-12).X) <= 1e-9


def test_net_loss_gradient_and_adam_match_oracle(wd):
    dims, U, W, R, E = case(dims=(4, 4, 2, 4), L=2)
    ctx = wd.wd_create(dev(U), dims, 0.13, 1.0)
    net = wd.wd_net_create(4, 4, W)
    loss, grads = wd.wd_net_loss_grad(ctx, net, dev(R), dev(E))
    lat = O.Lattice(dims)
    loss_ref, grads_ref = N.loss_and_grad(U, lat, W, R, E)
    assert abs(loss - loss_ref) <= NET_TOL * loss_ref
    for g, gr in zip(grads, grads_ref):
        assert rel(g, gr) <= GRAD_TOL
    wd.wd_net_adam_step(net, 1e-3)
    W1 = wd.wd_net_get_weights(net)
    W1_ref = N.adam_step(W, grads_ref, {}, 1e-3)
    gmax = max(np.abs(g).max() for g in grads_ref)
    for a, b, w, g in zip(W1, W1_ref, W, grads_ref):
        # the first Adam step moves each real parameter by lr * g / |g|; compare it wherever the
        # gradient is clearly above the FP32 noise of the GPU gradient (elsewhere its sign is noise)
        for part in (np.real, np.imag):
            big = np.abs(part(g)) > 1e-2 * gmax
            assert big.sum() > 0
            assert np.max(np.abs(part(a - w)[big] - part(b - w)[big])) <= 1e-5


def test_net_is_gauge_covariant_on_gpu(wd):
    dims, U, W, R, _ = case(dims=(4, 2, 3, 4))
    lat = O.Lattice(dims)
    Om = I.random_gauge_transform(dims, seed=9)
    Up = np.empty_like(U)
    for mu in range(4):
        Up[:, mu] = Om @ U[:, mu] @ np.conj(np.swapaxes(Om[lat.fwd[mu]], -1, -2))
    rot = lambda z: np.einsum("vab,vsbl->vsal", Om, z)
    net = wd.wd_net_create(4, 4, W)
    a = host(wd.wd_net_apply(wd.wd_create(dev(Up), dims, 0.13, 1.0), net, dev(rot(R))))
    b = rot(host(wd.wd_net_apply(wd.wd_create(dev(U), dims, 0.13, 1.0), net, dev(R))))
    assert rel(a, b) <= NET_TOL


def test_training_lowers_the_loss_and_the_net_preconditions_the_solve(wd):
    dims, kappa = (4, 4, 4, 4), 0.125
    U = I.random_links(dims, 0.3, seed=0)
    ctx = wd.wd_create(dev(U), dims, kappa, 1.0)
    R = dev(I.z4_noise(dims, 12, seed=5))
    E, info = wd.bbicggr_solve(ctx, R, j=4, tol=1e-10)       # e = A^{-1} r from the plain solver
    assert info["status"] == wd.WD_OK
    net = wd.wd_net_create(4, 4, I.network_weights(4, 4, seed=3, noise=0.01))
    first = wd.wd_net_loss_grad(ctx, net, R, E, want_grad=False)[0]
    for _ in range(60):
        wd.wd_net_loss_grad(ctx, net, R, E, want_grad=False)
        wd.wd_net_adam_step(net, 2e-3)
    last = wd.wd_net_loss_grad(ctx, net, R, E, want_grad=False)[0]
    assert last < 0.7 * first
    op = O.WilsonClover(U, dims, kappa, 1.0)
    B = I.z4_noise(dims, 4, seed=11)
    X, info = wd.bbicggr_solve(ctx, dev(B), j=4, tol=1e-12, net=net)
    assert info["status"] == wd.WD_OK
    assert S.true_residual(op, B, host(X)).max() <= 1e-12


def test_trained_network_needs_fewer_iterations_than_no_preconditioner(wd):
    """What the trained network gains: trained on (r, A^{-1} r) pairs from the plain solver on 8
    seeded 8^4 configurations, then used as M on two held-out configurations, block BiCGGR needs
    well under half the iterations it needs without a preconditioner (j = 0), and the FP64 true
    residual still reaches 1e-12."""
    import torch
    from paper_0907_3261_gb300 import train_net as T
    dims, kappa, csw, L, eps = (8, 8, 8, 8), 0.13, 1.0, 12, 0.2
    d = torch.device("cuda", 0)
    pairs = T.make_pairs(wd, I, torch, dims, kappa, csw, range(8), L, eps, 12, d)
    net = wd.wd_net_create(4, 4, I.network_weights(4, 4, seed=7, noise=0.01))
    T.train(wd, net, pairs, 400, 3e-3, log_every=0)
    for s in (16, 17):
        links = I.random_links(dims, eps, seed=s)
        op = O.WilsonClover(links, dims, kappa, csw)
        ctx = wd.wd_create(dev(links), dims, kappa, csw)
        B = I.z4_noise(dims, L, seed=2000 + s)
        _, none = wd.bbicggr_solve(ctx, dev(B), j=0, tol=1e-12, maxit=3000)
        Xn, withnet = wd.bbicggr_solve(ctx, dev(B), j=12, tol=1e-12, net=net, maxit=3000)
        assert none["status"] == withnet["status"] == wd.WD_OK
        assert withnet["fallbacks"] == 0
        assert withnet["iters"] < 0.5 * none["iters"], (withnet["iters"], none["iters"])
        assert S.true_residual(op, B, host(Xn)).max() <= 1e-12
