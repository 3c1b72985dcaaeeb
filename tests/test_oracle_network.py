"""Pins for the oracle of the learned preconditioner network (CPU only)."""
import numpy as np
import pytest

from oracle import network as N
from oracle import operator as O
from paper_0907_3261_gb300 import inputs as I
import pins


def setup(dims=(2, 2, 2, 4), L=2, seed=0, noise=0.3, layers=3, hidden=2):
    U = I.random_links(dims, 0.5, seed=seed)
    lat = O.Lattice(dims)
    W = I.network_weights(layers, hidden, seed=seed + 1, noise=noise)
    R = I.gaussian_block(dims, L, seed=seed + 2)
    E = I.gaussian_block(dims, L, seed=seed + 3)
    return U, lat, W, R, E


def test_identity_initialisation_is_identity_map():
    U, lat, _, R, _ = setup()
    W = I.network_weights(4, 4, seed=0, noise=0.0)
    Y, _ = N.forward(U, lat, W, R)
    assert np.allclose(Y, R, atol=1e-14)


def test_gradient_matches_finite_differences():
    """d loss / d Re W = 2 Re G and d loss / d Im W = 2 Im G, checked entry by entry on a random
    sample of entries of every layer with central differences."""
    U, lat, W, R, E = setup()
    loss, G = N.loss_and_grad(U, lat, W, R, E)
    rng = np.random.default_rng(0)
    h = 1e-6
    for li in range(len(W)):
        for _ in range(12):
            idx = tuple(rng.integers(0, s) for s in W[li].shape)
            for part, unit in (("re", 1.0), ("im", 1j)):
                Wp = [w.copy() for w in W]
                Wm = [w.copy() for w in W]
                Wp[li][idx] += unit * h
                Wm[li][idx] -= unit * h
                fd = (N.loss_and_grad(U, lat, Wp, R, E)[0] - N.loss_and_grad(U, lat, Wm, R, E)[0]) / (2 * h)
                an = 2 * (G[li][idx].real if part == "re" else G[li][idx].imag)
                assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (li, idx, part, fd, an)


def test_network_is_linear_in_the_spinor():
    U, lat, W, R, E = setup()
    a, b = 0.7 - 0.2j, -1.3 + 0.4j
    Y1, _ = N.forward(U, lat, W, a * R + b * E)
    Y2 = a * N.forward(U, lat, W, R)[0] + b * N.forward(U, lat, W, E)[0]
    assert np.linalg.norm(Y1 - Y2) / np.linalg.norm(Y2) < 1e-13


def test_network_is_gauge_covariant():
    dims = (3, 2, 2, 4)
    U = I.random_links(dims, 0.5, seed=4)
    lat = O.Lattice(dims)
    Om = I.random_gauge_transform(dims, seed=5)
    Up = np.empty_like(U)
    for mu in range(4):
        Up[:, mu] = Om @ U[:, mu] @ np.conj(np.swapaxes(Om[lat.fwd[mu]], -1, -2))
    W = I.network_weights(4, 2, seed=3, noise=0.4)
    psi = I.gaussian_block(dims, 2, seed=6)
    rot = lambda z: np.einsum("vab,vsbl->vsal", Om, z)
    lhs = N.forward(Up, lat, W, rot(psi))[0]
    rhs = rot(N.forward(U, lat, W, psi)[0])
    assert np.linalg.norm(lhs - rhs) / np.linalg.norm(rhs) < 1e-13


def test_one_layer_wilson_hopping_special_case():
    """With W_0 = 1, W_{+mu} = kappa (1 - g_mu) and W_{-mu} = kappa (1 + g_mu), one layer is 1 + kappa H,
    which for c_SW = 0 equals 2 - A with A the (independently pinned) oracle operator."""
    dims = (3, 4, 2, 4)
    kappa = 0.11
    U = I.random_links(dims, 0.5, seed=7)
    lat = O.Lattice(dims)
    g = pins.chiral_basis()
    W = np.zeros((9, 1, 1, 4, 4), dtype=complex)
    W[0, 0, 0] = np.eye(4)
    for mu in range(4):
        W[1 + mu, 0, 0] = kappa * (np.eye(4) - g[mu])
        W[5 + mu, 0, 0] = kappa * (np.eye(4) + g[mu])
    psi = I.gaussian_block(dims, 3, seed=8)
    Y = N.forward(U, lat, [W], psi)[0]
    A = O.WilsonClover(U, dims, kappa, 0.0)
    want = 2 * psi - A.apply(psi)
    assert np.linalg.norm(Y - want) / np.linalg.norm(want) < 1e-13


def test_adam_first_step_closed_form():
    """With zero moments, bias correction makes the first Adam step -lr * g / (|g| + eps) per real
    parameter."""
    W = [np.array([[1.0 + 2.0j, -0.5j]])]
    G = [np.array([[0.25 - 1.0j, 3.0 + 0.0j]])]
    lr = 0.01
    eps = 1e-12
    new = N.adam_step(W, G, {}, lr, eps=eps)[0]
    g_re, g_im = 2 * G[0].real, 2 * G[0].imag
    step_re = -lr * g_re / (np.abs(g_re) + eps)
    step_im = -lr * g_im / (np.abs(g_im) + eps)
    assert np.allclose(new, W[0] + step_re + 1j * step_im, atol=1e-15)
