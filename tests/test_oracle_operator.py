"""Pins for the oracle's clover Wilson-Dirac operator (CPU only)."""
import numpy as np
import pytest

from oracle import operator as O
from paper_0907_3261_gb300 import inputs as I
import pins

TOL = 1e-13


def test_gamma_basis_is_the_stated_chiral_basis():
    g = O.gamma_matrices()
    ref = pins.chiral_basis()
    assert np.array_equal(g, ref)
    for m in range(4):
        assert np.allclose(g[m], g[m].conj().T)
        for n in range(4):
            assert np.allclose(g[m] @ g[n] + g[n] @ g[m], 2 * (m == n) * np.eye(4))
    assert np.allclose(O.gamma5(), np.diag([1, 1, -1, -1]))


@pytest.mark.parametrize("mu,nu", [(a, b) for a in range(4) for b in range(a + 1, 4)])
def test_sigma_matches_pauli_closed_form(mu, nu):
    assert np.allclose(O.sigma(mu, nu), pins.sigma_closed_form(mu, nu), atol=1e-15)


@pytest.mark.parametrize("dims,n", [((4, 4, 4, 4), (1, 0, 2, 3)), ((3, 5, 4, 6), (1, 2, 1, 5)),
                                    ((2, 2, 2, 2), (1, 1, 0, 1)), ((4, 4, 4, 4), (0, 0, 0, 0))])
def test_free_field_plane_wave_symbol(dims, n):
    assert pins.free_field_error(O.WilsonClover, dims=dims, n=n) < TOL


def test_gamma5_hermiticity():
    assert pins.gamma5_hermiticity_error(O.WilsonClover) < TOL


def test_gamma5_hermiticity_dense_2444():
    dims = (2, 4, 4, 4)
    op = O.WilsonClover(I.random_links(dims, 0.5, seed=8), dims, 0.125, 1.2)
    A = op.dense()
    g5 = np.kron(np.eye(op.lat.V), np.kron(np.diag([1, 1, -1, -1]), np.eye(3)))
    assert np.abs(g5 @ A @ g5 - A.conj().T).max() < 1e-14


def test_gauge_covariance():
    assert pins.gauge_covariance_error(O.WilsonClover) < TOL


def test_abelian_flux_clover_closed_form():
    assert pins.abelian_flux_error(O.WilsonClover) < TOL


def test_clover_block_structure_random_links():
    """A_D is Hermitian and commutes with gamma_5 (no chirality-mixing entries)."""
    dims = (3, 4, 5, 6)
    op = O.WilsonClover(I.random_links(dims, 0.6, seed=9), dims, 0.12, 1.5)
    AD = op.AD
    assert np.abs(AD - np.conj(np.swapaxes(AD, -1, -2))).max() < 1e-15
    assert np.abs(AD[:, 0:6, 6:12]).max() == 0.0
    assert np.abs(AD[:, 6:12, 0:6]).max() == 0.0


def test_csw_zero_gives_unit_site_diagonal():
    dims = (3, 4, 3, 4)
    op = O.WilsonClover(I.random_links(dims, 0.6, seed=9), dims, 0.12, 0.0)
    assert np.abs(op.AD - np.eye(12)).max() == 0.0


def test_hopping_is_nearest_neighbour_and_kappa_linear():
    """A depends on kappa as A_D(kappa) - kappa H: A(k1) - A(k2) with c_SW = 0 is -(k1-k2) H,
    and H couples a point source only to its 8 neighbours (16 on 2 sites per direction)."""
    dims = (4, 4, 4, 4)
    U = I.random_links(dims, 0.4, seed=10)
    a1 = O.WilsonClover(U, dims, 0.1, 0.0)
    a2 = O.WilsonClover(U, dims, 0.2, 0.0)
    src = I.point_sources(dims, 1)
    h = (a1.apply(src) - a2.apply(src)) / 0.1
    touched = np.nonzero(np.abs(h).reshape(a1.lat.V, -1).sum(1))[0]
    assert set(touched) == set(a1.lat.fwd[:, 0]) | set(a1.lat.bwd[:, 0])
