"""Pins of oracle/stored.py (the Jacobi splitting with an FP32-stored operator) and a second,
independent dense assembly of A from its entry formula."""
import numpy as np
import pytest

from oracle import operator as O
from oracle import solver as S
from oracle import stored as ST
from paper_0907_3261_gb300 import inputs as I
import pins


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (2, 3, 2, 3)])
def test_apply_equals_the_entry_by_entry_assembly(dims):
    """A = A_D - kappa H with H assembled entry by entry from its definition (pins.py): the oracle's
    stencil, probed with unit vectors, is the same N x N matrix.  On extent-2 directions the
    forward and backward neighbours coincide and their blocks add."""
    links = I.random_links(dims, 0.4, seed=3)
    op = O.WilsonClover(links, dims, 0.13, 1.3)
    A_entries = op.dense_site_diagonal() - op.kappa * pins.dense_hopping_from_entries(links, dims)
    assert rel(op.dense(), A_entries) < 1e-14


@pytest.mark.parametrize("j", [0, 1, 2, 5])
def test_exact_pieces_reproduce_the_pinned_polynomial(j):
    """With unrounded pieces, sweeps G <- A_D^{-1}(U + kappa H G) from G = 0 are the Jacobi
    polynomial of Sec. 2 that solver.jacobi computes (pinned against dense matrices there)."""
    dims = (3, 4, 5, 6)
    links = I.random_links(dims, 0.3, seed=2)
    op = O.WilsonClover(links, dims, 0.12, 1.0)
    R = I.gaussian_block(dims, 4, seed=5)
    got = ST.jacobi_splitting(ST.exact_pieces(op), R, j)
    assert rel(got, S.jacobi(op, R, j)) < 1e-13


@pytest.mark.parametrize("j", [1, 2, 5])
def test_splitting_with_stored_pieces_is_the_dense_polynomial(j):
    """On 2^4 with the FP32-stored pieces: G = sum_{i<j} (kappa D H)^i D U, with H assembled entry
    by entry from the rounded links and D the block diagonal of the rounded inverse blocks."""
    dims = (2, 2, 2, 2)
    links = I.random_links(dims, 0.3, seed=0)
    op = O.WilsonClover(links, dims, 0.125, 1.0)
    pc = ST.fp32_pieces(op)
    H = pins.dense_hopping_from_entries(pc.U, dims)
    D = pins.block_diagonal(pc.Dinv)
    u = I.gaussian_block(dims, 3, seed=7)
    un = u.reshape(op.N, 3)
    T = pc.kappa * D @ H
    want = np.zeros_like(un)
    term = D @ un
    for _ in range(j):
        want = want + term
        term = T @ term
    got = ST.jacobi_splitting(pc, u, j).reshape(op.N, 3)
    assert rel(got, want) < 1e-13


def test_fp32_pieces_are_rounded_hermitian_and_chiral():
    dims = (3, 4, 5, 6)
    links = I.random_links(dims, 0.3, seed=2)
    op = O.WilsonClover(links, dims, 0.12, 1.0)
    pc = ST.fp32_pieces(op)
    assert np.array_equal(pc.U, pc.U.astype(np.complex64).astype(np.complex128))
    assert np.array_equal(pc.Dinv, pc.Dinv.astype(np.complex64).astype(np.complex128))
    assert pc.kappa == float(np.float32(0.12)) and pc.kappa != 0.12
    for c in (slice(0, 6), slice(6, 12)):
        blk = pc.Dinv[:, c, c]
        assert np.array_equal(blk, np.conj(np.swapaxes(blk, -1, -2)))
    assert not pc.Dinv[:, 0:6, 6:12].any() and not pc.Dinv[:, 6:12, 0:6].any()
    R = I.gaussian_block(dims, 3, seed=1)
    e = rel(ST.jacobi_splitting(pc, R, 5), S.jacobi(op, R, 5))
    assert 1e-9 < e < 1e-6         # the rounding of the stored operator, and nothing more


def test_csw_zero_inverse_is_exactly_the_identity():
    """c_SW = 0 gives A_D = 1, so the stored inverse blocks are exactly 1 and only the links and
    kappa carry FP32 rounding."""
    dims = (2, 3, 2, 4)
    op = O.WilsonClover(I.random_links(dims, 0.3, seed=1), dims, 0.12, 0.0)
    pc = ST.fp32_pieces(op)
    assert np.array_equal(pc.Dinv, np.broadcast_to(np.eye(12), pc.Dinv.shape))


def test_rounding_margin_detects_midpoints():
    one = 1.0
    mid = 1.0 + 2.0 ** -24          # exactly halfway between 1 and the next FP32 number
    assert pins.fp32_rounding_margin(np.array([mid])) == 0.0
    # the midpoints next to 1 are 1 + 2^-24 above and 1 - 2^-25 below (the binade changes at 1)
    assert pins.fp32_rounding_margin(np.array([one])) == pytest.approx(2.0 ** -25, rel=1e-12)
