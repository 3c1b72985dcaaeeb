"""The Jacobi preconditioner built from an FP32-stored operator -- test infrastructure only.

The preconditioner of Sec. 2 only has to be a fixed linear matrix M.  The mixed-precision forms of
the method keep the pieces M is built from -- the links, the inverse site blocks A_D^{-1} and kappa
-- rounded to FP32, and carry out the Jacobi splitting of the Sec. 2 polynomial,
    G_0 = 0,   G_{i+1} = A_D^{-1} (U + kappa H G_i),   i < j,
with those stored pieces.  This module states that M in FP64 arithmetic, so that a low-precision
implementation of the arithmetic on the spinors can be compared with it at the precision of that
arithmetic rather than at FP32's:

  * links: every entry rounded to complex64 (all 18 reals of a link);
  * A_D^{-1}: A_D is Hermitian (sigma_{mu nu} and F_{mu nu} are) and commutes with gamma_5, so its
    inverse is two Hermitian 6 x 6 chiral blocks; each block is taken as its Hermitian part
    (A + A^H) / 2 and rounded to complex64, its diagonal real, the off-chirality blocks zero;
  * kappa rounded to float32.

Parity status: pinned (tests/test_oracle_stored.py: with unrounded pieces the splitting equals the
pinned polynomial of ``solver.jacobi``; on 2^4 it equals the dense polynomial
sum_{i<j} (kappa D H)^i D U built from independently assembled dense D and H; rounding each piece
changes G by no more than FP32 rounding).
"""
from __future__ import annotations

import numpy as np

from .operator import Lattice, hopping_term


class StoredOperator:
    """The pieces of the Jacobi splitting: links U, inverse site blocks Dinv ([V][12][12]),
    kappa, on a lattice."""

    def __init__(self, lat: Lattice, U: np.ndarray, Dinv: np.ndarray, kappa: float):
        self.lat = lat
        self.U = np.asarray(U, dtype=np.complex128)
        self.Dinv = np.asarray(Dinv, dtype=np.complex128)
        self.kappa = float(kappa)

    def hopping(self, psi: np.ndarray) -> np.ndarray:
        return hopping_term(self.U, self.lat, psi)

    def apply_dinv(self, psi: np.ndarray) -> np.ndarray:
        psi = psi.reshape(self.lat.V, 12, -1)
        return np.einsum("vij,vjl->vil", self.Dinv, psi).reshape(self.lat.V, 4, 3, -1)


def exact_pieces(op) -> StoredOperator:
    """The unrounded pieces of a ``WilsonClover`` operator."""
    return StoredOperator(op.lat, op.U, op.AD_inv, op.kappa)


def fp32_pieces(op) -> StoredOperator:
    """The pieces rounded to FP32 as described in the module docstring."""
    U32 = op.U.astype(np.complex64).astype(np.complex128)
    D = np.zeros_like(op.AD_inv)
    for c in (slice(0, 6), slice(6, 12)):          # chirality +: spins 0, 1; -: spins 2, 3
        blk = op.AD_inv[:, c, c]
        herm = 0.5 * (blk + np.conj(np.swapaxes(blk, -1, -2)))
        herm = herm.astype(np.complex64).astype(np.complex128)
        idx = np.arange(6)
        herm[:, idx, idx] = herm[:, idx, idx].real
        D[:, c, c] = herm
    return StoredOperator(op.lat, U32, D, float(np.float32(op.kappa)))


def jacobi_splitting(pieces: StoredOperator, U: np.ndarray, j: int) -> np.ndarray:
    """G = M U by j sweeps G <- A_D^{-1} (U + kappa H G) from G = 0 (Sec. 2); G = U for j = 0."""
    if j == 0:
        return U.copy()
    G = np.zeros_like(U)
    for _ in range(j):
        G = pieces.apply_dinv(U + pieces.kappa * pieces.hopping(G))
    return G
