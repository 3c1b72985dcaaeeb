"""Oracle for the Jacobi preconditioner and preconditioned block BiCGGR (Sec. 2) -- test only.

``jacobi`` follows the Jacobi polynomial of Sec. 2: j sweeps of the splitting A = A_D - (A_D - A)
from the zero initial guess G_{k,0} = 0 (Sec. 3.3), so that
    G_k = sum_{i=0}^{j-1} (I - A_D^{-1} A)^i A_D^{-1} U_k      (j >= 1),      G_k = U_k  (j = 0).
Each sweep is written as the textbook Jacobi update G <- G + A_D^{-1} (U - A G).

``bbicggr`` follows the algorithm box of Sec. 2 line for line in its notation (R, P, F, V, W,
alpha, zeta, S, U, G, Y, gamma), with X_0 and R~_0 = R_0 as in Sec. 3.3.  Readings where the paper
is silent:
  * the stopping test max_i ||r_k^(i)|| / ||b^(i)|| <= eps is evaluated on R_0 and right after
    every R_{k+1} update, and the loop leaves before F_{k+1} = M R_{k+1}: this ordering is the one
    that reproduces every #MVM entry of Table 1, #MVM/L = 2(j+1)k + 1;
  * a j-step Jacobi counts as j MVMs (Sec. 3.3 counts it so, although the first sweep from
    G_{k,0} = 0 needs no product with A);
  * the L x L systems are solved by LU with partial pivoting (LAPACK getrf/getrs via scipy);
    the system counts as singular -- a breakdown, the rank loss of Sec. 4 in its exact form -- when
    a pivot is not finite or its modulus is below PIVOT_RTOL times the largest pivot modulus;
  * divergence: the run stops once the largest relative residual exceeds 1e2 (Sec. 3.3, the
    j = 0 runs of Fig. 2); breakdown also when Tr[W^H W] = 0.

``solve`` adds the true-residual check at exit: if some column of ||B - AX|| / ||B|| is above the
tolerance, block BiCGGR is restarted from X (at most ``max_restarts`` times).

Parity status: pinned (tests/test_oracle_solver.py: Jacobi vs the dense polynomial on 2^4, solve
vs dense LU on 2^4, free-field closed-form solve, per-iteration algebraic invariants, Table 1
#MVM identity).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg

OK = 0
NOT_CONVERGED = 4
DIVERGED = 5
BREAKDOWN = 6
PIVOT_RTOL = 1e-13


class Breakdown(Exception):
    pass


def solve_small(C: np.ndarray, rhs: np.ndarray) -> np.ndarray:
    """Solve C Z = rhs (L x L) by LU with partial pivoting; raise Breakdown if C is singular."""
    if not np.isfinite(C).all() or not np.isfinite(rhs).all():
        raise Breakdown("non-finite L x L system")
    lu, piv = scipy.linalg.lu_factor(C, check_finite=False)
    d = np.abs(np.diag(lu))
    if not np.isfinite(d).all() or d.max() == 0 or d.min() < PIVOT_RTOL * d.max():
        raise Breakdown("singular L x L system")
    return scipy.linalg.lu_solve((lu, piv), rhs, check_finite=False)


def jacobi(op, U: np.ndarray, j: int, counter=None) -> np.ndarray:
    """G = M U for the j-step Jacobi preconditioner with G_{k,0} = 0 (Sec. 2)."""
    if j == 0:
        return U.copy()
    G = np.zeros_like(U)
    for _ in range(j):
        G = G + op.apply_site_diagonal(U - op.apply(G), inverse=True)
        if counter is not None:
            counter[0] += 1
    return G


def column_norms(X: np.ndarray) -> np.ndarray:
    """||x^(i)||_2 for every column i of an N x L block."""
    L = X.shape[-1]
    return np.sqrt(np.sum(np.abs(X.reshape(-1, L)) ** 2, axis=0))


def herm_product(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """A^H B for N x L blocks (an L x L matrix)."""
    L = A.shape[-1]
    return A.reshape(-1, L).conj().T @ B.reshape(-1, L)


def right_multiply(X: np.ndarray, C: np.ndarray) -> np.ndarray:
    """X C for an N x L block X and an L x L matrix C."""
    L = X.shape[-1]
    return (X.reshape(-1, L) @ C).reshape(X.shape)


def direction_u(P, V, zeta, alpha):
    """U_k = S_k alpha_k with S_k = P_k - zeta_k V_k (Sec. 2, algorithm box)."""
    S = P - zeta * V                           # S_k = P_k - zeta_k V_k
    return right_multiply(S, alpha)            # U_k = S_k alpha_k


def solution_update(X, R, F, G, W, Y, zeta):
    """X_{k+1} = X_k + zeta_k F_k + G_k and R_{k+1} = R_k - zeta_k W_k - Y_k (Sec. 2, algorithm
    box)."""
    return X + zeta * F + G, R - zeta * W - Y


def direction_pv(R_new, Uk, W_new, Y, gamma):
    """P_{k+1} = R_{k+1} + U_k gamma_k and V_{k+1} = W_{k+1} + Y_k gamma_k (Sec. 2, algorithm
    box)."""
    return R_new + right_multiply(Uk, gamma), W_new + right_multiply(Y, gamma)


@dataclass
class SolveResult:
    X: np.ndarray
    status: int
    iters: int                 # outer iterations k (sum over restarts)
    mvm: int                   # MVMs per column, counted as the paper counts them
    rec_resid: np.ndarray      # final recursive residual per column, relative to ||b||
    true_resid: np.ndarray     # ||B - AX|| / ||B|| per column
    history: list = field(default_factory=list)   # max_i relative residual after every update
    restarts: int = 0


def bbicggr(op, B, X0, j, eps, maxit=10000, div_thresh=1e2, on_iter=None):
    """Preconditioned block BiCGGR, the algorithm box of Sec. 2.

    Returns (X, status, k, mvm_per_column, final relative recursive residuals, history).
    ``on_iter(state)`` is called after every outer iteration with the iteration's matrices
    (used by the invariant tests).
    """
    count = [0]

    def A(Z):
        count[0] += 1
        return op.apply(Z)

    def M(Z):
        return jacobi(op, Z, j, counter=count)

    bnorm = column_norms(B)
    X = X0.copy()
    R = B - A(X)                                   # Compute R_0 = B - A X_0
    P = R.copy()                                   # Set P_0 = R_0
    Rt = R.copy()                                  # Choose R~_0 = R_0
    hist = [float(np.max(column_norms(R) / bnorm))]
    if hist[-1] <= eps:
        return X, OK, 0, count[0], column_norms(R) / bnorm, hist
    F = M(R)                                       # F_0 = M R_0
    W = A(F)                                       # V_0 = W_0 = A F_0
    V = W.copy()
    k = 0
    while True:
        if k >= maxit:
            return X, NOT_CONVERGED, k, count[0], column_norms(R) / bnorm, hist
        try:                                       # (R~_0^H V_k) alpha_k = R~_0^H R_k
            alpha = solve_small(herm_product(Rt, V), herm_product(Rt, R))
        except Breakdown:
            return X, BREAKDOWN, k, count[0], column_norms(R) / bnorm, hist
        ww = np.vdot(W, W)                         # Tr[W^H W]
        if ww == 0:
            return X, BREAKDOWN, k, count[0], column_norms(R) / bnorm, hist
        zeta = np.vdot(W, R) / ww                  # zeta_k = Tr[W^H R] / Tr[W^H W]
        Uk = direction_u(P, V, zeta, alpha)        # U_k = (P_k - zeta_k V_k) alpha_k
        G = M(Uk)                                  # G_k = M U_k
        Y = A(G)                                   # Y_k = A G_k
        X, R_new = solution_update(X, R, F, G, W, Y, zeta)   # X_{k+1}, R_{k+1}
        k += 1
        rel = column_norms(R_new) / bnorm
        hist.append(float(np.max(rel)))
        state = dict(k=k - 1, R=R, P=P, V=V, W=W, F=F, alpha=alpha, zeta=zeta, U=Uk, G=G, Y=Y,
                     X_new=X, R_new=R_new, Rt=Rt)
        if not np.isfinite(hist[-1]):
            return X, BREAKDOWN, k, count[0], rel, hist
        if hist[-1] <= eps:
            if on_iter is not None:
                on_iter(state)
            return X, OK, k, count[0], rel, hist
        if hist[-1] > div_thresh:
            return X, DIVERGED, k, count[0], rel, hist
        F = M(R_new)                               # F_{k+1} = M R_{k+1}
        W = A(F)                                   # W_{k+1} = A F_{k+1}
        try:                                       # (R~_0^H R_k) gamma_k = R~_0^H R_{k+1} / zeta_k
            gamma = solve_small(herm_product(Rt, R), herm_product(Rt, R_new) / zeta)
        except Breakdown:
            return X, BREAKDOWN, k, count[0], rel, hist
        state.update(F_new=F, W_new=W, gamma=gamma)
        P, V = direction_pv(R_new, Uk, W, Y, gamma)   # P_{k+1}, V_{k+1}
        state.update(P_new=P, V_new=V)
        if on_iter is not None:
            on_iter(state)
        R = R_new


def true_residual(op, B, X):
    """||b^(i) - A x^(i)|| / ||b^(i)|| per column."""
    return column_norms(B - op.apply(X)) / column_norms(B)


def solve(op, B, X0=None, j=0, tol=1e-12, maxit=10000, max_restarts=3, div_thresh=1e2):
    """Block BiCGGR to recursive residual ``tol``, then restarts from X while the true residual
    of some column is above ``tol``."""
    X = np.zeros_like(B) if X0 is None else X0.copy()
    iters = mvm = 0
    hist = []
    restarts = 0
    while True:
        X, status, k, nm, rec, h = bbicggr(op, B, X, j, tol, maxit - iters, div_thresh)
        iters += k
        mvm += nm
        hist += h
        tr = true_residual(op, B, X)
        if status != OK or np.max(tr) <= tol or restarts >= max_restarts:
            if status == OK and np.max(tr) > tol:
                status = NOT_CONVERGED
            return SolveResult(X, status, iters, mvm, rec, tr, hist, restarts)
        restarts += 1
