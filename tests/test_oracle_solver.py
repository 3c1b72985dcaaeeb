"""Pins for the oracle's Jacobi preconditioner and block BiCGGR (CPU only)."""
import os

import numpy as np
import pytest

from oracle import operator as O
from oracle import solver as S
from paper_0907_3261_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def small_op(dims=(2, 2, 2, 2), kappa=0.115, csw=1.0, eps=0.3, seed=0):
    return O.WilsonClover(I.random_links(dims, eps, seed), dims, kappa, csw)


# ---------------------------------------------------------------- Jacobi (Sec. 2 polynomial)
@pytest.mark.parametrize("j", [0, 1, 2, 5])
def test_jacobi_equals_dense_polynomial(j):
    """G = sum_{i<j} (I - A_D^{-1} A)^i A_D^{-1} U, evaluated with dense N x N matrices."""
    op = small_op(kappa=0.12, csw=1.4, eps=0.5)
    A = op.dense()
    Dinv = np.linalg.inv(op.dense_site_diagonal())
    Uk = I.gaussian_block(op.lat.dims, 3, seed=5)
    u = Uk.reshape(op.N, 3)
    if j == 0:
        want = u
    else:
        T = np.eye(op.N) - Dinv @ A
        want = np.zeros_like(u)
        term = Dinv @ u
        for _ in range(j):
            want = want + term
            term = T @ term
    got = S.jacobi(op, Uk, j).reshape(op.N, 3)
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-13


def test_jacobi_without_clover_is_neumann_series_in_hopping():
    """c_SW = 0: A_D = 1, so G = sum_{i<j} (kappa H)^i U with H = (1 - A) / kappa."""
    op = small_op(dims=(2, 2, 2, 4), kappa=0.11, csw=0.0, eps=0.5)
    H = (np.eye(op.N) - op.dense()) / op.kappa
    Uk = I.gaussian_block(op.lat.dims, 2, seed=6).reshape(op.N, 2)
    want = sum(np.linalg.matrix_power(op.kappa * H, i) @ Uk for i in range(4))
    got = S.jacobi(op, Uk.reshape(op.lat.V, 4, 3, 2), 4).reshape(op.N, 2)
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-13


# ---------------------------------------------------------------- solve vs exact solutions
@pytest.mark.parametrize("j,L", [(0, 1), (0, 4), (2, 4), (4, 12)])
def test_solve_matches_dense_lu_on_2_4(j, L):
    """X of block BiCGGR equals the dense LU solution of A X = B on a 2^4 lattice (N = 192),
    where the forward and backward neighbours of every site coincide."""
    op = small_op()
    B = I.z4_noise(op.lat.dims, L, seed=1)
    X_lu = np.linalg.solve(op.dense(), B.reshape(op.N, L))
    r = S.solve(op, B, j=j, tol=1e-12)
    assert r.status == S.OK
    assert r.true_resid.max() <= 1e-12
    assert np.linalg.norm(r.X.reshape(op.N, L) - X_lu) / np.linalg.norm(X_lu) < 1e-10


def test_free_field_solve_closed_form():
    """U = 1: A^{-1} on a plane wave is [a - 2 i kappa sum gamma_mu s_mu] / (a^2 + 4 kappa^2 sum s^2)
    with a = 1 - 2 kappa sum cos p_mu, s_mu = sin p_mu.  Every source column mixes three momenta
    (a column of a single momentum would converge alone and make the block Gram matrix singular)."""
    import pins
    dims = (4, 4, 4, 8)
    kappa = 0.12
    op = O.WilsonClover(I.unit_links(dims), dims, kappa, 1.0)
    c = pins.coords(dims)
    g = pins.chiral_basis()
    moms = [(0, 0, 0, 0), (1, 0, 0, 1), (1, 2, 3, 5)]
    L = 3
    B = np.zeros((op.lat.V, 4, 3, L), dtype=complex)
    X_exact = np.zeros_like(B)
    u = I.complex_gaussian(3, 77, 12 * L * len(moms)).reshape(len(moms), 4, 3, L)
    for m, n in enumerate(moms):
        p = 2 * np.pi * np.asarray(n) / np.asarray(dims)
        wave = np.exp(1j * c @ p)[:, None, None, None] * u[m][None]
        a = 1 - 2 * kappa * np.cos(p).sum()
        s = np.sin(p)
        inv = (a * np.eye(4) - 2j * kappa * sum(g[mu] * s[mu] for mu in range(4))) / (
            a * a + 4 * kappa ** 2 * (s * s).sum())
        B += wave
        X_exact += np.einsum("st,vtal->vsal", inv, wave)
    r = S.solve(op, B, j=3, tol=1e-12)
    assert r.status == S.OK
    assert np.linalg.norm(r.X - X_exact) / np.linalg.norm(X_exact) < 1e-10


# ---------------------------------------------------------------- algebraic invariants
def test_bbicggr_invariants_every_iteration():
    """Exact-arithmetic relations of the algorithm box, checked at every outer iteration:
    F = M R, W = A M R, V = A M P, G = M U, Y = A G, R~_0^H (R - V alpha) = 0 (definition of alpha),
    Tr[W^H (R - zeta W)] = 0 (zeta minimises ||R - zeta W||_F), R_{k+1} = (I - zeta A M)(R - V alpha),
    and R_{k+1} = B - A X_{k+1} (the property block BiCGGR is built for)."""
    dims = (4, 4, 4, 4)
    op = O.WilsonClover(I.random_links(dims, 0.3, 0), dims, 0.115, 1.0)
    B = I.point_sources(dims, 4)
    j = 4
    M = lambda Z: S.jacobi(op, Z, j)
    AM = lambda Z: op.apply(M(Z))
    worst = {}

    def note(name, a, b):
        worst[name] = max(worst.get(name, 0.0), np.linalg.norm(a - b) / np.linalg.norm(b))

    def check(st):
        note("F=MR", st["F"], M(st["R"]))
        note("W=AMR", st["W"], AM(st["R"]))
        note("V=AMP", st["V"], AM(st["P"]))
        note("G=MU", st["G"], M(st["U"]))
        note("Y=AG", st["Y"], op.apply(st["G"]))
        Q = st["R"] - S.right_multiply(st["V"], st["alpha"])
        worst["alpha"] = max(worst.get("alpha", 0.0), np.abs(S.herm_product(st["Rt"], Q)).max()
                             / np.abs(S.herm_product(st["Rt"], st["R"])).max())
        t = np.vdot(st["W"], st["R"] - st["zeta"] * st["W"])
        worst["zeta"] = max(worst.get("zeta", 0.0), abs(t) / abs(np.vdot(st["W"], st["R"])))
        note("R_next", st["R_new"], Q - st["zeta"] * AM(Q))
        gap = np.linalg.norm(st["R_new"] - (B - op.apply(st["X_new"]))) / np.linalg.norm(B)
        worst["R=B-AX"] = max(worst.get("R=B-AX", 0.0), gap)

    X, status, k, nmvm, rec, hist = S.bbicggr(op, B, np.zeros_like(B), j, 1e-12, on_iter=check)
    assert status == S.OK and k >= 5
    for name, v in worst.items():
        bound = 1e-14 if name == "R=B-AX" else 1e-10
        assert v < bound, (name, v)
    assert S.true_residual(op, B, X).max() < 1e-12


def test_recursive_residual_tracks_true_residual():
    """Sec. 1: block BiCGGR removes the true/recursive residual gap of block BiCGSTAB."""
    dims = (4, 4, 4, 4)
    op = O.WilsonClover(I.random_links(dims, 0.3, 0), dims, 0.12, 1.0)
    B = I.z4_noise(dims, 4, seed=1)
    X, status, k, _, rec, _ = S.bbicggr(op, B, np.zeros_like(B), 2, 1e-13)
    assert status == S.OK
    assert S.true_residual(op, B, X).max() < 1e-12


# ---------------------------------------------------------------- #MVM accounting (Table 1)
def read_table1():
    rows = []
    with open(os.path.join(GOLDEN, "table1_iterations.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            L, j, k, m = line.split()
            rows.append((int(L), int(j), float(k), float(m)))
    return rows


def test_table1_mvm_identity():
    """Every #MVM/L entry of Table 1 equals 2(j+1)k + 1 (to the table's 0.1 rounding)."""
    rows = read_table1()
    assert len(rows) == 33
    for L, j, k, m in rows:
        assert abs(2 * (j + 1) * k + 1 - m) < 0.05 + 1e-9, (L, j, k, m)


@pytest.mark.parametrize("j,L", [(0, 1), (3, 2), (4, 4)])
def test_oracle_mvm_count_follows_table1(j, L):
    """The MVMs the oracle performs (A products plus j per Jacobi call) equal 2(j+1)k + 1."""
    dims = (4, 4, 4, 4)
    op = O.WilsonClover(I.random_links(dims, 0.3, 0), dims, 0.115, 1.0)
    B = I.z4_noise(dims, L, seed=1)
    X, status, k, nmvm, _, _ = S.bbicggr(op, B, np.zeros_like(B), j, 1e-12)
    assert status == S.OK
    assert nmvm == 2 * (j + 1) * k + 1


# ---------------------------------------------------------------- error paths (Sec. 3.3)
def test_status_not_converged_divergence_and_breakdown():
    op = small_op(dims=(2, 2, 2, 4))
    B = I.z4_noise(op.lat.dims, 2, seed=1)
    r = S.bbicggr(op, B, np.zeros_like(B), 1, 1e-12, maxit=2)
    assert r[1] == S.NOT_CONVERGED and r[2] == 2
    r = S.bbicggr(op, B, np.zeros_like(B), 1, 1e-12, div_thresh=1e-6)
    assert r[1] == S.DIVERGED and r[2] == 1
    B2 = B.copy()
    B2[..., 1] = B2[..., 0]                    # rank-deficient block: R~_0^H V_0 is singular
    r = S.bbicggr(op, B2, np.zeros_like(B2), 1, 1e-12)
    assert r[1] == S.BREAKDOWN and r[2] == 0
