"""Pins of the C++ oracle (oracle/cpp/oracle.cpp): the closed forms and symmetries that pin the numpy
oracle, a dense LU solve on 2^4 with A assembled entry by entry, the Table 1 #MVM identity, and
agreement with the independently written numpy oracle.  Planted mistakes, compiled from edited
copies of the source, must each break at least one pin."""
import os
import subprocess

import numpy as np
import pytest

from oracle import cpp
from oracle import operator as O
from oracle import solver as S
from paper_0907_3261_gb300 import inputs as I
import pins

PIN_TOL = 1e-10


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def make(library=None):
    return lambda U, dims, kappa, csw: cpp.CppOracle(U, dims, kappa, csw, library=library)


def test_cpp_operator_satisfies_every_pin():
    errs = pins.all_operator_pins(make())
    assert max(errs.values()) < 1e-13, errs


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (2, 3, 2, 3)])
def test_cpp_apply_equals_the_entry_by_entry_assembly(dims):
    links = I.random_links(dims, 0.4, seed=3)
    op = O.WilsonClover(links, dims, 0.13, 1.3)
    c = cpp.CppOracle(links, dims, 0.13, 1.3)
    N = 12 * int(np.prod(dims))
    eye = np.eye(N, dtype=complex).reshape(N // 12, 4, 3, N)
    A_cpp = c.apply(eye).reshape(N, N)
    A_entries = op.dense_site_diagonal() - 0.13 * pins.dense_hopping_from_entries(links, dims)
    assert rel(A_cpp, A_entries) < 1e-14


@pytest.mark.parametrize("j", [0, 1, 2, 5])
def test_cpp_agrees_with_the_numpy_oracle(j):
    dims = (3, 4, 5, 6)
    links = I.random_links(dims, 0.4, seed=2)
    op = O.WilsonClover(links, dims, 0.12, 1.0)
    c = cpp.CppOracle(links, dims, 0.12, 1.0)
    X = I.gaussian_block(dims, 5, seed=3)
    assert rel(c.apply(X), op.apply(X)) < 1e-14
    assert rel(c.apply_site_diagonal(X, inverse=True),
               op.apply_site_diagonal(X, inverse=True)) < 1e-14
    assert rel(c.jacobi(X, j), S.jacobi(op, X, j)) < 1e-13


@pytest.mark.parametrize("B_kind,L,j", [("point", 4, 4), ("z4", 12, 4), ("z4", 3, 0)])
def test_cpp_solve_agrees_with_the_numpy_oracle(B_kind, L, j):
    dims = (4, 4, 4, 4)
    links = I.random_links(dims, 0.3, seed=0)
    op = O.WilsonClover(links, dims, 0.115, 1.0)
    B = I.point_sources(dims, L) if B_kind == "point" else I.z4_noise(dims, L, seed=1)
    ref = S.solve(op, B, j=j, tol=1e-12)
    X, st, k, restarts, mvm, tr = cpp.CppOracle(links, dims, 0.115, 1.0).solve(B, j)
    assert st == 0 and k == ref.iters and mvm == ref.mvm
    if restarts == 0:
        assert mvm == 2 * (j + 1) * k + 1           # Table 1's identity, per column
    assert tr.max() <= 1e-12
    assert rel(X, ref.X) < 1e-10


@pytest.mark.parametrize("L", [1, 4])
def test_cpp_solve_equals_dense_lu_on_2_4(L):
    dims = (2, 2, 2, 2)
    links = I.random_links(dims, 0.3, seed=0)
    op = O.WilsonClover(links, dims, 0.115, 1.0)
    A = op.dense_site_diagonal() - 0.115 * pins.dense_hopping_from_entries(links, dims)
    B = I.z4_noise(dims, L, seed=1)
    X, st, *_ = cpp.CppOracle(links, dims, 0.115, 1.0).solve(B, 2)
    X_lu = np.linalg.solve(A, B.reshape(op.N, L))
    assert st == 0 and rel(X.reshape(op.N, L), X_lu) < 1e-10


def test_stepper_reproduces_the_solve():
    dims = (4, 4, 4, 4)
    links = I.random_links(dims, 0.3, seed=0)
    B = I.z4_noise(dims, 4, seed=1)
    c = cpp.CppOracle(links, dims, 0.115, 1.0)
    X, st, k, restarts, mvm, tr = c.solve(B, 4, max_restarts=0)
    s = cpp.Stepper(links, dims, 0.115, 1.0)
    assert s.start(B, 4) == cpp.RUNNING
    steps = 0
    while s.status == cpp.RUNNING:
        s.step()
        steps += 1
    Xs, rec, trs, ks, mvms = s.result()
    assert s.status == st == 0 and steps == ks == k and mvms == mvm
    assert np.array_equal(Xs, X) and np.array_equal(trs, tr)
    s.close()


MUTATIONS = {
    "projector_sign": ("const double sg = dir == 0 ? -1.0 : 1.0;",
                       "const double sg = dir == 0 ? 1.0 : -1.0;"),
    "no_dagger_backward": ("(dir == 0 ? u[a * 3 + b] : std::conj(u[b * 3 + a]))",
                           "(dir == 0 ? u[a * 3 + b] : u[a * 3 + b])"),
    "clover_sign": ("-= kappa * csw * sig[mu][nu][a][b]", "+= kappa * csw * sig[mu][nu][a][b]"),
    "leaf_not_daggered": ("L(xmm, mu, a); dag3(a, a);", "L(xmm, mu, a);"),
    "jacobi_sign": ("G[e] += D[e];", "G[e] -= D[e];"),
    "zeta_conjugated": ("vdot(W.data(), R.data(), (long)n) / ww",
                        "vdot(R.data(), W.data(), (long)n) / ww"),
    "gamma_missing_zeta": ("rhs[e] = rtr_new[e] / zeta;", "rhs[e] = rtr_new[e];"),
    "p_update_uses_y": ("right_mul(Uk.data(), gamma.data(), N, L, S.data());",
                        "right_mul(Y.data(), gamma.data(), N, L, S.data());"),
}


def mutant_error(library):
    """The largest pin error of a compiled mutant: operator pins, the dense Jacobi polynomial and
    the dense LU solve on 2^4 (inf when the mutant fails outright)."""
    try:
        errs = list(pins.all_operator_pins(make(library)).values())
        dims = (2, 2, 2, 2)
        links = I.random_links(dims, 0.3, seed=0)
        op = O.WilsonClover(links, dims, 0.115, 1.0)
        A = op.dense_site_diagonal() - 0.115 * pins.dense_hopping_from_entries(links, dims)
        c = cpp.CppOracle(links, dims, 0.115, 1.0, library=library)
        u = I.gaussian_block(dims, 2, seed=5)
        errs.append(rel(c.jacobi(u, 3).reshape(op.N, 2),
                        pins.dense_jacobi_polynomial(A, op.dense_site_diagonal(), 3)
                        @ u.reshape(op.N, 2)))
        B = I.z4_noise(dims, 3, seed=1)
        X, st, *_ = c.solve(B, 2, maxit=300)
        errs.append(rel(X.reshape(op.N, 3), np.linalg.solve(A, B.reshape(op.N, 3))))
        errs.append(history_error(library))
        e = max(errs)
        return e if np.isfinite(e) else np.inf
    except Exception:
        return np.inf


def history_error(library=None):
    """Largest relative difference between the C++ oracle's residual after every outer iteration
    (read step by step) and the history of the numpy oracle, whose iteration is pinned by the
    per-iteration invariants of the algorithm box; inf if the iteration counts differ.  Mistakes in
    the direction recurrences that the method corrects for (the solve still converges) change this
    path."""
    dims = (4, 4, 4, 4)
    links = I.random_links(dims, 0.3, seed=0)
    B = I.z4_noise(dims, 4, seed=1)
    op = O.WilsonClover(links, dims, 0.115, 1.0)
    X0 = np.zeros_like(B)
    _, status, k, _, _, hist = S.bbicggr(op, B, X0, 3, 1e-12)
    s = cpp.Stepper(links, dims, 0.115, 1.0, library=library)
    s.start(B, 3)
    got = [s.result(true_resid=False)[1].max()]
    while s.status == cpp.RUNNING and len(got) <= 3 * k:
        s.step()
        got.append(s.result(true_resid=False)[1].max())
    s.close()
    if len(got) != len(hist):
        return np.inf
    return float(np.max(np.abs(np.array(got) - hist) / np.array(hist)))


def test_cpp_residual_history_follows_the_numpy_oracle():
    assert history_error() < 1e-6


def test_unmutated_cpp_passes_the_mutant_pins():
    assert mutant_error(cpp.lib()) < 1e-10


@pytest.mark.parametrize("kind", sorted(MUTATIONS))
def test_cpp_mutation_is_caught(kind, tmp_path):
    old, new = MUTATIONS[kind]
    src = open(cpp.SRC).read()
    assert src.count(old) == 1, old
    path = tmp_path / "mutant.cpp"
    path.write_text(src.replace(old, new))
    so = str(tmp_path / "libmutant.so")
    subprocess.run(["g++", *cpp.FLAGS, str(path), "-o", so], check=True)
    assert mutant_error(cpp.load(so)) > PIN_TOL
