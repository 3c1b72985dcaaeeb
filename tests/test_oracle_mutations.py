"""Plant plausible mistakes in the oracle (on the CPU) and check that the pins catch each one.

Each mutation is a one-line edit of the oracle's own source text, executed as a fresh module; a pin
set that a dropped term, a wrong sign, a wrong index or a transposed operand slips through would not
pin anything, so every mutation must push at least one pin far above rounding.
"""
import sys
import types

import numpy as np
import pytest

from oracle import operator as O
from oracle import solver as S
from paper_0907_3261_gb300 import inputs as I
import pins

PIN_TOL = 1e-10


def mutated_module(module, edits):
    src = open(module.__file__).read()
    for old, new in edits:
        assert src.count(old) == 1, old
        src = src.replace(old, new)
    name = module.__name__ + "_mutated"
    mod = types.ModuleType(name)
    sys.modules[name] = mod          # dataclasses look their module up here
    try:
        exec(compile(src, module.__file__ + "[mutated]", "exec"), mod.__dict__)
    finally:
        del sys.modules[name]
    return mod.__dict__


OPERATOR_MUTATIONS = {
    "swap_projectors": [('one - g[mu], up', 'one + g[mu], up'),
                        ('one + g[mu], dn', 'one - g[mu], dn')],
    "no_dagger_backward": [('_dag(U_back), psi', 'U_back, psi')],
    "backward_link_at_x": [('U_back = U[lat.bwd[mu], mu]', 'U_back = U[:, mu]')],
    "transpose_forward": [('"vab,vsbl->vsal", U[:, mu]', '"vba,vsbl->vsal", U[:, mu]')],
    "backward_reads_forward": [('psi[lat.bwd[mu]])', 'psi[lat.fwd[mu]])')],
    "hopping_sign": [('(psi) - self.kappa * self.hopping', '(psi) + self.kappa * self.hopping')],
    "hopping_factor_two": [('(psi) - self.kappa * self.hopping',
                            '(psi) - 2 * self.kappa * self.hopping')],
    "gamma_t_sign": [('g[3, 0:2, 2:4] = np.eye(2)', 'g[3, 0:2, 2:4] = -np.eye(2)'),
                     ('g[3, 2:4, 0:2] = np.eye(2)', 'g[3, 2:4, 0:2] = -np.eye(2)')],
    "leaf_order": [('leaf1 = Um @ Un[x_pm]', 'leaf1 = Un[x_pm] @ Um')],
    "leaf_reversed": [('Q = leaf1 + leaf2 + leaf3 + leaf4', 'Q = leaf1 + _dag(leaf2) + leaf3 + leaf4')],
    "leaf_dropped": [('Q = leaf1 + leaf2 + leaf3 + leaf4', 'Q = leaf1 + leaf2 + leaf4')],
    "leaf_wrong_site": [('@ Un[x_mn_pm] @', '@ Un[x_pm] @')],
    "normalisation": [('(Q - _dag(Q)) / 8j', '(Q - _dag(Q)) / 4j')],
    "not_antihermitian_part": [('(Q - _dag(Q)) / 8j', 'Q / 4j')],
    "clover_sign": [('AD -= kappa * csw * term', 'AD += kappa * csw * term')],
    "clover_half": [('AD -= kappa * csw * term', 'AD -= 0.5 * kappa * csw * term')],
    "sigma_sign": [('return 0.5j * (g[mu]', 'return -0.5j * (g[mu]')],
    "neighbour_step_two": [('cf[mu] = (coords[mu] + 1)', 'cf[mu] = (coords[mu] + 2)')],
}


@pytest.mark.parametrize("kind", sorted(OPERATOR_MUTATIONS))
def test_operator_mutation_is_caught(kind):
    ns = mutated_module(O, OPERATOR_MUTATIONS[kind])
    errs = pins.all_operator_pins(ns["WilsonClover"])
    assert max(errs.values()) > PIN_TOL, errs


def test_unmutated_operator_passes_every_pin():
    errs = pins.all_operator_pins(O.WilsonClover)
    assert max(errs.values()) < 1e-13, errs


# ---------------------------------------------------------------- solver mutations
def solver_pin_error(ns):
    """Dense-LU solve on 2^4 and the two-step Jacobi polynomial; the larger relative error."""
    dims = (2, 2, 2, 2)
    op = O.WilsonClover(I.random_links(dims, 0.3, 0), dims, 0.115, 1.0)
    A = op.dense()
    B = I.z4_noise(dims, 4, seed=1)
    X_lu = np.linalg.solve(A, B.reshape(op.N, 4))
    try:
        r = ns["solve"](op, B, j=2, tol=1e-12, maxit=300, max_restarts=0)
        e_solve = np.linalg.norm(r.X.reshape(op.N, 4) - X_lu) / np.linalg.norm(X_lu)
    except Exception:
        e_solve = np.inf
    Dinv = np.linalg.inv(op.dense_site_diagonal())
    u = I.gaussian_block(dims, 2, seed=5).reshape(op.N, 2)
    want = Dinv @ u + (np.eye(op.N) - Dinv @ A) @ (Dinv @ u)
    got = ns["jacobi"](op, u.reshape(op.lat.V, 4, 3, 2), 2).reshape(op.N, 2)
    e_jac = np.linalg.norm(got - want) / np.linalg.norm(want)
    e = max(e_solve, e_jac)
    return e if np.isfinite(e) else np.inf


SOLVER_MUTATIONS = {
    "jacobi_sign": [('G = G + op.apply_site_diagonal', 'G = G - op.apply_site_diagonal')],
    "jacobi_no_inverse": [('op.apply_site_diagonal(U - op.apply(G), inverse=True)',
                           '(U - op.apply(G))')],
    "gram_no_conj": [('A.reshape(-1, L).conj().T @ B', 'A.reshape(-1, L).T @ B')],
    "gram_transposed": [('return A.reshape(-1, L).conj().T @ B.reshape(-1, L)',
                         'return B.reshape(-1, L).conj().T @ A.reshape(-1, L)')],
    "right_multiply_transposed": [('(X.reshape(-1, L) @ C)', '(X.reshape(-1, L) @ C.T)')],
    "alpha_system_swapped": [('solve_small(herm_product(Rt, V), herm_product(Rt, R))',
                              'solve_small(herm_product(Rt, R), herm_product(Rt, V))')],
    "zeta_conjugated": [('zeta = np.vdot(W, R) / ww', 'zeta = np.vdot(R, W) / ww')],
    "s_sign": [('S = P - zeta * V', 'S = P + zeta * V')],
    "x_update_drops_zeta": [('return X + zeta * F + G, R', 'return X + F + G, R')],
    "r_update_sign": [('R - zeta * W - Y', 'R - zeta * W + Y')],
    "gamma_missing_zeta": [('herm_product(Rt, R_new) / zeta)', 'herm_product(Rt, R_new))')],
    "p_update_uses_y": [('return R_new + right_multiply(Uk, gamma)',
                         'return R_new + right_multiply(Y, gamma)')],
    "v_update_uses_u": [('W_new + right_multiply(Y, gamma)', 'W_new + right_multiply(Uk, gamma)')],
    "w_not_refreshed": [('W = A(F)                                   # W_{k+1}',
                         'W = W                                      # W_{k+1}')],
}


def invariant_error(ns):
    dims = (2, 2, 2, 4)
    op = O.WilsonClover(I.random_links(dims, 0.4, 2), dims, 0.12, 1.2)
    B = I.z4_noise(dims, 3, seed=4)
    try:
        return pins.solver_invariant_error(ns["bbicggr"], op, B, j=2)
    except Exception:
        return np.inf


@pytest.mark.parametrize("kind", sorted(SOLVER_MUTATIONS))
def test_solver_mutation_is_caught(kind):
    ns = mutated_module(S, SOLVER_MUTATIONS[kind])
    assert max(solver_pin_error(ns), invariant_error(ns)) > PIN_TOL


def test_unmutated_solver_passes_pins():
    assert solver_pin_error(S.__dict__) < 1e-10
    assert invariant_error(S.__dict__) < 1e-10


# ---------------------------------------------------------------- network oracle mutations
from oracle import network as NET

NETWORK_MUTATIONS = {
    "adjoint_direction_not_swapped": [("return transport(U, lat, phi, d + 4 if d <= 4 else d - 4)",
                                       "return transport(U, lat, phi, d)")],
    "gradient_missing_conj": [('G[d, co, c] = np.einsum("vsal,vtal->st", delta[co], np.conj(t))',
                               'G[d, co, c] = np.einsum("vsal,vtal->st", delta[co], t)')],
    "adjoint_weight_not_conjugated": [('np.einsum("ts,vtal->vsal", np.conj(W[d, co, c]), delta[co])',
                                       'np.einsum("ts,vtal->vsal", W[d, co, c], delta[co])')],
    "backward_transport_wrong_link": [("_dag(U[lat.bwd[mu], mu]), psi[lat.bwd[mu]]",
                                       "_dag(U[:, mu]), psi[lat.bwd[mu]]")],
    "loss_not_normalised": [("delta = (diff / (L * en2))[None]", "delta = (diff / L)[None]")],
    "adam_no_bias_correction": [("mhat = m / (1 - beta1 ** t)", "mhat = m")],
}


def network_pin_error(ns):
    """Finite-difference gradient pin, gauge covariance and the Adam closed form, as in
    tests/test_oracle_network.py, on the mutated module."""
    import test_oracle_network as T
    errs = []
    U, lat, W, R, E = T.setup()
    try:
        loss, G = ns["loss_and_grad"](U, lat, W, R, E)
        h = 1e-6
        rng = np.random.default_rng(1)
        for li in range(len(W)):
            for _ in range(6):
                idx = tuple(rng.integers(0, s) for s in W[li].shape)
                Wp = [w.copy() for w in W]
                Wm = [w.copy() for w in W]
                Wp[li][idx] += h
                Wm[li][idx] -= h
                fd = (NET.loss_and_grad(U, lat, Wp, R, E)[0] - NET.loss_and_grad(U, lat, Wm, R, E)[0]) / (2 * h)
                errs.append(abs(fd - 2 * G[li][idx].real) / max(1.0, abs(fd)))
        errs.append(abs(loss - NET.loss_and_grad(U, lat, W, R, E)[0]))
    except Exception:
        return np.inf
    dims = (3, 2, 2, 4)
    Uc = I.random_links(dims, 0.5, seed=4)
    latc = O.Lattice(dims)
    Om = I.random_gauge_transform(dims, seed=5)
    Up = np.empty_like(Uc)
    for mu in range(4):
        Up[:, mu] = Om @ Uc[:, mu] @ np.conj(np.swapaxes(Om[latc.fwd[mu]], -1, -2))
    Wc = I.network_weights(4, 2, seed=3, noise=0.4)
    psi = I.gaussian_block(dims, 2, seed=6)
    rot = lambda z: np.einsum("vab,vsbl->vsal", Om, z)
    a = ns["forward"](Up, latc, Wc, rot(psi))[0]
    b = rot(ns["forward"](Uc, latc, Wc, psi)[0])
    errs.append(np.linalg.norm(a - b) / np.linalg.norm(b))
    Wa, Ga = [np.array([[1.0 + 2.0j]])], [np.array([[0.25 - 1.0j]])]
    na = ns["adam_step"](Wa, Ga, {}, 0.01, eps=1e-12)[0]
    errs.append(abs(na[0, 0] - (Wa[0][0, 0] - 0.01 + 0.01j)))
    return max(errs)


# central differences with h = 1e-6 leave ~1e-7 of truncation and rounding in the unmutated
# check, so the network pins separate mutations at 1e-4 instead of PIN_TOL
NET_PIN_TOL = 1e-4


@pytest.mark.parametrize("kind", sorted(NETWORK_MUTATIONS))
def test_network_mutation_is_caught(kind):
    ns = mutated_module(NET, NETWORK_MUTATIONS[kind])
    assert network_pin_error(ns) > NET_PIN_TOL


def test_unmutated_network_passes_pins():
    assert network_pin_error(NET.__dict__) < 1e-5


# ---------------------------------------------------------------- stored-operator oracle mutations
from oracle import stored as ST

STORED_MUTATIONS = {
    "splitting_kappa_sign": [("U + pieces.kappa * pieces.hopping(G)",
                              "U - pieces.kappa * pieces.hopping(G)")],
    "splitting_accumulates": [("G = pieces.apply_dinv(U", "G = G + pieces.apply_dinv(U")],
    "dinv_transposed": [('"vij,vjl->vil", self.Dinv', '"vji,vjl->vil", self.Dinv')],
    "hermitian_part_without_conj": [("0.5 * (blk + np.conj(np.swapaxes(blk, -1, -2)))",
                                     "0.5 * (blk + np.swapaxes(blk, -1, -2))")],
    "one_chirality_only": [("for c in (slice(0, 6), slice(6, 12)):", "for c in (slice(0, 6),):")],
    "links_not_rounded_kappa_squared": [("float(np.float32(op.kappa))",
                                         "float(np.float32(op.kappa)) ** 2")],
}


def stored_pin_error(ns):
    """The pins of tests/test_oracle_stored.py on the mutated module: exact pieces against the
    pinned polynomial, stored pieces against the dense polynomial on 2^4, and the size of the
    stored operator's rounding effect (FP32 level, not more)."""
    try:
        dims = (2, 3, 2, 3)
        op = O.WilsonClover(I.random_links(dims, 0.3, seed=2), dims, 0.12, 1.0)
        R = I.gaussian_block(dims, 2, seed=5)
        e1 = pins.rel(ns["jacobi_splitting"](ns["exact_pieces"](op), R, 3), S.jacobi(op, R, 3))
        d2 = (2, 2, 2, 2)
        op2 = O.WilsonClover(I.random_links(d2, 0.3, seed=0), d2, 0.125, 1.0)
        pc = ns["fp32_pieces"](op2)
        H = pins.dense_hopping_from_entries(pc.U, d2)
        D = pins.block_diagonal(pc.Dinv)
        u = I.gaussian_block(d2, 2, seed=7).reshape(op2.N, 2)
        want = D @ u + pc.kappa * D @ H @ (D @ u)
        got = ns["jacobi_splitting"](pc, u.reshape(op2.lat.V, 4, 3, 2), 2).reshape(op2.N, 2)
        e2 = pins.rel(got, want)
        r32 = pins.rel(ns["jacobi_splitting"](pc, u.reshape(op2.lat.V, 4, 3, 2), 4),
                       S.jacobi(op2, u.reshape(op2.lat.V, 4, 3, 2), 4))
        e3 = 0.0 if r32 < 1e-6 else np.inf
        e = max(e1, e2, e3)
        return e if np.isfinite(e) else np.inf
    except Exception:
        return np.inf


@pytest.mark.parametrize("kind", sorted(STORED_MUTATIONS))
def test_stored_mutation_is_caught(kind):
    ns = mutated_module(ST, STORED_MUTATIONS[kind])
    assert stored_pin_error(ns) > PIN_TOL


def test_unmutated_stored_passes_pins():
    assert stored_pin_error(ST.__dict__) < 1e-13
