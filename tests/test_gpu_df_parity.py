"""The double-float kernels against the oracle at their own precision (needs a GB300).

The double-float Jacobi sweeps keep the operator in FP32 (links, A_D^{-1}, kappa) and carry the
spinors as FP32 pairs.  Compared with the FP64 operator they can only agree to FP32 rounding, which
an FP32 kernel would also meet.  So here the oracle gets the operator the kernels store
(oracle/stored.py: links rounded to complex64 -- all 18 reals, the sweeps told to read 18 --,
each 6 x 6 block of A_D^{-1} as its Hermitian part rounded to complex64, kappa as float32) and
computes the Jacobi splitting of Sec. 2 in FP64.  The kernels' own arithmetic is then the only
difference, and it is held to 1e-12 of the largest |G| element by element: about 60 products and
additions per component and sweep at ~2^-47 each, over at most 12 sweeps of a contracting
iteration.  An error in the low words of any one term (a wrong sign in one projector entry of the
correction, a dropped rounding error) is of order 2^-24 ~ 6e-8 and fails by four orders.

The update kernels of the direction recurrences (bb_update_u, bb_update_xr, bb_update_pv, with
precision 1 = double-float products) are compared with the oracle's restatement of the algorithm
box's updates element by element, against the dot-product error bound of their arithmetic.
"""
import functools

import numpy as np
import pytest

from oracle import operator as O
from oracle import solver as S
from oracle import stored as ST
from paper_0907_3261_gb300 import inputs as I
import pins

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DF_ELEMENT_TOL = 1e-12        # max |G - G_oracle| / max |G_oracle|
U_DF = 2.0 ** -47             # per-operation error of the double-float arithmetic (~2 x 2^-48)
U_64 = 2.0 ** -53
# The FP64 A_D^{-1} the library builds (Gauss-Jordan, FP64) and the oracle's (LAPACK) differ by a
# few FP64 ulps of the block's scale; an entry closer than this to an FP32 rounding midpoint could
# round differently on the two sides, so such lattices are not used (see stored_case).
INVERSE_MARGIN = 1e-14
# scalar 1 RHS, scalar 2 RHS, packed, packed with grid sums
TILES = [(1, 128, 0, 0), (2, 128, 0, 0), (1, 128, 0, 1), (1, 128, 0, 2)]


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


def herm_blocks(op):
    """The Hermitian parts of the two 6 x 6 blocks of A_D^{-1}, the values both sides round."""
    out = []
    for c in (slice(0, 6), slice(6, 12)):
        blk = op.AD_inv[:, c, c]
        out.append(0.5 * (blk + np.conj(np.swapaxes(blk, -1, -2))))
    return np.stack(out)


def inverse_is_safe(op):
    if op.csw == 0.0:
        return True                   # A_D^{-1} = 1 exactly on both sides
    h = herm_blocks(op)
    x, d = pins.fp32_midpoint_distance(h)
    return d.min() > INVERSE_MARGIN * np.abs(h).max()


@functools.lru_cache(maxsize=None)
def stored_case(dims, csw, kappa=0.125):
    """(links, R, oracle operator) with the first link seed from 2 whose A_D^{-1} blocks keep every
    real part INVERSE_MARGIN away from an FP32 rounding midpoint."""
    L = 12 if np.prod(dims) >= 4096 else 6
    for seed in range(2, 40):
        links = I.random_links(dims, 0.3, seed=seed)
        op = O.WilsonClover(links, dims, kappa, csw)
        if inverse_is_safe(op):
            return links, I.gaussian_block(dims, L, seed=5), op
    raise AssertionError("no safe link seed")


@functools.lru_cache(maxsize=None)
def stored_oracle(dims, csw, j):
    links, R, op = stored_case(dims, csw)
    return ST.jacobi_splitting(ST.fp32_pieces(op), R, j)


def element_error(G, ref):
    return np.abs(G - ref).max() / np.abs(ref).max()


@pytest.mark.parametrize("tile", TILES)
@pytest.mark.parametrize("j", [1, 2, 12])
@pytest.mark.parametrize("csw", [0.0, 1.0])
@pytest.mark.parametrize("dims", [(3, 4, 5, 6), (4, 4, 4, 4)])
def test_df_sweeps_match_the_stored_operator_oracle(wd, dims, csw, j, tile):
    links, R, op = stored_case(dims, csw)
    L = R.shape[-1]
    ctx = wd.wd_create(dev(links), dims, op.kappa, csw)
    wd.wd_set_link_reals(ctx, 18)
    wd.wd_set_tile(ctx, L, *tile, precision=4)
    G = host(wd.jacobi_precond(ctx, dev(R), j, precision=4))
    ref = stored_oracle(dims, csw, j)
    assert element_error(G, ref) <= DF_ELEMENT_TOL, (element_error(G, ref), tile)
    # against the FP64 operator the same G is only FP32-close: the test sees the difference
    if csw:
        full = S.jacobi(op, R, j)
        assert element_error(G, full) > 1e3 * DF_ELEMENT_TOL
    wd.wd_destroy(ctx)


@pytest.mark.parametrize("tile", TILES)
@pytest.mark.parametrize("j", [2, 12])
def test_df_sweeps_8x8x8x16(wd, j, tile):
    """8^3 x 16, L = 12, c_SW = 0 (exact unit A_D^{-1}, so only the links and kappa are rounded)."""
    dims = (8, 8, 8, 16)
    links, R, op = stored_case(dims, 0.0)
    ctx = wd.wd_create(dev(links), dims, op.kappa, 0.0)
    wd.wd_set_link_reals(ctx, 18)
    wd.wd_set_tile(ctx, 12, *tile, precision=4)
    G = host(wd.jacobi_precond(ctx, dev(R), j, precision=4))
    assert element_error(G, stored_oracle(dims, 0.0, j)) <= DF_ELEMENT_TOL
    wd.wd_destroy(ctx)


def test_df_sweeps_full_size_16x16x16x32(wd):
    """The bench lattice and L = 12 in the tile the autotuner picks, two sweeps."""
    dims, j = (16, 16, 16, 32), 2
    links, R, op = stored_case(dims, 0.0, kappa=0.134)
    ctx = wd.wd_create(dev(links), dims, op.kappa, 0.0)
    wd.wd_set_link_reals(ctx, 18)
    G = host(wd.jacobi_precond(ctx, dev(R), j, precision=4))
    assert wd.wd_tuned_tile(ctx, 12, precision=4) in TILES
    ref = ST.jacobi_splitting(ST.fp32_pieces(op), R, j)
    assert element_error(G, ref) <= DF_ELEMENT_TOL
    wd.wd_destroy(ctx)


# ---------------------------------------------------------------- update kernels
def update_inputs(dims, L, seed):
    blocks = [I.gaussian_block(dims, L, seed=seed + i) for i in range(9)]
    c = I.complex_gaussian(seed, 77, 2 * L * L + 1)
    return blocks, c[:L * L].reshape(L, L), c[L * L:2 * L * L].reshape(L, L), c[-1]


def bound(A, C, u, L):
    """Dot-product error bound of (A C)[n, b] = sum_a A[n, a] C[a, b]: (L + 4) u sum |terms|."""
    An = np.abs(A.reshape(-1, L))
    return (L + 4) * u * (An @ np.abs(C))


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("dims,L", [((3, 4, 5, 6), 7), ((8, 8, 8, 16), 12)])
def test_update_kernels_match_the_oracle_restatement(wd, dims, L, precision):
    (P, V, X, F, G, R, W, Y, Rt), alpha, gamma, zeta = update_inputs(dims, L, seed=21)
    links = I.random_links(dims, 0.2, seed=0)
    ctx = wd.wd_create(dev(links), dims, 0.12, 1.0)
    u = U_DF if precision else U_64
    N = 12 * int(np.prod(dims))

    # U = (P - zeta V) alpha
    Ud = dev(np.zeros_like(P))
    wd.bb_update_u(ctx, dev(P), dev(V), Ud, zeta, alpha, precision=precision)
    U_ref = S.direction_u(P, V, zeta, alpha)
    Sabs = np.abs(P) + np.abs(zeta) * np.abs(V)
    err = np.abs(host(Ud) - U_ref).reshape(N, L)
    assert (err <= bound(Sabs, alpha, u, L) + 4 * u * np.abs(U_ref.reshape(N, L))).all()
    assert err.max() / np.abs(U_ref).max() <= 1e-13

    # X += zeta F + G, R -= zeta W + Y, R~_0^H R, ||r_i||^2 (the X, R updates are FP64 always)
    Xd, Rd = dev(X), dev(R)
    rtr, nrm = wd.bb_update_xr(ctx, Xd, dev(F), dev(G), Rd, dev(W), dev(Y), dev(Rt), zeta,
                               precision=precision)
    X_ref, R_ref = S.solution_update(X, R, F, G, W, Y, zeta)
    for got, ref, a, b in ((host(Xd), X_ref, F, G), (host(Rd), R_ref, W, Y)):
        lim = 8 * U_64 * (np.abs(ref) + np.abs(zeta) * np.abs(a) + np.abs(b))
        assert (np.abs(got - ref) <= lim).all()
    gram_ref = S.herm_product(Rt, R_ref)
    gram_lim = 2.0 ** -40 * (np.abs(Rt.reshape(N, L)).T @ np.abs(R_ref.reshape(N, L)))
    assert (np.abs(rtr - gram_ref) <= gram_lim).all()
    assert np.allclose(nrm, S.column_norms(R_ref) ** 2, rtol=1e-13, atol=0)

    # P = R + U gamma, V = W + Y gamma, R~_0^H V
    Pd, Vd = dev(np.zeros_like(P)), dev(np.zeros_like(V))
    rtv = wd.bb_update_pv(ctx, Pd, Vd, dev(R_ref), dev(W), dev(U_ref), dev(Y), dev(Rt), gamma,
                          precision=precision)
    P_ref, V_ref = S.direction_pv(R_ref, U_ref, W, Y, gamma)
    for got, ref, base, M in ((host(Pd), P_ref, R_ref, U_ref), (host(Vd), V_ref, W, Y)):
        err = np.abs(got - ref).reshape(N, L)
        lim = bound(M, gamma, u, L) + 4 * u * (np.abs(ref) + np.abs(base)).reshape(N, L)
        assert (err <= lim).all()
        assert err.max() / np.abs(ref).max() <= 1e-13
    gv_ref = S.herm_product(Rt, V_ref)
    gv_lim = 2.0 ** -40 * (np.abs(Rt.reshape(N, L)).T @ np.abs(V_ref.reshape(N, L)))
    assert (np.abs(rtv - gv_ref) <= gv_lim).all()
    wd.wd_destroy(ctx)


def test_update_entry_points_reject_host_blocks_and_bad_precision(wd):
    dims, L = (2, 2, 2, 4), 3
    ctx = wd.wd_create(dev(I.random_links(dims, 0.2, seed=0)), dims, 0.12, 1.0)
    P = I.gaussian_block(dims, L, seed=1)
    with pytest.raises(wd.WDError):
        wd.bb_update_u(ctx, P, P.copy(), np.zeros_like(P), 0.5, np.eye(L))
    with pytest.raises(wd.WDError):
        wd.bb_update_u(ctx, dev(P), dev(P), dev(P), 0.5, np.eye(L), precision=2)
    wd.wd_destroy(ctx)


def test_grid_sum_tile_needs_unitary_links(wd):
    """The grid-sum sweep bounds each hop's partial sums by the largest projected spinor entry,
    which needs link rows and columns of norm <= 1.  Links scaled by 1.1 are refused for it, and
    the autotuner does not pick it."""
    dims, L = (3, 4, 5, 6), 6
    links = I.random_links(dims, 0.3, seed=2) * 1.1
    ctx = wd.wd_create(dev(links), dims, 0.12, 1.0)
    with pytest.raises(wd.WDError):
        wd.wd_set_tile(ctx, L, 1, 128, 0, 2, precision=4)
    R = I.gaussian_block(dims, L, seed=5)
    G = host(wd.jacobi_precond(ctx, dev(R), 3, precision=4))
    assert wd.wd_tuned_tile(ctx, L, precision=4)[3] != 2
    op = O.WilsonClover(links, dims, 0.12, 1.0)
    assert element_error(G, S.jacobi(op, R, 3)) <= 1e-5
    wd.wd_destroy(ctx)
