"""Low-precision preconditioner: BF16 block storage and the 12-real link format, against the FP64
oracle through the C-ABI (needs a GB300)."""
import numpy as np
import pytest

from oracle import operator as O
from oracle import solver as S
from paper_0907_3261_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SOLVE_X_TOL = 1e-9
TRUE_RES_TOL = 1e-12
MIXED_TOL = 1e-5     # FP32 sweeps (derivation beside the FP32 tests in test_gpu_parity.py)
BF16_U = 2.0 ** -8   # unit roundoff of BF16: 8 significant bits, round to nearest even


def bf16_tol(j):
    """Relative error bound of j sweeps on BF16-stored blocks.  The copy of U and every sweep's
    output are rounded to BF16 once (relative error <= u per real component, so <= u in norm);
    FP32 arithmetic adds ~1e-5 at most.  An error made in sweep i reaches the result through the
    Jacobi iteration matrix, which contracts at the kappa values tested, so the j + 1 roundings add
    up to at most (j + 1) u."""
    return (j + 1) * BF16_U


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
    return np.linalg.norm(a - b) / np.linalg.norm(b)


# ---------------------------------------------------------------- link format
def test_link_format_follows_the_links(wd):
    """SU(3) links give the 12-real format; links with a U(1) phase (unitary, det != 1) fail the
    row-2 check and give 18 reals.  Both formats reproduce the oracle's Jacobi polynomial."""
    dims, L, j = (3, 4, 5, 6), 4, 5
    links = I.random_links(dims, 0.4, seed=2)
    R = I.gaussian_block(dims, L, seed=5)
    ctx = wd.wd_create(dev(links), dims, 0.12, 1.0)
    assert wd.wd_link_reals(ctx) == 12
    ref = S.jacobi(O.WilsonClover(links, dims, 0.12, 1.0), R, j)
    G12 = host(wd.jacobi_precond(ctx, dev(R), j, precision=1))
    wd.wd_set_link_reals(ctx, 18)
    assert wd.wd_link_reals(ctx) == 18
    G18 = host(wd.jacobi_precond(ctx, dev(R), j, precision=1))
    assert rel(G12, ref) <= MIXED_TOL and rel(G18, ref) <= MIXED_TOL
    assert rel(G12, G18) <= MIXED_TOL
    with pytest.raises(wd.WDError):
        wd.wd_set_link_reals(ctx, 9)

    phased = links * np.exp(0.3j)
    ctx2 = wd.wd_create(dev(phased), dims, 0.12, 1.0)
    assert wd.wd_link_reals(ctx2) == 18
    with pytest.raises(wd.WDError):
        wd.wd_set_link_reals(ctx2, 12)
    ref2 = S.jacobi(O.WilsonClover(phased, dims, 0.12, 1.0), R, j)
    assert rel(host(wd.jacobi_precond(ctx2, dev(R), j, precision=1)), ref2) <= MIXED_TOL
    assert rel(host(wd.jacobi_precond(ctx2, dev(R), j, precision=3)), ref2) <= bf16_tol(j)


# ---------------------------------------------------------------- BF16 storage (precision 3)
@pytest.mark.parametrize("j", [1, 2, 5, 12])
@pytest.mark.parametrize("dims,L", [((4, 4, 4, 4), 4), ((3, 4, 5, 6), 7), ((8, 8, 8, 16), 12)])
def test_jacobi_bf16_matches_oracle(wd, j, dims, L):
    links = I.random_links(dims, 0.3, seed=2)
    op = O.WilsonClover(links, dims, 0.12, 1.0)
    R = I.gaussian_block(dims, L, seed=5)
    ctx = wd.wd_create(dev(links), dims, 0.12, 1.0)
    G = host(wd.jacobi_precond(ctx, dev(R), j, precision=3))
    G_ref = S.jacobi(op, R, j)
    err = rel(G, G_ref)
    assert err <= bf16_tol(j)
    assert err > 10 * MIXED_TOL   # the blocks really are BF16: well above FP32 rounding
    assert np.abs(G - G_ref).max() / np.abs(G_ref).max() <= bf16_tol(j)


TILES = [(1, 64, 0, 0), (1, 128, 0, 0), (1, 256, 0, 0), (2, 64, 0, 0), (2, 128, 0, 0),
         (2, 256, 0, 0), (0, 128, 0, 0), (2, 64, 8, 0), (1, 64, 8, 0), (2, 64, 0, 1),
         (1, 64, 12, 0)]


@pytest.mark.parametrize("tile", TILES)
def test_bf16_sweep_tiles_match_oracle(wd, tile):
    dims, L, j = (3, 4, 5, 6), 6, 5
    links = I.random_links(dims, 0.4, seed=2)
    op = O.WilsonClover(links, dims, 0.12, 1.0)
    R = I.gaussian_block(dims, L, seed=5)
    ctx = wd.wd_create(dev(links), dims, 0.12, 1.0)
    wd.wd_set_tile(ctx, L, *tile, precision=3)
    G = host(wd.jacobi_precond(ctx, dev(R), j, precision=3))
    assert wd.wd_tuned_tile(ctx, L, precision=3) == tile
    assert wd.wd_tuned_tile(ctx, L, precision=1) is None    # separate tables per storage
    assert rel(G, S.jacobi(op, R, j)) <= bf16_tol(j)


def test_bf16_autotuner_and_ragged_L(wd):
    dims, L = (4, 4, 4, 8), 3
    links = I.random_links(dims, 0.3, seed=0)
    ctx = wd.wd_create(dev(links), dims, 0.12, 1.0)
    R = I.z4_noise(dims, L, seed=1)
    G = host(wd.jacobi_precond(ctx, dev(R), 4, precision=3))
    r, b, m, st = wd.wd_tuned_tile(ctx, L, precision=3)
    assert (r, b, m, st) in TILES and r != 2          # L = 3 admits no 2-RHS tile
    assert rel(G, S.jacobi(O.WilsonClover(links, dims, 0.12, 1.0), R, 4)) <= bf16_tol(4)
    with pytest.raises(wd.WDError):
        wd.jacobi_precond(ctx, dev(R), 4, precision=2)   # 2 is a solver option, not a storage


@pytest.mark.parametrize("B_kind,L,j", [("point", 4, 4), ("z4", 12, 4), ("z4", 3, 1)])
def test_bf16_solve_matches_fp64_oracle(wd, B_kind, L, j):
    """BF16 storage changes M only: the FP64 outer recurrences still reach the FP64 solution,
    falling back to the FP64 preconditioner if the BF16 one stalls."""
    dims = (4, 4, 4, 4)
    links = I.random_links(dims, 0.3, seed=0)
    op = O.WilsonClover(links, dims, 0.115, 1.0)
    B = I.point_sources(dims, L) if B_kind == "point" else I.z4_noise(dims, L, seed=1)
    ref = S.solve(op, B, j=j, tol=1e-12)
    ctx = wd.wd_create(dev(links), dims, 0.115, 1.0)
    Xg, info = wd.bbicggr_solve(ctx, dev(B), j=j, tol=1e-12, precision=3)
    Xg = host(Xg)
    assert info["status"] == wd.WD_OK
    assert info["fallbacks"] in (0, 1)
    assert S.true_residual(op, B, Xg).max() <= TRUE_RES_TOL
    assert rel(Xg, ref.X) <= SOLVE_X_TOL


def test_bf16_solve_8_8_8_16(wd):
    dims = (8, 8, 8, 16)
    links = I.random_links(dims, 0.2, seed=0)
    op = O.WilsonClover(links, dims, 0.125, 1.0)
    B = I.z4_noise(dims, 12, seed=1)
    ctx = wd.wd_create(dev(links), dims, 0.125, 1.0)
    X64, i64 = wd.bbicggr_solve(ctx, dev(B), j=12, tol=1e-12)
    X16, i16 = wd.bbicggr_solve(ctx, dev(B), j=12, tol=1e-12, precision=3)
    assert i64["status"] == i16["status"] == wd.WD_OK
    assert S.true_residual(op, B, host(X16)).max() <= TRUE_RES_TOL
    assert rel(host(X16), host(X64)) <= SOLVE_X_TOL


# ---------------------------------------------------------------- double-float sweeps (precision 4)
# The operator (links, A_D^{-1}, kappa) is stored in FP32, so M is the Jacobi polynomial of an
# operator whose entries carry FP32 rounding: the same 1e-5 bound as the FP32 sweeps applies.  The
# spinor arithmetic is double-float (~2^-48 per operation), so M is linear to ~1e-13: about 100
# terms per component and sweep at 2^-48 = 3.6e-15, over j <= 12 sweeps.
DF_LINEARITY_TOL = 1e-12


@pytest.mark.parametrize("j", [1, 2, 5, 12])
@pytest.mark.parametrize("dims,L", [((4, 4, 4, 4), 4), ((3, 4, 5, 6), 7), ((8, 8, 8, 16), 12)])
def test_jacobi_df_matches_oracle(wd, j, dims, L):
    links = I.random_links(dims, 0.3, seed=2)
    op = O.WilsonClover(links, dims, 0.12, 1.0)
    R = I.gaussian_block(dims, L, seed=5)
    ctx = wd.wd_create(dev(links), dims, 0.12, 1.0)
    G = host(wd.jacobi_precond(ctx, dev(R), j, precision=4))
    G_ref = S.jacobi(op, R, j)
    assert rel(G, G_ref) <= MIXED_TOL
    assert np.abs(G - G_ref).max() / np.abs(G_ref).max() <= MIXED_TOL


def nonlinearity(wd, ctx, x, y, j, precision):
    """|| M(a x + b y) - (a M(x) + b M(y)) || / || M(a x + b y) || for complex a, b."""
    a, b = 0.7 - 0.4j, -1.3 + 0.2j
    z = a * x + b * y
    Mz = host(wd.jacobi_precond(ctx, dev(z), j, precision=precision))
    Mx = host(wd.jacobi_precond(ctx, dev(x), j, precision=precision))
    My = host(wd.jacobi_precond(ctx, dev(y), j, precision=precision))
    return rel(a * Mx + b * My, Mz)


@pytest.mark.parametrize("dims,L,j", [((4, 4, 4, 8), 6, 12), ((16, 16, 16, 32), 12, 12)])
def test_df_preconditioner_is_linear(wd, dims, L, j):
    """Double-float M is linear to ~1e-13 at any size, in every double-float tile, FP32 M only
    to ~1e-7 -- the property block BiCGGR relies on (the test also shows that it tells the two
    apart)."""
    links = I.random_links(dims, 0.2, seed=0)
    ctx = wd.wd_create(dev(links), dims, 0.134, 1.0)
    x = I.z4_noise(dims, L, seed=3)
    y = I.gaussian_block(dims, L, seed=4)
    for tile in ((1, 128, 0, 0), (1, 128, 0, 1), (1, 128, 0, 2)):
        wd.wd_set_tile(ctx, L, *tile, precision=4)
        assert nonlinearity(wd, ctx, x, y, j, 4) <= DF_LINEARITY_TOL
    assert nonlinearity(wd, ctx, x, y, j, 1) > 100 * DF_LINEARITY_TOL


@pytest.mark.parametrize("tile", [(1, 128, 0, 0), (1, 128, 0, 1), (1, 128, 0, 2)])
def test_df_preconditioner_scales_exactly(wd, tile):
    """The FP64 <-> double-float conversions work from the IEEE bit fields (exponent, fraction).
    Scaling the input by 2^k, with every value and intermediate still a normal FP32 number, scales
    each rounding step exactly, so M(2^k R) = 2^k M(R) bit for bit; M(0) = 0.  A wrong exponent
    bias or fraction shift in either conversion breaks the equality."""
    dims, L, j = (4, 4, 4, 8), 5, 4
    links = I.random_links(dims, 0.3, seed=1)
    ctx = wd.wd_create(dev(links), dims, 0.125, 1.0)
    wd.wd_set_tile(ctx, L, *tile, precision=4)
    R = I.gaussian_block(dims, L, seed=6)
    G = host(wd.jacobi_precond(ctx, dev(R), j, precision=4))
    for k in (-30, -7, 9, 60):
        Gk = host(wd.jacobi_precond(ctx, dev(R * 2.0 ** k), j, precision=4))
        assert np.array_equal(Gk, G * 2.0 ** k), k
    Z = host(wd.jacobi_precond(ctx, dev(np.zeros_like(R)), j, precision=4))
    assert not Z.any()


@pytest.mark.parametrize("precision", [4, 5])
@pytest.mark.parametrize("B_kind,L,j", [("point", 4, 4), ("z4", 12, 4), ("z4", 3, 1)])
def test_df_solve_matches_fp64_oracle(wd, B_kind, L, j, precision):
    """precision 4: double-float sweeps; 5: also double-float direction recurrences."""
    dims = (4, 4, 4, 4)
    links = I.random_links(dims, 0.3, seed=0)
    op = O.WilsonClover(links, dims, 0.115, 1.0)
    B = I.point_sources(dims, L) if B_kind == "point" else I.z4_noise(dims, L, seed=1)
    ref = S.solve(op, B, j=j, tol=1e-12)
    ctx = wd.wd_create(dev(links), dims, 0.115, 1.0)
    Xg, info = wd.bbicggr_solve(ctx, dev(B), j=j, tol=1e-12, precision=precision)
    Xg = host(Xg)
    assert info["status"] == wd.WD_OK and info["fallbacks"] == 0
    assert S.true_residual(op, B, Xg).max() <= TRUE_RES_TOL
    assert rel(Xg, ref.X) <= SOLVE_X_TOL
    assert abs(info["iters"] - ref.iters) <= max(2, ref.iters // 10)


def test_df_solve_near_critical_needs_no_fallback(wd):
    """Near the critical kappa, where the FP32 preconditioner stalls block BiCGGR and falls back
    to FP64, the double-float preconditioner converges like the FP64 one."""
    dims = (6, 6, 6, 6)
    links = I.random_links(dims, 0.2, seed=0)
    op = O.WilsonClover(links, dims, 0.134, 1.0)
    B = I.z4_noise(dims, 4, seed=1)
    ctx = wd.wd_create(dev(links), dims, 0.134, 1.0)
    X64, i64 = wd.bbicggr_solve(ctx, dev(B), j=4, tol=1e-12, maxit=2000)
    Xdf, idf = wd.bbicggr_solve(ctx, dev(B), j=4, tol=1e-12, precision=4, maxit=2000)
    assert i64["status"] == idf["status"] == wd.WD_OK
    assert idf["fallbacks"] == 0
    assert idf["iters"] <= i64["iters"] + 5
    assert S.true_residual(op, B, host(Xdf)).max() <= TRUE_RES_TOL
    assert rel(host(Xdf), host(X64)) <= SOLVE_X_TOL


@pytest.mark.parametrize("tile", [(1, 128, 0, 0), (2, 128, 0, 0), (1, 128, 0, 1), (1, 128, 0, 2)])
def test_df_sweep_tiles_match_oracle(wd, tile):
    """Both double-float tiles (1 or 2 RHS per thread) compute the same sweep, and the autotuner
    keeps one of them."""
    dims, L, j = (3, 4, 5, 6), 6, 5
    links = I.random_links(dims, 0.4, seed=2)
    op = O.WilsonClover(links, dims, 0.12, 1.0)
    R = I.gaussian_block(dims, L, seed=5)
    ctx = wd.wd_create(dev(links), dims, 0.12, 1.0)
    wd.wd_set_tile(ctx, L, *tile, precision=4)
    G = host(wd.jacobi_precond(ctx, dev(R), j, precision=4))
    assert wd.wd_tuned_tile(ctx, L, precision=4) == tile
    assert rel(G, S.jacobi(op, R, j)) <= MIXED_TOL
    ctx2 = wd.wd_create(dev(links), dims, 0.12, 1.0)
    G2 = host(wd.jacobi_precond(ctx2, dev(R), j, precision=4))
    assert wd.wd_tuned_tile(ctx2, L, precision=4) in ((1, 128, 0, 0), (2, 128, 0, 0),
                                                     (1, 128, 0, 1), (1, 128, 0, 2))
    assert rel(G2, G) <= 1e-13          # the tiles differ only in the order of operations
    with pytest.raises(wd.WDError):
        wd.wd_set_tile(ctx, 3, 2, 128, precision=4)     # 2 does not divide L = 3
    with pytest.raises(wd.WDError):
        wd.wd_set_tile(ctx, 4, 2, 128, 0, 1, precision=4)   # the packed variant takes 1 RHS


@pytest.mark.parametrize("L", [1, 4, 12])
@pytest.mark.parametrize("kappa", [0.125, 0.134])
def test_df_dirs_form_across_L_and_kappa(wd, L, kappa):
    """The default form (precision 5) on 8^3 x 16 for several L and kappa up to the bench's
    near-critical value: oracle true residual <= 1e-12 per column, no fallback, and the FP64
    form's solution to 1e-9."""
    dims = (8, 8, 8, 16)
    links = I.random_links(dims, 0.2, seed=0)
    op = O.WilsonClover(links, dims, kappa, 1.0)
    B = I.z4_noise(dims, L, seed=3)
    ctx = wd.wd_create(dev(links), dims, kappa, 1.0)
    X5, i5 = wd.bbicggr_solve(ctx, dev(B), j=12, tol=1e-12, precision=5)
    X0, i0 = wd.bbicggr_solve(ctx, dev(B), j=12, tol=1e-12, precision=0)
    assert i5["status"] == i0["status"] == wd.WD_OK
    assert i5["fallbacks"] == 0
    X5 = host(X5)
    assert S.true_residual(op, B, X5).max() <= TRUE_RES_TOL
    assert rel(X5, host(X0)) <= SOLVE_X_TOL


def test_fp64_solve_scales_exactly(wd):
    """Every step of the FP64 solver is scale-covariant: the stopping, pivot and stall tests are
    relative, and scaling B by 2^k scales each FP64 rounding step exactly.  So X(2^k B) = 2^k X(B)
    bit for bit with the same iteration count.  (The double-float forms are left out: their
    bit-field conversion keeps the full low word only for |value| >= 2^-79, so a solve scaled far
    down rounds its smallest block entries differently, though it still converges.)"""
    dims, L = (4, 4, 4, 8), 4
    links = I.random_links(dims, 0.3, seed=1)
    ctx = wd.wd_create(dev(links), dims, 0.125, 1.0)
    B = I.z4_noise(dims, L, seed=2)
    X1, i1 = wd.bbicggr_solve(ctx, dev(B), j=4, tol=1e-12, precision=0)
    X1 = host(X1)
    assert i1["status"] == wd.WD_OK
    for k in (-30, 40):
        Xk, ik = wd.bbicggr_solve(ctx, dev(B * 2.0 ** k), j=4, tol=1e-12, precision=0)
        assert ik["iters"] == i1["iters"], k
        assert np.array_equal(host(Xk), X1 * 2.0 ** k), k


def test_precision2_solve_scaled_far_down(wd):
    """B scaled by 2^-30: the double-float direction recurrences (precision 2) still converge in
    the unscaled iteration count to true residual <= 1e-12; their bit-field conversion keeps a
    full low word down to |value| 2^-79, far below the entries of this solve."""
    dims, L = (4, 4, 4, 8), 4
    links = I.random_links(dims, 0.3, seed=1)
    op = O.WilsonClover(links, dims, 0.125, 1.0)
    ctx = wd.wd_create(dev(links), dims, 0.125, 1.0)
    B = I.z4_noise(dims, L, seed=2)
    X1, i1 = wd.bbicggr_solve(ctx, dev(B), j=4, tol=1e-12, precision=2)
    Bk = B * 2.0 ** -30
    Xk, ik = wd.bbicggr_solve(ctx, dev(Bk), j=4, tol=1e-12, precision=2)
    assert i1["status"] == ik["status"] == wd.WD_OK
    assert ik["fallbacks"] == 0
    assert ik["iters"] == i1["iters"]
    assert S.true_residual(op, Bk, host(Xk)).max() <= TRUE_RES_TOL
