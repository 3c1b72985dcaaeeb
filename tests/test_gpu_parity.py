"""CUDA path vs the FP64 oracle, through the C-ABI (needs a GB300)."""
import numpy as np
import pytest

from oracle import operator as O
from oracle import solver as S
from paper_0907_3261_gb300 import inputs as I
import pins

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

APPLY_TOL = 1e-12     # relative, wd_apply vs oracle
SOLVE_X_TOL = 1e-9    # ||X - X_oracle|| / ||X||
TRUE_RES_TOL = 1e-12  # per column
# FP32 Jacobi sweeps: each sweep sums ~100 FP32 products per component (8 hops x 2 x 3 colour
# terms, the 6x6 inverse block); with unit roundoff 2^-24 = 6e-8 the worst-case relative error of a
# sweep is ~100 x 6e-8 = 6e-6, and later sweeps carry earlier errors forward contracted by the
# Jacobi iteration matrix.  1e-5 bounds j <= 12 sweeps at the kappa values tested.
MIXED_TOL = 1e-5


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


def max_elem_rel(a, b):
    """Largest entry-wise difference relative to the largest entry of the reference."""
    return np.abs(a - b).max() / np.abs(b).max()


class GpuOp:
    """The CUDA operator behind the pins' interface (apply only)."""

    def __init__(self, wd, links, dims, kappa, csw):
        self.ctx = wd.wd_create(dev(links), dims, kappa, csw)
        self.wd = wd

    def apply(self, psi):
        return host(self.wd.wd_apply(self.ctx, dev(psi)))


CASES = [((4, 4, 4, 4), 4, 0.3, 0.115, 1.0),     # the 4^4 point-source workload
         ((2, 2, 2, 2), 3, 0.5, 0.125, 1.3),     # forward and backward neighbours coincide
         ((3, 4, 5, 6), 5, 0.6, 0.13, 1.7),      # odd extents, ragged last block
         ((8, 8, 8, 16), 12, 0.2, 0.12, 1.0),    # 8^3 x 16, L = 12
         ((4, 4, 4, 8), 1, 0.3, 0.12, 1.0),      # L = 1
         ((2, 4, 2, 4), 16, 0.4, 0.12, 1.0)]     # L = WD_LMAX


@pytest.mark.parametrize("dims,L,eps,kappa,csw", CASES)
def test_wd_apply_matches_oracle(wd, dims, L, eps, kappa, csw):
    links = I.random_links(dims, eps, seed=0)
    op = O.WilsonClover(links, dims, kappa, csw)
    X = I.gaussian_block(dims, L, seed=3)
    ctx = wd.wd_create(dev(links), dims, kappa, csw)
    Y = host(wd.wd_apply(ctx, dev(X)))
    Y_ref = op.apply(X)
    assert rel(Y, Y_ref) <= APPLY_TOL
    assert max_elem_rel(Y, Y_ref) <= APPLY_TOL


def test_wd_apply_host_buffers_match_device(wd):
    dims = (3, 4, 5, 6)
    links = I.random_links(dims, 0.5, seed=1)
    X = I.gaussian_block(dims, 6, seed=4)
    ctx = wd.wd_create(links, dims, 0.12, 1.2)           # links from host memory
    Yh = wd.wd_apply(ctx, X)                              # host in, host out
    Yd = host(wd.wd_apply(ctx, dev(X)))
    assert np.array_equal(Yh, Yd)


def test_gpu_operator_satisfies_pins(wd):
    make = lambda U, d, k, c: GpuOp(wd, U, d, k, c)
    assert pins.free_field_error(make) < 1e-13
    assert pins.free_field_error(make, dims=(3, 5, 4, 6), n=(1, 2, 1, 5)) < 1e-13
    assert pins.gamma5_hermiticity_error(make) < 1e-13
    assert pins.gauge_covariance_error(make) < 1e-13


def test_gpu_clover_inverse_matches_the_abelian_flux_closed_form(wd):
    """Constant U(1) flux through every plaquette of one plane (pins.abelian_flux_links): the
    library's A_D must be 1 - kappa c_SW sigma_{mu nu} diag(sin phi, -sin phi, 0) exactly.  One
    Jacobi sweep from G = 0 applies the library's A_D^{-1}; it is compared with the inverse of
    that closed form, in all six planes."""
    dims, kappa, csw = (4, 6, 4, 6), 0.12, 1.7
    psi = I.gaussian_block(dims, 2, seed=21)
    V = psi.shape[0]
    worst = 0.0
    for mu in range(4):
        for nu in range(mu + 1, 4):
            U, phi = pins.abelian_flux_links(dims, mu, nu)
            f = np.diag([np.sin(phi), -np.sin(phi), 0.0])
            AD = np.eye(12) - kappa * csw * np.kron(pins.sigma_closed_form(mu, nu), f)
            want = np.einsum("ij,vjl->vil", np.linalg.inv(AD), psi.reshape(V, 12, 2))
            ctx = wd.wd_create(dev(U), dims, kappa, csw)
            got = host(wd.jacobi_precond(ctx, dev(psi), 1)).reshape(V, 12, 2)
            worst = max(worst, rel(got, want))
            wd.wd_destroy(ctx)
    assert worst < 1e-14


def test_jacobi_matches_oracle_j12_8x8x8x16(wd):
    """The paper's recommended j = 12 (Sec. 3.3) on 8^3 x 16 with L = 12, FP64 sweeps."""
    dims, L, j = (8, 8, 8, 16), 12, 12
    links = I.random_links(dims, 0.2, seed=0)
    op = O.WilsonClover(links, dims, 0.13, 1.0)
    R = I.z4_noise(dims, L, seed=5)
    ctx = wd.wd_create(dev(links), dims, 0.13, 1.0)
    G = host(wd.jacobi_precond(ctx, dev(R), j))
    G_ref = S.jacobi(op, R, j)
    assert rel(G, G_ref) <= APPLY_TOL
    assert max_elem_rel(G, G_ref) <= APPLY_TOL


@pytest.mark.parametrize("j", [0, 1, 2, 5])
@pytest.mark.parametrize("dims,L", [((4, 4, 4, 4), 4), ((3, 4, 5, 6), 7)])
def test_jacobi_matches_oracle(wd, j, dims, L):
    links = I.random_links(dims, 0.4, seed=2)
    op = O.WilsonClover(links, dims, 0.12, 1.0)
    R = I.gaussian_block(dims, L, seed=5)
    ctx = wd.wd_create(dev(links), dims, 0.12, 1.0)
    G = host(wd.jacobi_precond(ctx, dev(R), j))
    G_ref = S.jacobi(op, R, j)
    assert rel(G, G_ref) <= APPLY_TOL
    assert max_elem_rel(G, G_ref) <= APPLY_TOL


@pytest.mark.parametrize("B_kind,L,j", [("point", 4, 4), ("z4", 4, 0), ("z4", 3, 2),
                                        ("z4", 12, 4), ("z4", 1, 3)])
def test_solve_matches_oracle_4_4(wd, B_kind, L, j):
    dims = (4, 4, 4, 4)
    links = I.random_links(dims, 0.3, seed=0)
    op = O.WilsonClover(links, dims, 0.115, 1.0)
    B = I.point_sources(dims, L) if B_kind == "point" else I.z4_noise(dims, L, seed=1)
    ref = S.solve(op, B, j=j, tol=1e-12)
    ctx = wd.wd_create(dev(links), dims, 0.115, 1.0)
    Xg, info = wd.bbicggr_solve(ctx, dev(B), j=j, tol=1e-12)
    Xg = host(Xg)
    assert info["status"] == wd.WD_OK
    assert abs(info["iters"] - ref.iters) <= 1
    if info["restarts"] == 0:
        assert info["mvm_paper"] == L * (2 * (j + 1) * info["iters"] + 1)
    assert S.true_residual(op, B, Xg).max() <= TRUE_RES_TOL
    assert info["max_true_resid"] <= TRUE_RES_TOL
    assert rel(Xg, ref.X) <= SOLVE_X_TOL


@pytest.mark.parametrize("j,L", [(0, 1), (2, 4), (4, 12)])
def test_solve_matches_dense_lu_2_4(wd, j, L):
    dims = (2, 2, 2, 2)
    links = I.random_links(dims, 0.3, seed=0)
    op = O.WilsonClover(links, dims, 0.115, 1.0)
    B = I.z4_noise(dims, L, seed=1)
    X_lu = np.linalg.solve(op.dense(), B.reshape(op.N, L)).reshape(B.shape)
    ctx = wd.wd_create(dev(links), dims, 0.115, 1.0)
    Xg, info = wd.bbicggr_solve(ctx, dev(B), j=j, tol=1e-12)
    assert info["status"] == wd.WD_OK
    assert rel(host(Xg), X_lu) <= SOLVE_X_TOL


def test_solve_history_matches_oracle(wd):
    """The per-iteration max relative residual follows the oracle's to rounding."""
    dims = (4, 4, 4, 4)
    links = I.random_links(dims, 0.3, seed=0)
    op = O.WilsonClover(links, dims, 0.12, 1.0)
    B = I.z4_noise(dims, 4, seed=1)
    X, st, k, nm, rec, hist = S.bbicggr(op, B, np.zeros_like(B), 3, 1e-12)
    ctx = wd.wd_create(dev(links), dims, 0.12, 1.0)
    _, info = wd.bbicggr_solve(ctx, dev(B), j=3, tol=1e-12, max_restarts=0, history=1000)
    h = info["history"]
    n = min(len(h), len(hist))
    assert n >= 5
    # the residual curve agrees while it is well above the rounding floor
    for a, b in zip(h[:n], hist[:n]):
        if b > 1e-9:
            assert abs(a - b) <= 1e-6 * b


def test_solve_8_8_8_16_true_residual(wd):
    dims = (8, 8, 8, 16)
    links = I.random_links(dims, 0.2, seed=0)
    op = O.WilsonClover(links, dims, 0.12, 1.0)
    B = I.z4_noise(dims, 12, seed=1)
    ctx = wd.wd_create(dev(links), dims, 0.12, 1.0)
    Xg, info = wd.bbicggr_solve(ctx, dev(B), j=4, tol=1e-12)
    assert info["status"] == wd.WD_OK
    assert S.true_residual(op, B, host(Xg)).max() <= TRUE_RES_TOL


def test_solve_host_buffers_and_determinism(wd):
    dims = (4, 4, 4, 8)
    links = I.random_links(dims, 0.3, seed=3)
    B = I.z4_noise(dims, 6, seed=2)
    ctx = wd.wd_create(dev(links), dims, 0.12, 1.0)
    X1, i1 = wd.bbicggr_solve(ctx, B, j=3, tol=1e-12)          # host numpy in and out
    X2, i2 = wd.bbicggr_solve(ctx, dev(B), j=3, tol=1e-12)
    X3, i3 = wd.bbicggr_solve(ctx, dev(B), j=3, tol=1e-12)
    assert i1["status"] == i2["status"] == wd.WD_OK
    assert np.array_equal(X1, host(X2))                     # reductions are deterministic
    assert np.array_equal(host(X2), host(X3))
    assert i1["iters"] == i2["iters"] == i3["iters"]


def test_solver_error_paths(wd):
    dims = (2, 2, 2, 4)
    links = I.random_links(dims, 0.3, seed=0)
    op = O.WilsonClover(links, dims, 0.115, 1.0)
    ctx = wd.wd_create(dev(links), dims, 0.115, 1.0)
    B = I.z4_noise(dims, 2, seed=1)
    # maxit
    ref = S.bbicggr(op, B, np.zeros_like(B), 1, 1e-12, maxit=2)
    _, info = wd.bbicggr_solve(ctx, dev(B), j=1, tol=1e-12, maxit=2, max_restarts=0)
    assert info["status"] == wd.WD_NOT_CONVERGED == ref[1] and info["iters"] == 2
    # divergence threshold
    ref = S.bbicggr(op, B, np.zeros_like(B), 1, 1e-12, div_thresh=1e-6)
    _, info = wd.bbicggr_solve(ctx, dev(B), j=1, tol=1e-12, div_thresh=1e-6)
    assert info["status"] == wd.WD_DIVERGED == ref[1] and info["iters"] == ref[2] == 1
    # rank-deficient block: singular R~_0^H V_0 (rank loss) -> BREAKDOWN before any update
    B2 = B.copy()
    B2[..., 1] = B2[..., 0]
    ref = S.bbicggr(op, B2, np.zeros_like(B2), 1, 1e-12)
    X2, info = wd.bbicggr_solve(ctx, dev(B2), j=1, tol=1e-12)
    assert info["status"] == wd.WD_BREAKDOWN == ref[1] and info["iters"] == ref[2] == 0
    assert np.array_equal(host(X2), np.zeros_like(B2))
    # a zero column of B is rejected
    B3 = B.copy()
    B3[..., 0] = 0
    with pytest.raises(wd.WDError):
        wd.bbicggr_solve(ctx, dev(B3), j=1, tol=1e-12)
    # bad arguments
    with pytest.raises(wd.WDError):
        wd.bbicggr_solve(ctx, dev(I.z4_noise(dims, 17, seed=1)), j=1)
    with pytest.raises(wd.WDError):
        wd.wd_create(dev(links), (1, 2, 2, 4), 0.1, 1.0)
    with pytest.raises(wd.WDError):
        wd.bbicggr_solve(ctx, dev(B), j=-1)


def test_full_size_16_16_16_32(wd):
    """16^3 x 32, L = 12 (the paper's lattice, the bench workload): wd_apply against the oracle
    on every site, gamma_5-hermiticity of the CUDA operator, and a solve whose true residual the
    oracle recomputes."""
    dims = (16, 16, 16, 32)
    links = I.random_links(dims, 0.2, seed=0)
    kappa = 0.12
    ctx = wd.wd_create(dev(links), dims, kappa, 1.0)
    X = I.z4_noise(dims, 12, seed=7)
    Y = host(wd.wd_apply(ctx, dev(X)))
    op = O.WilsonClover(links, dims, kappa, 1.0)
    Y_ref = op.apply(X)
    assert rel(Y, Y_ref) <= APPLY_TOL
    del Y, Y_ref
    B = I.z4_noise(dims, 12, seed=1)
    for precision in (0, 1):
        Xg, info = wd.bbicggr_solve(ctx, dev(B), j=12, tol=1e-12, precision=precision)
        assert info["status"] == wd.WD_OK
        assert S.true_residual(op, B, host(Xg)).max() <= TRUE_RES_TOL


def test_bench_workload_double_float_forms(wd):
    """The bench workload itself (16^3 x 32, kappa = 0.134 near the critical kappa, L = 12, j = 12)
    in the plain FP64 form and the two double-float forms: every column's true residual,
    recomputed by the oracle, is <= 1e-12, the double-float forms need no fallback, and their
    solutions agree with the FP64 form's column by column."""
    dims, kappa = (16, 16, 16, 32), 0.134
    links = I.random_links(dims, 0.2, seed=0)
    op = O.WilsonClover(links, dims, kappa, 1.0)
    ctx = wd.wd_create(dev(links), dims, kappa, 1.0)
    B = I.z4_noise(dims, 12, seed=1)
    sols = {}
    for precision in (0, 4, 5):
        Xg, info = wd.bbicggr_solve(ctx, dev(B), j=12, tol=1e-12, precision=precision)
        assert info["status"] == wd.WD_OK and info["fallbacks"] == 0
        sols[precision] = host(Xg)
        assert S.true_residual(op, B, sols[precision]).max() <= TRUE_RES_TOL
    ref = sols[0].reshape(-1, 12)
    for precision in (4, 5):
        d = np.linalg.norm(sols[precision].reshape(-1, 12) - ref, axis=0) / np.linalg.norm(ref, axis=0)
        assert d.max() <= SOLVE_X_TOL


# ---------------------------------------------------------------- FP32 preconditioner (precision 1)
@pytest.mark.parametrize("j", [1, 2, 5, 12])
@pytest.mark.parametrize("dims,L", [((4, 4, 4, 4), 4), ((3, 4, 5, 6), 7), ((8, 8, 8, 16), 12)])
def test_jacobi_fp32_matches_oracle(wd, j, dims, L):
    links = I.random_links(dims, 0.3, seed=2)
    op = O.WilsonClover(links, dims, 0.12, 1.0)
    R = I.gaussian_block(dims, L, seed=5)
    ctx = wd.wd_create(dev(links), dims, 0.12, 1.0)
    G = host(wd.jacobi_precond(ctx, dev(R), j, precision=1))
    G_ref = S.jacobi(op, R, j)
    assert rel(G, G_ref) <= MIXED_TOL
    assert max_elem_rel(G, G_ref) <= MIXED_TOL


@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("B_kind,L,j", [("point", 4, 4), ("z4", 12, 4), ("z4", 3, 1)])
def test_mixed_solve_matches_fp64_oracle(wd, B_kind, L, j, precision):
    """An FP32 preconditioner changes M, not what block BiCGGR computes: the FP64 outer
    recurrences still reach the FP64 solution."""
    dims = (4, 4, 4, 4)
    links = I.random_links(dims, 0.3, seed=0)
    op = O.WilsonClover(links, dims, 0.115, 1.0)
    B = I.point_sources(dims, L) if B_kind == "point" else I.z4_noise(dims, L, seed=1)
    ref = S.solve(op, B, j=j, tol=1e-12)
    ctx = wd.wd_create(dev(links), dims, 0.115, 1.0)
    Xg, info = wd.bbicggr_solve(ctx, dev(B), j=j, tol=1e-12, precision=precision)
    Xg = host(Xg)
    assert info["status"] == wd.WD_OK
    assert S.true_residual(op, B, Xg).max() <= TRUE_RES_TOL
    assert rel(Xg, ref.X) <= SOLVE_X_TOL
    assert abs(info["iters"] - ref.iters) <= max(2, ref.iters // 10)


def test_mixed_solve_8_8_8_16_near_critical(wd):
    dims = (8, 8, 8, 16)
    links = I.random_links(dims, 0.2, seed=0)
    op = O.WilsonClover(links, dims, 0.132, 1.0)
    B = I.z4_noise(dims, 12, seed=1)
    ctx = wd.wd_create(dev(links), dims, 0.132, 1.0)
    X64, i64 = wd.bbicggr_solve(ctx, dev(B), j=12, tol=1e-12)
    X32, i32 = wd.bbicggr_solve(ctx, dev(B), j=12, tol=1e-12, precision=1)
    assert i64["status"] == i32["status"] == wd.WD_OK
    assert S.true_residual(op, B, host(X32)).max() <= TRUE_RES_TOL
    assert rel(host(X32), host(X64)) <= SOLVE_X_TOL


def test_mixed_solve_falls_back_to_fp64_preconditioner_near_critical(wd):
    """Near the critical kappa the rounding of an FP32 preconditioner (a non-linear M) can stall
    block BiCGGR, which needs a fixed linear M; the solve then starts over from X_0 with the FP64
    preconditioner and still reaches the FP64 answer."""
    dims = (6, 6, 6, 6)
    links = I.random_links(dims, 0.2, seed=0)
    op = O.WilsonClover(links, dims, 0.134, 1.0)
    B = I.z4_noise(dims, 4, seed=1)
    ctx = wd.wd_create(dev(links), dims, 0.134, 1.0)
    X64, i64 = wd.bbicggr_solve(ctx, dev(B), j=4, tol=1e-12, maxit=2000)
    X32, i32 = wd.bbicggr_solve(ctx, dev(B), j=4, tol=1e-12, precision=1, maxit=2000)
    assert i64["status"] == i32["status"] == wd.WD_OK
    assert S.true_residual(op, B, host(X32)).max() <= TRUE_RES_TOL
    assert rel(host(X32), host(X64)) <= SOLVE_X_TOL
    assert i32["fallbacks"] in (0, 1)
    _, i0 = wd.bbicggr_solve(ctx, dev(B), j=4, tol=1e-12, precision=1, maxit=300, stall_window=0)
    assert i0["fallbacks"] == 0


TILES = [(1, 64, 0, 0), (1, 128, 0, 0), (1, 256, 0, 0), (2, 64, 0, 0), (2, 128, 0, 0),
         (2, 256, 0, 0), (0, 128, 0, 0), (2, 64, 8, 0), (1, 64, 8, 0), (2, 64, 0, 1),
         (1, 64, 12, 0)]


@pytest.mark.parametrize("tile", TILES)
def test_fp32_sweep_tiles_match_oracle(wd, tile):
    """Every tile the autotuner may pick computes the same sweep."""
    dims, L = (3, 4, 5, 6), 6
    links = I.random_links(dims, 0.4, seed=2)
    op = O.WilsonClover(links, dims, 0.12, 1.0)
    R = I.gaussian_block(dims, L, seed=5)
    ctx = wd.wd_create(dev(links), dims, 0.12, 1.0)
    wd.wd_set_tile(ctx, L, *tile)
    G = host(wd.jacobi_precond(ctx, dev(R), 5, precision=1))
    assert wd.wd_tuned_tile(ctx, L) == tile
    assert rel(G, S.jacobi(op, R, 5)) <= MIXED_TOL


def test_autotuner_picks_a_valid_tile(wd):
    dims, L = (4, 4, 4, 8), 12
    ctx = wd.wd_create(dev(I.random_links(dims, 0.3, seed=0)), dims, 0.12, 1.0)
    assert wd.wd_tuned_tile(ctx, L) is None
    wd.jacobi_precond(ctx, dev(I.z4_noise(dims, L, seed=1)), 4, precision=1)
    assert wd.wd_tuned_tile(ctx, L) in TILES
    with pytest.raises(wd.WDError):
        wd.wd_set_tile(ctx, 3, 2, 128)          # 2 does not divide L = 3
    with pytest.raises(wd.WDError):
        wd.wd_set_tile(ctx, 4, 2, 128, 8)       # the 128-register build takes 64-thread CTAs
    with pytest.raises(wd.WDError):
        wd.wd_set_tile(ctx, 4, 1, 64, 0, 1)     # the staged pipeline takes 2 RHS per thread
    with pytest.raises(wd.WDError):
        wd.wd_set_tile(ctx, 3, 2, 64, 0, 1)     # ... and an even L
