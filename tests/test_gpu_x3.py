"""The FP32-lane form of the FP64 stencil (csrc/dslash_x3.cu, wd_set_apply_form 1) against the FP64
oracle and against the FP64-pipe form (needs a GB300).

Its hopping sums are exact up to ~2^-52 of their bound before one FP64 rounding, so it must agree
with the oracle as closely as FP64 arithmetic does (the FP64-pipe form rounds after every
operation), reproduce exactly representable results bit for bit, and scale exactly by powers of two.
"""
import numpy as np
import pytest

from oracle import operator as O
from oracle import solver as S
from paper_0907_3261_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# FP64 stencil accuracy: each output sums ~60 products of unit-size entries, so FP64 rounding is
# ~60 x 2^-53 ~ 7e-15 of the largest entry at worst; both forms stay below 1e-14.
X3_TOL = 1e-14


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


def max_elem_rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def both_forms(wd, links, dims, kappa, csw, X):
    ctx = wd.wd_create(dev(links), dims, kappa, csw)
    assert wd.wd_get_apply_form(ctx) == 1          # unitary links: the FP32-lane form by default
    Y1 = host(wd.wd_apply(ctx, dev(X)))
    wd.wd_set_apply_form(ctx, 0)
    Y0 = host(wd.wd_apply(ctx, dev(X)))
    return Y1, Y0


@pytest.mark.parametrize("dims,L", [((2, 2, 2, 2), 1), ((3, 4, 5, 6), 5), ((4, 4, 4, 4), 12),
                                    ((8, 8, 8, 16), 12), ((6, 4, 2, 8), 16)])
def test_x3_apply_matches_oracle(wd, dims, L):
    links = I.random_links(dims, 0.4, seed=3)
    X = I.gaussian_block(dims, L, seed=4)
    Y1, Y0 = both_forms(wd, links, dims, 0.13, 1.3, X)
    Yo = O.WilsonClover(links, dims, 0.13, 1.3).apply(X)
    assert max_elem_rel(Y1, Yo) < X3_TOL
    assert max_elem_rel(Y0, Yo) < X3_TOL
    assert max_elem_rel(Y1, Y0) < X3_TOL


def test_x3_every_element_to_its_own_scale(wd):
    """Entries spread over 2^-40 .. 2^40 by site: each output entry agrees with the oracle relative
    to the largest input entry among its neighbours and itself, as FP64 arithmetic would."""
    dims = (4, 4, 4, 8)
    links = I.random_links(dims, 0.3, seed=5)
    X = I.gaussian_block(dims, 3, seed=6)
    V = int(np.prod(dims))
    scale = 2.0 ** np.random.default_rng(7).integers(-40, 41, size=V)
    X = X * scale[:, None, None, None]
    Y1, _ = both_forms(wd, links, dims, 0.12, 1.0, X)
    op = O.WilsonClover(links, dims, 0.12, 1.0)
    Yo = op.apply(X)
    # the neighbourhood scale of every site: max |x| over the site and its 8 neighbours
    m = np.abs(X).reshape(V, -1).max(axis=1).reshape(dims[::-1])
    nb = m.copy()
    for ax in range(4):
        nb = np.maximum(nb, np.maximum(np.roll(m, 1, axis=ax), np.roll(m, -1, axis=ax)))
    err = np.abs(Y1 - Yo).reshape(V, -1).max(axis=1)
    assert (err <= 1e-14 * nb.reshape(V)).all()


def test_x3_exact_results_are_reproduced_bit_for_bit(wd):
    """Signed permutation links (unitary, entries 0, +-1, +-i), kappa = 1/8, c_SW = 0 and small
    integer spinors: every operation of A X is exact in FP64, so both forms and the oracle agree
    bit for bit."""
    dims = (4, 4, 4, 4)
    V = int(np.prod(dims))
    rng = np.random.default_rng(11)
    links = np.zeros((V, 4, 3, 3), dtype=complex)
    phases = np.array([1, -1, 1j, -1j])
    for s in range(V):
        for mu in range(4):
            perm = rng.permutation(3)
            for a in range(3):
                links[s, mu, a, perm[a]] = phases[rng.integers(4)]
    X = (rng.integers(-64, 65, size=(V, 4, 3, 5))
         + 1j * rng.integers(-64, 65, size=(V, 4, 3, 5))).astype(complex)
    Y1, Y0 = both_forms(wd, links, dims, 0.125, 0.0, X)
    Yo = O.WilsonClover(links, dims, 0.125, 0.0).apply(X)
    assert np.array_equal(Y1, Yo) and np.array_equal(Y0, Yo)


@pytest.mark.parametrize("j", [-300, -40, 40, 300])
def test_x3_scales_exactly(wd, j):
    dims = (4, 4, 4, 4)
    links = I.random_links(dims, 0.3, seed=1)
    X = I.gaussian_block(dims, 4, seed=2)
    ctx = wd.wd_create(dev(links), dims, 0.12, 1.0)
    Y = host(wd.wd_apply(ctx, dev(X)))
    Ys = host(wd.wd_apply(ctx, dev(X * 2.0 ** j)))
    assert np.array_equal(Ys, Y * 2.0 ** j)


def test_x3_zero_and_non_finite_inputs(wd):
    dims = (4, 4, 4, 4)
    links = I.random_links(dims, 0.3, seed=1)
    ctx = wd.wd_create(dev(links), dims, 0.12, 1.0)
    Z = np.zeros_like(I.gaussian_block(dims, 2, seed=2))
    assert np.array_equal(host(wd.wd_apply(ctx, dev(Z))), Z)
    X = I.gaussian_block(dims, 2, seed=2)
    X.reshape(-1)[0] = np.nan                       # site 0, spin 0, colour 0, rhs 0 (real part)
    Y = host(wd.wd_apply(ctx, dev(X)))
    V = int(np.prod(dims))
    bad = ~np.isfinite(Y).reshape(V, -1).all(axis=1)
    # rhs 0 of site 0 and of its 8 neighbours (site = x + 4 (y + 4 (z + 4 t)))
    expect = {0, 1, 3, 4, 12, 16, 48, 64, 192}
    assert set(np.nonzero(bad)[0]) == expect
    assert np.isfinite(Y.reshape(V, 12, 2)[..., 1]).all()   # rhs 1 untouched


@pytest.mark.parametrize("j", [1, 2, 5, 12])
def test_x3_jacobi_matches_oracle(wd, j):
    dims = (8, 8, 8, 16)
    links = I.random_links(dims, 0.2, seed=0)
    R = I.z4_noise(dims, 4, seed=1)
    ctx = wd.wd_create(dev(links), dims, 0.13, 1.0)
    assert wd.wd_get_apply_form(ctx) == 1
    G = host(wd.jacobi_precond(ctx, dev(R), j))
    Go = S.jacobi(O.WilsonClover(links, dims, 0.13, 1.0), R, j)
    assert max_elem_rel(G, Go) < 1e-13


@pytest.mark.parametrize("precision", [0, 5])
def test_x3_solve_matches_fp64_pipe_form(wd, precision):
    """The whole solve with either stencil form: the same iterations and solutions that agree to
    the solve's own accuracy; both reach the FP64 true residual."""
    dims = (8, 8, 8, 16)
    links = I.random_links(dims, 0.2, seed=0)
    B = I.z4_noise(dims, 12, seed=1)
    op = O.WilsonClover(links, dims, 0.13, 1.0)
    out = {}
    for form in (1, 0):
        ctx = wd.wd_create(dev(links), dims, 0.13, 1.0)
        wd.wd_set_apply_form(ctx, form)
        X, info = wd.bbicggr_solve(ctx, dev(B), j=12, tol=1e-12, precision=precision)
        assert info["status"] == wd.WD_OK
        X = host(X)
        assert S.true_residual(op, B, X).max() <= 1e-12
        out[form] = (X, info["iters"])
    assert abs(out[1][1] - out[0][1]) <= 1
    assert np.linalg.norm(out[1][0] - out[0][0]) <= 1e-10 * np.linalg.norm(out[0][0])


def test_x3_needs_unitary_links(wd):
    dims = (4, 4, 4, 4)
    links = I.random_links(dims, 0.3, seed=1) * 1.01
    ctx = wd.wd_create(dev(links), dims, 0.12, 1.0)
    assert wd.wd_get_apply_form(ctx) == 0
    with pytest.raises(wd.WDError):
        wd.wd_set_apply_form(ctx, 1)
    X = I.gaussian_block(dims, 2, seed=2)
    Yo = O.WilsonClover(links, dims, 0.12, 1.0).apply(X)
    assert max_elem_rel(host(wd.wd_apply(ctx, dev(X))), Yo) < X3_TOL


@pytest.mark.parametrize("kappa,precision", [(0.13, 0), (0.13, 5), (0.134, 5)])
def test_recursive_residual_stays_on_the_true_residual(wd, kappa, precision):
    """The recursive residual R (R -= zeta W + Y each iteration, never recomputed from X) stays
    on B - A X to FP64 accuracy through a whole solve: the products W = A F and Y = A G carry no
    error the recursion could accumulate beyond ~1e-15 of ||B||."""
    dims = (8, 8, 8, 16)
    links = I.random_links(dims, 0.2, seed=0)
    B = I.z4_noise(dims, 12, seed=1)
    ctx = wd.wd_create(dev(links), dims, kappa, 1.0)
    with pytest.raises(wd.WDError):
        wd.wd_copy_residual(ctx, torch.empty_like(dev(B)))      # no solve yet
    X, info = wd.bbicggr_solve(ctx, dev(B), j=12, tol=1e-12, precision=precision, maxit=2000)
    assert info["status"] == wd.WD_OK
    R = host(wd.wd_copy_residual(ctx, torch.empty_like(dev(B))))
    op = O.WilsonClover(links, dims, kappa, 1.0)
    T = B - op.apply(host(X))
    V = int(np.prod(dims))
    gap = (np.linalg.norm((R - T).reshape(V * 12, -1), axis=0)
           / np.linalg.norm(B.reshape(V * 12, -1), axis=0))
    assert gap.max() <= 1e-13
    with pytest.raises(wd.WDError):
        wd.wd_copy_residual(ctx, torch.empty_like(dev(B[..., :4])))   # another L


def test_x3_full_size_element_wise(wd):
    """The bench lattice (16^3 x 32, L = 12, near-critical kappa): every entry of the FP32-lane
    form's A X against the oracle and against the FP64-pipe form."""
    dims = (16, 16, 16, 32)
    links = I.random_links(dims, 0.2, seed=0)
    X = I.z4_noise(dims, 12, seed=7)
    Y1, Y0 = both_forms(wd, links, dims, 0.134, 1.0, X)
    Yo = O.WilsonClover(links, dims, 0.134, 1.0).apply(X)
    assert max_elem_rel(Y1, Yo) < X3_TOL
    assert max_elem_rel(Y1, Y0) < X3_TOL
