"""Checks that pin the oracle to facts other than itself (closed forms, symmetries, dense solves).

Each function returns a relative error; the pin tests assert it is at rounding level and the
mutation tests assert that a planted mistake drives at least one of them far above it.
"""
import numpy as np

from paper_0907_3261_gb300 import inputs as I

PAULI = [np.array([[0, 1], [1, 0]], dtype=complex),
         np.array([[0, -1j], [1j, 0]], dtype=complex),
         np.array([[1, 0], [0, -1]], dtype=complex)]


def chiral_basis():
    """The stated convention: gamma_k = [[0, -i s_k], [i s_k, 0]], gamma_t = [[0, 1], [1, 0]]."""
    z = np.zeros((2, 2))
    g = [np.block([[z, -1j * s], [1j * s, z]]) for s in PAULI]
    g.append(np.block([[z, np.eye(2)], [np.eye(2), z]]))
    return np.array(g)


def sigma_closed_form(mu, nu):
    """sigma_{mu nu} in the chiral basis from the Pauli algebra s_j s_k = d_jk + i e_jkl s_l:
    sigma_{jk} = -e_jkl (s_l (+) s_l) for spatial j, k and sigma_{j t} = s_j (+) (-s_j)."""
    z = np.zeros((2, 2))
    if nu == 3:
        s = PAULI[mu]
        return np.block([[s, z], [z, -s]])
    l = 3 - mu - nu
    eps = 1.0 if (mu, nu, l) in ((0, 1, 2), (1, 2, 0), (2, 0, 1)) else -1.0
    s = PAULI[l]
    return -eps * np.block([[s, z], [z, s]])


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def coords(dims):
    lx, ly, lz, lt = dims
    s = np.arange(lx * ly * lz * lt)
    return np.stack([s % lx, (s // lx) % ly, (s // (lx * ly)) % lz, s // (lx * ly * lz)], axis=1)


def free_field_error(make_op, dims=(4, 4, 4, 4), kappa=0.13, csw=1.0, n=(1, 0, 2, 3), L=3):
    """A on a plane wave e^{ip.x} u with U = 1 equals the symbol
    [1 - 2 kappa sum cos p_mu + 2 i kappa sum gamma_mu sin p_mu] (discrete Fourier transform of the
    nearest-neighbour stencil; F = 0 for unit links so the clover term vanishes)."""
    op = make_op(I.unit_links(dims), dims, kappa, csw)
    p = 2 * np.pi * np.asarray(n) / np.asarray(dims)
    phase = np.exp(1j * coords(dims) @ p)
    u = I.complex_gaussian(7, 99, 12 * L).reshape(4, 3, L)
    psi = phase[:, None, None, None] * u[None]
    g = chiral_basis()
    sym = (1 - 2 * kappa * np.cos(p).sum()) * np.eye(4) + 2j * kappa * sum(
        g[m] * np.sin(p[m]) for m in range(4))
    expect = np.einsum("st,vtal->vsal", sym, psi)
    return rel(op.apply(psi), expect)


def gamma5_hermiticity_error(make_op, dims=(3, 4, 5, 6), kappa=0.124, csw=1.3, eps=0.5):
    """<phi, g5 A g5 psi> = <A phi, psi> for random phi, psi on rough links."""
    U = I.random_links(dims, eps, seed=3)
    op = make_op(U, dims, kappa, csw)
    phi = I.gaussian_block(dims, 2, seed=11)
    psi = I.gaussian_block(dims, 2, seed=12)
    g5 = np.diag([1.0, 1.0, -1.0, -1.0])
    g5A = lambda z: np.einsum("st,vtal->vsal", g5, z)
    lhs = np.vdot(phi, g5A(op.apply(g5A(psi))))
    rhs = np.vdot(op.apply(phi), psi)
    return abs(lhs - rhs) / abs(rhs)


def gauge_covariance_error(make_op, dims=(3, 4, 5, 6), kappa=0.124, csw=1.3, eps=0.5):
    """A[U'](Omega psi) = Omega A[U] psi with U'_mu(x) = Omega(x) U_mu(x) Omega(x+mu)^H."""
    U = I.random_links(dims, eps, seed=4)
    Om = I.random_gauge_transform(dims, seed=5)
    c = coords(dims)
    lx, ly, lz, lt = dims
    Up = np.empty_like(U)
    for mu in range(4):
        cf = c.copy()
        cf[:, mu] = (cf[:, mu] + 1) % dims[mu]
        fwd = cf[:, 0] + lx * (cf[:, 1] + ly * (cf[:, 2] + lz * cf[:, 3]))
        Up[:, mu] = Om @ U[:, mu] @ np.conj(np.swapaxes(Om[fwd], -1, -2))
    psi = I.gaussian_block(dims, 2, seed=13)
    rot = lambda z: np.einsum("vab,vsbl->vsal", Om, z)
    lhs = make_op(Up, dims, kappa, csw).apply(rot(psi))
    rhs = rot(make_op(U, dims, kappa, csw).apply(psi))
    return rel(lhs, rhs)


def abelian_flux_links(dims, mu, nu, n=1):
    """Constant U(1) flux phi = 2 pi n / (L_mu L_nu) through every (mu, nu) plaquette, embedded as
    diag(e^{i a}, e^{-i a}, 1): U_nu(x) = e^{i phi x_mu}, U_mu(x) = 1 except the twist
    U_mu(x) = e^{-i phi L_mu x_nu} on the last mu-slice, all other links 1."""
    c = coords(dims)
    V = len(c)
    phi = 2 * np.pi * n / (dims[mu] * dims[nu])
    ang = np.zeros((V, 4))
    ang[:, nu] = phi * c[:, mu]
    last = c[:, mu] == dims[mu] - 1
    ang[last, mu] = -phi * dims[mu] * c[last, nu]
    U = np.zeros((V, 4, 3, 3), dtype=complex)
    U[..., 0, 0] = np.exp(1j * ang)
    U[..., 1, 1] = np.exp(-1j * ang)
    U[..., 2, 2] = 1.0
    return U, phi


def abelian_flux_error(make_op, dims=(4, 6, 4, 6), kappa=0.12, csw=1.7):
    """Every plaquette of the (mu, nu) plane is diag(e^{i phi}, e^{-i phi}, 1), so F_{mu nu} =
    diag(sin phi, -sin phi, 0), the other F vanish, and A_D = 1 - kappa c_SW sigma_{mu nu} F_{mu nu}
    exactly, with sigma_{mu nu} from the Pauli algebra.  Largest error over the six planes."""
    worst = 0.0
    for mu in range(4):
        for nu in range(mu + 1, 4):
            U, phi = abelian_flux_links(dims, mu, nu)
            op = make_op(U, dims, kappa, csw)
            f = np.diag([np.sin(phi), -np.sin(phi), 0.0])
            expect = np.eye(12) - kappa * csw * np.kron(sigma_closed_form(mu, nu), f)
            psi = I.gaussian_block(dims, 2, seed=21)
            V = psi.shape[0]
            got = op.apply_site_diagonal(psi)
            want = np.einsum("ij,vjl->vil", expect, psi.reshape(V, 12, 2)).reshape(psi.shape)
            worst = max(worst, rel(got, want))
    return worst


def all_operator_pins(make_op):
    return {
        "free_field": free_field_error(make_op),
        "free_field_odd": free_field_error(make_op, dims=(3, 5, 4, 6), n=(1, 2, 1, 5)),
        "gamma5_hermiticity": gamma5_hermiticity_error(make_op),
        "gauge_covariance": gauge_covariance_error(make_op),
        "abelian_flux": abelian_flux_error(make_op),
    }


def dense_jacobi_polynomial(A, D, j):
    """M = sum_{i<j} (I - D^{-1} A)^i D^{-1} as a dense matrix (M = I for j = 0)."""
    n = A.shape[0]
    if j == 0:
        return np.eye(n, dtype=complex)
    Dinv = np.linalg.inv(D)
    T = np.eye(n) - Dinv @ A
    M = np.zeros((n, n), dtype=complex)
    term = Dinv.copy()
    for _ in range(j):
        M += term
        term = T @ term
    return M


def solver_invariant_error(bbicggr, op, B, j, eps=1e-12, maxit=300):
    """Run ``bbicggr`` on a small lattice and check, with dense A and M built independently, the
    exact relations of the algorithm box at every outer iteration:
      F = M R, W = A F, V = A M P, G = M U, Y = A G          (how the blocks are defined),
      R~_0^H (R - V alpha) = 0                               (the equation that defines alpha),
      Tr[W^H (R - zeta W)] = 0                               (zeta minimises ||R - zeta W||_F),
      R~_0^H (V alpha gamma + A M (R - V alpha)) = 0         (gamma = alpha^{-1} beta with beta the
                                                              block BiCGSTAB coefficient
                                                              -(R~_0^H V)^{-1} R~_0^H A M S),
      R_{k+1} = B - A X_{k+1}, relative to ||B||             (the GR property),
    and that the run ends within N/L iterations (finite termination of a block Krylov method).
    Returns the worst relative violation."""
    N = op.N
    L = B.shape[-1]
    A = op.dense()
    M = dense_jacobi_polynomial(A, op.dense_site_diagonal(), j)
    flat = lambda Z: Z.reshape(N, L)
    bn = np.linalg.norm(flat(B))
    worst = [0.0]

    def note(v):
        worst[0] = max(worst[0], float(v) if np.isfinite(v) else np.inf)

    def rel_(a, b):
        return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)

    def check(st):
        R, P, V, W, F = (flat(st[k]) for k in ("R", "P", "V", "W", "F"))
        G, Y, Uk, Rt = (flat(st[k]) for k in ("G", "Y", "U", "Rt"))
        al, ze = st["alpha"], st["zeta"]
        note(rel_(F, M @ R))
        note(rel_(W, A @ F))
        note(rel_(V, A @ M @ P))
        note(rel_(G, M @ Uk))
        note(rel_(Y, A @ G))
        note(np.abs(Rt.conj().T @ (R - V @ al)).max() / np.abs(Rt.conj().T @ R).max())
        note(abs(np.vdot(W, R - ze * W)) / abs(np.vdot(W, R)))
        if "gamma" in st:
            t = Rt.conj().T @ (A @ M @ (R - V @ al))
            note(np.abs(Rt.conj().T @ V @ al @ st["gamma"] + t).max() / np.abs(t).max())
        note(np.linalg.norm(flat(st["R_new"]) - (flat(B) - A @ flat(st["X_new"]))) / bn * 1e3)

    X, status, k, _, _, _ = bbicggr(op, B, np.zeros_like(B), j, eps, maxit=maxit, on_iter=check)
    if status != 0 or k > N // L:
        return np.inf
    note(np.linalg.norm(np.linalg.solve(A, flat(B)) - flat(X)) / np.linalg.norm(flat(X)) * 1e-2)
    return worst[0]


def dense_hopping_from_entries(links, dims):
    """The N x N hopping matrix H written entry by entry from its definition, with the stated
    chiral basis: the 12 x 12 block of row site x and column site x + mu is (1 - gamma_mu) (x)
    U_mu(x), that of column site x - mu is (1 + gamma_mu) (x) U_mu(x - mu)^H; blocks add where two
    neighbours coincide (extent 2).  Neighbours come from explicit periodic coordinate arithmetic,
    not from the oracle's neighbour tables."""
    dims = tuple(int(d) for d in dims)
    lx, ly, lz, lt = dims
    V = lx * ly * lz * lt
    U = np.asarray(links).reshape(V, 4, 3, 3)
    g = chiral_basis()
    one = np.eye(4)
    c = coords(dims)
    H = np.zeros((12 * V, 12 * V), dtype=complex)

    def site(cc):
        return int(cc[0] + lx * (cc[1] + ly * (cc[2] + lz * cc[3])))

    for x in range(V):
        for mu in range(4):
            up = c[x].copy()
            up[mu] = (up[mu] + 1) % dims[mu]
            dn = c[x].copy()
            dn[mu] = (dn[mu] - 1) % dims[mu]
            y, z = site(up), site(dn)
            H[12 * x:12 * x + 12, 12 * y:12 * y + 12] += np.kron(one - g[mu], U[x, mu])
            H[12 * x:12 * x + 12, 12 * z:12 * z + 12] += np.kron(one + g[mu], U[z, mu].conj().T)
    return H


def block_diagonal(blocks):
    """The N x N matrix with the given 12 x 12 site blocks ([V][12][12]) on its diagonal."""
    V = blocks.shape[0]
    D = np.zeros((12 * V, 12 * V), dtype=complex)
    for v in range(V):
        D[12 * v:12 * v + 12, 12 * v:12 * v + 12] = blocks[v]
    return D


def fp32_midpoint_distance(values):
    """For every non-zero real or imaginary part x of ``values``: |x - m| for the FP32 rounding
    midpoint m (halfway between two adjacent FP32 numbers) nearest to x.  Two FP64 computations of
    the same quantity that differ by less than this round to the same FP32 number."""
    x = np.concatenate([np.ravel(np.real(values)), np.ravel(np.imag(values))]).astype(np.float64)
    x = x[x != 0.0]
    f = x.astype(np.float32)
    up = np.nextafter(f, np.float32(np.inf)).astype(np.float64)
    dn = np.nextafter(f, np.float32(-np.inf)).astype(np.float64)
    f = f.astype(np.float64)
    return x, np.minimum(np.abs(x - 0.5 * (f + up)), np.abs(x - 0.5 * (f + dn)))


def fp32_rounding_margin(values):
    """Smallest midpoint distance (fp32_midpoint_distance) relative to |x|; inf if all are 0."""
    x, d = fp32_midpoint_distance(values)
    return float(np.min(d / np.abs(x))) if x.size else np.inf
