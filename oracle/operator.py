"""Oracle for the clover Wilson-Dirac matrix A (Eq. (1), Sec. 2) -- test infrastructure only.

The paper treats A as an N x N sparse non-Hermitian matrix with N = Lx*Ly*Lz*Lt*3*4 (Sec. 2) and
names its parameters kappa and c_SW (Sec. 3.1); its explicit form is left to Ref. [blockbicggr_app].
This module writes the operator out as the textbook definition in kappa normalisation:

    (A psi)(x) = A_D(x) psi(x)
                 - kappa * sum_mu [ (1 - gamma_mu) U_mu(x)        psi(x + mu)
                                  + (1 + gamma_mu) U_mu(x - mu)^H psi(x - mu) ]

    A_D(x) = 1 - kappa * c_SW * sum_{mu<nu} sigma_{mu nu} (x) F_{mu nu}(x)      (12 x 12 per site)
    sigma_{mu nu} = (i/2) [gamma_mu, gamma_nu]
    F_{mu nu} = (Q_{mu nu} - Q_{mu nu}^H) / (8 i),   Q = sum of the four plaquette leaves at x

with periodic boundaries and the chiral gamma basis
    gamma_k = [[0, -i s_k], [i s_k, 0]] (k = x, y, z),  gamma_t = [[0, 1], [1, 0]],
so that gamma_5 = gamma_x gamma_y gamma_z gamma_t = diag(1, 1, -1, -1).

"The diagonal part of the coefficient matrix" A_D (Sec. 2, below the Jacobi polynomial) is read as
the site-diagonal 12 x 12 block 1 + clover.

Pins (tests/test_oracle_operator.py): free-field plane-wave symbol, gamma_5-hermiticity, gauge
covariance, constant abelian flux closed form of the clover term in all six planes, c_SW = 0.
Layout of every block vector: ``[V][4 spin][3 colour][L]`` complex128, site index
``x + Lx*(y + Ly*(z + Lz*t))``; links ``[V][4 mu][3][3]``.
"""
from __future__ import annotations

import numpy as np


def gamma_matrices() -> np.ndarray:
    """The four Euclidean gamma matrices of the chiral basis, ``[4][4][4]`` (mu = x, y, z, t)."""
    pauli = [np.array([[0, 1], [1, 0]], dtype=complex),
             np.array([[0, -1j], [1j, 0]], dtype=complex),
             np.array([[1, 0], [0, -1]], dtype=complex)]
    g = np.zeros((4, 4, 4), dtype=complex)
    for k in range(3):
        g[k, 0:2, 2:4] = -1j * pauli[k]
        g[k, 2:4, 0:2] = 1j * pauli[k]
    g[3, 0:2, 2:4] = np.eye(2)
    g[3, 2:4, 0:2] = np.eye(2)
    return g


def gamma5() -> np.ndarray:
    g = gamma_matrices()
    return g[0] @ g[1] @ g[2] @ g[3]


def sigma(mu: int, nu: int) -> np.ndarray:
    """sigma_{mu nu} = (i/2) [gamma_mu, gamma_nu]."""
    g = gamma_matrices()
    return 0.5j * (g[mu] @ g[nu] - g[nu] @ g[mu])


class Lattice:
    """Periodic 4-d lattice with site index x + Lx*(y + Ly*(z + Lz*t))."""

    def __init__(self, dims):
        self.dims = tuple(int(d) for d in dims)
        lx, ly, lz, lt = self.dims
        self.V = lx * ly * lz * lt
        s = np.arange(self.V)
        coords = [s % lx, (s // lx) % ly, (s // (lx * ly)) % lz, s // (lx * ly * lz)]
        self.fwd = np.empty((4, self.V), dtype=np.int64)   # site of x + mu
        self.bwd = np.empty((4, self.V), dtype=np.int64)   # site of x - mu
        for mu in range(4):
            cf = list(coords)
            cf[mu] = (coords[mu] + 1) % self.dims[mu]
            self.fwd[mu] = self.index(cf)
            cb = list(coords)
            cb[mu] = (coords[mu] - 1) % self.dims[mu]
            self.bwd[mu] = self.index(cb)

    def index(self, c):
        lx, ly, lz, _ = self.dims
        return c[0] + lx * (c[1] + ly * (c[2] + lz * c[3]))


def _dag(m: np.ndarray) -> np.ndarray:
    return np.conj(np.swapaxes(m, -1, -2))


def field_strength(links: np.ndarray, lat: Lattice) -> np.ndarray:
    """Clover-leaf field strength F_{mu nu}(x), Hermitian 3x3, ``[V][4][4][3][3]``.

    Q_{mu nu}(x) is the sum of the four counter-clockwise plaquettes in the (mu, nu) plane that
    touch x, each starting and ending at x; F = (Q - Q^H) / (8i), F_{nu mu} = -F_{mu nu}.
    """
    U = links
    F = np.zeros((lat.V, 4, 4, 3, 3), dtype=complex)
    fwd, bwd = lat.fwd, lat.bwd
    for mu in range(4):
        for nu in range(mu + 1, 4):
            Um, Un = U[:, mu], U[:, nu]
            x_pm, x_pn = fwd[mu], fwd[nu]
            x_mm, x_mn = bwd[mu], bwd[nu]
            x_mm_pn = fwd[nu][x_mm]
            x_mm_mn = bwd[nu][x_mm]
            x_mn_pm = fwd[mu][x_mn]
            leaf1 = Um @ Un[x_pm] @ _dag(Um[x_pn]) @ _dag(Un)
            leaf2 = Un @ _dag(Um[x_mm_pn]) @ _dag(Un[x_mm]) @ Um[x_mm]
            leaf3 = _dag(Um[x_mm]) @ _dag(Un[x_mm_mn]) @ Um[x_mm_mn] @ Un[x_mn]
            leaf4 = _dag(Un[x_mn]) @ Um[x_mn] @ Un[x_mn_pm] @ _dag(Um)
            Q = leaf1 + leaf2 + leaf3 + leaf4
            F[:, mu, nu] = (Q - _dag(Q)) / 8j
            F[:, nu, mu] = -F[:, mu, nu]
    return F


def site_diagonal(links: np.ndarray, lat: Lattice, kappa: float, csw: float) -> np.ndarray:
    """A_D(x) = 1 - kappa c_SW sum_{mu<nu} sigma_{mu nu} (x) F_{mu nu}(x): ``[V][12][12]``.

    Row/column index ``spin*3 + colour``.
    """
    F = field_strength(links, lat)
    AD = np.broadcast_to(np.eye(12, dtype=complex), (lat.V, 12, 12)).copy()
    for mu in range(4):
        for nu in range(mu + 1, 4):
            s = sigma(mu, nu)
            term = np.einsum("st,vab->vsatb", s, F[:, mu, nu]).reshape(lat.V, 12, 12)
            AD -= kappa * csw * term
    return AD


def hopping_term(U: np.ndarray, lat: Lattice, psi: np.ndarray) -> np.ndarray:
    """The hopping term of Eq. (1) for links U ([V][4][3][3]):
    H psi = sum_mu (1 - g_mu) U_mu(x) psi(x+mu) + (1 + g_mu) U_mu(x-mu)^H psi(x-mu)."""
    g = gamma_matrices()
    psi = psi.reshape(lat.V, 4, 3, -1)
    out = np.zeros_like(psi)
    one = np.eye(4)
    for mu in range(4):
        up = np.einsum("vab,vsbl->vsal", U[:, mu], psi[lat.fwd[mu]])
        out += np.einsum("st,vtal->vsal", one - g[mu], up)
        U_back = U[lat.bwd[mu], mu]
        dn = np.einsum("vab,vsbl->vsal", _dag(U_back), psi[lat.bwd[mu]])
        out += np.einsum("st,vtal->vsal", one + g[mu], dn)
    return out


class WilsonClover:
    """The matrix A of Eq. (1) for given links, kappa and c_SW."""

    def __init__(self, links: np.ndarray, dims, kappa: float, csw: float):
        self.lat = Lattice(dims)
        self.U = np.asarray(links, dtype=complex).reshape(self.lat.V, 4, 3, 3)
        self.kappa = float(kappa)
        self.csw = float(csw)
        self.AD = site_diagonal(self.U, self.lat, self.kappa, self.csw)
        self.AD_inv = np.linalg.inv(self.AD)
        self.g = gamma_matrices()
        self.N = 12 * self.lat.V

    # -- pieces of A -----------------------------------------------------------------------
    def hopping(self, psi: np.ndarray) -> np.ndarray:
        """H psi = sum_mu (1 - g_mu) U_mu(x) psi(x+mu) + (1 + g_mu) U_mu(x-mu)^H psi(x-mu)."""
        return hopping_term(self.U, self.lat, psi)

    def apply_site_diagonal(self, psi: np.ndarray, inverse: bool = False) -> np.ndarray:
        """A_D psi (or A_D^{-1} psi), site by site with the full 12 x 12 block."""
        psi = psi.reshape(self.lat.V, 12, -1)
        m = self.AD_inv if inverse else self.AD
        return np.einsum("vij,vjl->vil", m, psi).reshape(self.lat.V, 4, 3, -1)

    def apply(self, psi: np.ndarray) -> np.ndarray:
        """A psi = A_D psi - kappa H psi (Eq. (1))."""
        return self.apply_site_diagonal(psi) - self.kappa * self.hopping(psi)

    def apply_gamma5(self, psi: np.ndarray) -> np.ndarray:
        g5 = gamma5()
        return np.einsum("st,vtal->vsal", g5, psi.reshape(self.lat.V, 4, 3, -1))

    # -- dense forms (small lattices only) ---------------------------------------------------
    def dense(self) -> np.ndarray:
        """The N x N matrix, column n = A e_n (N <= a few thousand)."""
        eye = np.eye(self.N, dtype=complex).reshape(self.lat.V, 4, 3, self.N)
        return self.apply(eye).reshape(self.N, self.N)

    def dense_site_diagonal(self) -> np.ndarray:
        D = np.zeros((self.N, self.N), dtype=complex)
        for v in range(self.lat.V):
            D[12 * v:12 * v + 12, 12 * v:12 * v + 12] = self.AD[v]
        return D
