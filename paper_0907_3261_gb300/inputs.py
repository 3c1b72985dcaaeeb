"""Seeded synthetic inputs for the clover Wilson-Dirac solve: gauge links, sources, gauge transforms.

This module is the only code shared by the oracle-side tests and the CUDA path.  It holds none of
the method's arithmetic (no operator, no clover term, no solver step): it only draws random numbers
and shapes them into the inputs the paper's experiments use (Sec. 3.1: SU(3) gauge links on an
Lx*Ly*Lz*Lt lattice; point sources whose i-th component is one).  The paper's gauge ensembles are
not available, so links are synthetic: the SU(3) projection of (1 + eps*G) with G a complex
Gaussian 3x3 matrix.

Generator (counter based, identical on every platform up to the last ulp of log/cos/sin):
  * SplitMix64 finaliser applied to ``key + (n+1) * 0x9E3779B97F4A7C15`` (mod 2^64) for counter n,
    where ``key`` is the SplitMix64 finaliser of ``seed XOR stream_tag``.
  * Uniform u in (0, 1]: ``((z >> 11) + 1) * 2^-53``.
  * Complex Gaussian entry from two consecutive uniforms (u1, u2) by Box-Muller:
    ``r = sqrt(-2 ln u1)``, ``re = r cos(2 pi u2)``, ``im = r sin(2 pi u2)``: variance 1 per part.
  * Fill order of the link field: site, mu, row, col.

Layouts (row-major, complex128):
  * site index ``x + Lx*(y + Ly*(z + Lz*t))``;
  * links ``[site][mu][3][3]``, ``U_mu(x)`` the link from x to x+mu, mu = 0..3 <-> x, y, z, t;
  * block vectors (N x L) ``[site][spin 4][colour 3][rhs L]`` -- RHS innermost.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

STREAM_LINKS = 0x4C494E4B          # "LINK"
STREAM_SOURCE = 0x53524345         # "SRCE"
STREAM_GAUGE = 0x47415547          # "GAUG"
STREAM_VECTOR = 0x56454354         # "VECT"


def _mix(z: np.ndarray) -> np.ndarray:
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64(seed: int, stream: int, count: int) -> np.ndarray:
    """``count`` 64-bit outputs of the counter-based SplitMix64 stream (seed, stream)."""
    key = _mix(np.array([(seed ^ stream) & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64))[0]
    n = np.arange(1, count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = key + n * _GOLDEN
    return _mix(z)


def uniforms(seed: int, stream: int, count: int) -> np.ndarray:
    """Uniform doubles in (0, 1]."""
    z = splitmix64(seed, stream, count)
    return ((z >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)


def complex_gaussian(seed: int, stream: int, count: int) -> np.ndarray:
    """``count`` complex normal draws, variance 1 in each of the real and imaginary parts."""
    u = uniforms(seed, stream, 2 * count).reshape(count, 2)
    r = np.sqrt(-2.0 * np.log(u[:, 0]))
    ang = 2.0 * np.pi * u[:, 1]
    return r * np.cos(ang) + 1j * (r * np.sin(ang))


def project_su3(m: np.ndarray) -> np.ndarray:
    """Project a stack of 3x3 complex matrices onto SU(3).

    Gram-Schmidt on rows 0 and 1, then row 2 = conj(row0 x row1), which makes the matrix unitary
    with determinant exactly |row0 x row1|^2 = 1 (up to rounding).
    """
    m = np.asarray(m, dtype=np.complex128)
    a = m[..., 0, :]
    a = a / np.linalg.norm(a, axis=-1, keepdims=True)
    b = m[..., 1, :]
    b = b - np.sum(np.conj(a) * b, axis=-1, keepdims=True) * a
    b = b / np.linalg.norm(b, axis=-1, keepdims=True)
    c = np.conj(np.cross(a, b))
    return np.stack([a, b, c], axis=-2)


def volume(dims) -> int:
    lx, ly, lz, lt = (int(d) for d in dims)
    return lx * ly * lz * lt


def random_links(dims, eps: float, seed: int = 0) -> np.ndarray:
    """Links ``U_mu(x) = SU3proj(1 + eps*G)``, complex128 ``[V][4][3][3]``."""
    v = volume(dims)
    g = complex_gaussian(seed, STREAM_LINKS, v * 4 * 9).reshape(v, 4, 3, 3)
    return np.ascontiguousarray(project_su3(np.eye(3) + eps * g))


def unit_links(dims) -> np.ndarray:
    """Free field: every link is the 3x3 identity."""
    v = volume(dims)
    return np.ascontiguousarray(np.broadcast_to(np.eye(3, dtype=np.complex128), (v, 4, 3, 3)))


def random_gauge_transform(dims, seed: int = 0) -> np.ndarray:
    """Random SU(3) matrices ``Omega(x)``, ``[V][3][3]`` (projection of a pure Gaussian matrix)."""
    v = volume(dims)
    g = complex_gaussian(seed, STREAM_GAUGE, v * 9).reshape(v, 3, 3)
    return np.ascontiguousarray(project_su3(g))


def z4_noise(dims, L: int, seed: int = 1) -> np.ndarray:
    """Sources whose entries are drawn uniformly from {1, i, -1, -i}; ``[V][4][3][L]``."""
    v = volume(dims)
    z = splitmix64(seed, STREAM_SOURCE, v * 12 * L)
    k = (z >> np.uint64(62)).astype(np.int64)
    vals = np.array([1.0, 1j, -1.0, -1j], dtype=np.complex128)
    return np.ascontiguousarray(vals[k].reshape(v, 4, 3, L))


def point_sources(dims, L: int) -> np.ndarray:
    """Unit-vector sources (Sec. 3.3): every column has a single entry equal to one.

    Column i sits at spin ``i % 4``, colour ``(i // 4) % 3`` of site ``i // 12``: L=4 gives spins
    0..3 at colour 0 of site 0, L=12 gives all 12 spin-colour components of site 0.
    """
    v = volume(dims)
    if L > 12 * v:
        raise ValueError("more point sources than lattice components")
    b = np.zeros((v, 4, 3, L), dtype=np.complex128)
    for i in range(L):
        b[i // 12, i % 4, (i // 4) % 3, i] = 1.0
    return b


def gaussian_block(dims, L: int, seed: int = 2) -> np.ndarray:
    """A block vector with complex Gaussian entries, ``[V][4][3][L]``."""
    v = volume(dims)
    return np.ascontiguousarray(
        complex_gaussian(seed, STREAM_VECTOR, v * 12 * L).reshape(v, 4, 3, L))


STREAM_WEIGHTS = 0x57474854        # "WGHT"


def network_channels(layers: int = 4, hidden: int = 4):
    """Channel counts (1, hidden, ..., hidden, 1) of a network with ``layers`` layers."""
    return [1] + [hidden] * (layers - 1) + [1]


def network_weights(layers: int = 4, hidden: int = 4, seed: int = 0, noise: float = 0.01):
    """Initial weights of the preconditioner network, one complex array [9][C_out][C_in][4][4] per
    layer: the on-site (d = 0) blocks start as the identity map of the network (first layer copies
    the input to every channel, hidden layers are channel-diagonal, the last averages the
    channels), plus complex Gaussian noise of standard deviation ``noise`` on every entry."""
    ch = network_channels(layers, hidden)
    total = sum(9 * ch[i + 1] * ch[i] * 16 for i in range(layers))
    g = complex_gaussian(seed, STREAM_WEIGHTS, total) * noise
    out, off = [], 0
    for i in range(layers):
        cin, cout = ch[i], ch[i + 1]
        n = 9 * cout * cin * 16
        W = g[off:off + n].reshape(9, cout, cin, 4, 4).copy()
        off += n
        for co in range(cout):
            for c in range(cin):
                if cin == 1 or cout == 1 or co == c:
                    W[0, co, c] += np.eye(4) * (1.0 / cin if cout == 1 else 1.0)
        out.append(W)
    return out
