"""ctypes access to the C++ oracle (oracle/cpp/oracle.cpp) -- test infrastructure only.

The C++ oracle is a second, independent FP64 statement of the operator of Eq. (1), the Jacobi
polynomial and block BiCGGR of Sec. 2, run on host cores with OpenMP.  Only tests/, smoke() and
bench.py's CPU-baseline leg and reference arm use it.  ``build()`` compiles it with g++ (no CUDA);
__graft_entry__.build() does the same.

Parity status: pinned (tests/test_oracle_cpp.py: free-field symbol, gamma_5-hermiticity, gauge
covariance, abelian flux closed form, dense LU on 2^4, Table 1 #MVM identity, agreement with the
numpy oracle, and compiled planted mutations that the pins catch).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "cpp", "oracle.cpp")
LIB = os.path.join(HERE, "cpp", "liboracle.so")
FLAGS = ["-O3", "-std=c++17", "-fopenmp", "-fPIC", "-shared"]

_lib = None


def build(src: str = SRC, out: str = LIB) -> str:
    """Compile the C++ oracle (skipped when the library is newer than its source)."""
    if os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src):
        return out
    tmp = out + ".tmp"
    subprocess.run(["g++", *FLAGS, src, "-o", tmp], check=True)
    os.replace(tmp, out)
    return out


def load(path: str = LIB):
    L = C.CDLL(path)
    d, i, vp = C.c_double, C.c_int, C.c_void_p
    L.oracle_set_threads.argtypes = [i]
    L.oracle_set_threads.restype = i
    L.oracle_apply.argtypes = [vp, vp, d, d, vp, vp, i]
    L.oracle_site_diag.argtypes = [vp, vp, d, d, vp, vp, i, i]
    L.oracle_jacobi.argtypes = [vp, vp, d, d, vp, vp, i, i]
    L.oracle_solve.argtypes = [vp, vp, d, d, vp, vp, i, i, d, i, i, vp, vp]
    for n in ("oracle_apply", "oracle_site_diag", "oracle_jacobi", "oracle_solve"):
        getattr(L, n).restype = i
    L.oracle_create.argtypes = [vp, vp, d, d]
    L.oracle_create.restype = vp
    L.oracle_destroy.argtypes = [vp]
    L.oracle_destroy.restype = None
    L.oracle_start.argtypes = [vp, vp, vp, i, i, d]
    L.oracle_start.restype = i
    L.oracle_step.argtypes = [vp]
    L.oracle_step.restype = i
    L.oracle_result.argtypes = [vp, vp, vp, vp, vp]
    L.oracle_result.restype = None
    return L


def lib():
    global _lib
    if _lib is None:
        _lib = load(build())
    return _lib


def _c(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _dims(dims):
    return np.ascontiguousarray(dims, dtype=np.int32)


def _p(a):
    return C.c_void_p(a.ctypes.data)


def set_threads(n: int) -> int:
    """Use n OpenMP threads (n <= 0: leave as is); returns the count in use."""
    return int(lib().oracle_set_threads(int(n)))


class CppOracle:
    """The C++ oracle behind the numpy oracle's interface (apply, apply_site_diagonal)."""

    def __init__(self, links, dims, kappa, csw, library=None):
        self.links, self.dims = _c(links), _dims(dims)
        self.kappa, self.csw = float(kappa), float(csw)
        self.L_ = library or lib()

    def apply(self, psi):
        x = _c(psi)
        y = np.empty_like(x)
        self.L_.oracle_apply(_p(self.links), _p(self.dims), self.kappa, self.csw, _p(x), _p(y),
                             x.shape[-1])
        return y

    def apply_site_diagonal(self, psi, inverse=False):
        x = _c(psi)
        y = np.empty_like(x)
        self.L_.oracle_site_diag(_p(self.links), _p(self.dims), self.kappa, self.csw, _p(x),
                                 _p(y), x.shape[-1], int(bool(inverse)))
        return y

    def jacobi(self, U, j):
        u = _c(U)
        g = np.empty_like(u)
        self.L_.oracle_jacobi(_p(self.links), _p(self.dims), self.kappa, self.csw, _p(u), _p(g),
                              u.shape[-1], int(j))
        return g

    def solve(self, B, j, tol=1e-12, maxit=10000, max_restarts=3, X0=None):
        """(X, status, iters, restarts, mvm per column, true residual per column)."""
        b = _c(B)
        x = np.zeros_like(b) if X0 is None else _c(X0).copy()
        out = np.zeros(3, dtype=np.int64)
        tr = np.zeros(b.shape[-1])
        st = self.L_.oracle_solve(_p(self.links), _p(self.dims), self.kappa, self.csw, _p(b),
                                  _p(x), b.shape[-1], int(j), float(tol), int(maxit),
                                  int(max_restarts), _p(out), _p(tr))
        return x, int(st), int(out[0]), int(out[1]), int(out[2]), tr


RUNNING = -1


class Stepper:
    """The algorithm box one outer iteration at a time (bounded timing samples): the operator is
    built once; start() computes R_0, F_0 = M R_0 and W_0; each step() is one outer iteration."""

    def __init__(self, links, dims, kappa, csw, library=None):
        self.L_ = library or lib()
        self.links, self.dims = _c(links), _dims(dims)
        self.h = self.L_.oracle_create(_p(self.links), _p(self.dims), float(kappa), float(csw))
        if not self.h:
            raise RuntimeError("singular site block")

    def start(self, B, j, tol=1e-12, X0=None):
        self.B = _c(B)
        x0 = np.zeros_like(self.B) if X0 is None else _c(X0)
        self.status = self.L_.oracle_start(self.h, _p(self.B), _p(x0), self.B.shape[-1], int(j),
                                           float(tol))
        return self.status

    def step(self):
        self.status = self.L_.oracle_step(self.h)
        return self.status

    def result(self, true_resid=True):
        """(X, recursive residuals, true residuals or None, iterations, MVMs per column)."""
        X = np.empty_like(self.B)
        L = self.B.shape[-1]
        rec, tr = np.zeros(L), np.zeros(L)
        out = np.zeros(2, dtype=np.int64)
        self.L_.oracle_result(self.h, _p(X), _p(rec), _p(tr) if true_resid else None, _p(out))
        return X, rec, (tr if true_resid else None), int(out[0]), int(out[1])

    def close(self):
        if self.h:
            self.L_.oracle_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
