"""ctypes binding of the C-ABI in include/bbicggr.h: the same entry points, argument marshalling only.

Every computation runs in libbbicggr.so; this module converts torch tensors (device buffers) and
numpy arrays (host buffers) into pointers and sizes, passes the CUDA stream, and turns return
codes into exceptions.  Block vectors are complex128 arrays of shape (V, 4, 3, L) or (12*V, L).
If the library has not been built the first call raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libbbicggr.so")
HEADER = os.path.join(os.path.dirname(PKG), "include", "bbicggr.h")

WD_OK, WD_EINVAL, WD_ENOMEM, WD_ECUDA = 0, 1, 2, 3
WD_NOT_CONVERGED, WD_DIVERGED, WD_BREAKDOWN = 4, 5, 6
SOLVER_STATUSES = (WD_OK, WD_NOT_CONVERGED, WD_DIVERGED, WD_BREAKDOWN)
WD_LMAX = 16


class WDError(RuntimeError):
    def __init__(self, code: int, name: str, message: str):
        super().__init__(f"{name}: {message}")
        self.code = code


class Opts(C.Structure):
    _fields_ = [("maxit", C.c_int), ("div_thresh", C.c_double), ("max_restarts", C.c_int),
                ("precision", C.c_int), ("history", C.POINTER(C.c_double)),
                ("history_len", C.c_int), ("stall_window", C.c_int), ("net", C.c_void_p)]


class Info(C.Structure):
    _fields_ = [("status", C.c_int), ("iters", C.c_int), ("restarts", C.c_int),
                ("mvm_paper", C.c_longlong), ("mvm_actual", C.c_longlong),
                ("max_rec_resid", C.c_double), ("max_true_resid", C.c_double),
                ("rec_resid", C.POINTER(C.c_double)), ("true_resid", C.POINTER(C.c_double)),
                ("history_count", C.c_int), ("seconds", C.c_double), ("fallbacks", C.c_int)]


class Job(C.Structure):
    _fields_ = [("ctx", C.c_void_p), ("B", C.c_void_p), ("X", C.c_void_p), ("L", C.c_int),
                ("j", C.c_int), ("tol", C.c_double), ("opts", Opts), ("info", Info)]


EXCHANGE_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t,
                          C.c_void_p)
ALLREDUCE_FN = C.CFUNCTYPE(C.c_int, C.POINTER(C.c_double), C.c_int, C.c_void_p)


class DomainStruct(C.Structure):
    _fields_ = [("exchange", EXCHANGE_FN), ("allreduce", ALLREDUCE_FN), ("user", C.c_void_p)]


_lib = None


def declared_functions() -> list[str]:
    """Names of the functions include/bbicggr.h declares."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    pat = r"^[ \t]*(?:const[ \t]+)?\w+(?:[ \t]+|[ \t]*\*[ \t]*)(\w+)[ \t]*\("
    return sorted(set(re.findall(pat, text, flags=re.M)))


def lib():
    """Load libbbicggr.so (raises if it is missing: build it with paper_0907_3261_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: the CUDA library must be built "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
    L = C.CDLL(LIB_PATH)
    vp, i, d = C.c_void_p, C.c_int, C.c_double
    L.wd_create.argtypes = [C.POINTER(vp), vp, C.POINTER(C.c_int), d, d, vp]
    L.wd_destroy.argtypes = [vp]
    L.wd_destroy.restype = None
    L.wd_apply.argtypes = [vp, vp, vp, i, vp]
    L.jacobi_precond.argtypes = [vp, vp, vp, i, i, i, vp]
    L.bbicggr_solve.argtypes = [vp, vp, vp, i, i, d, C.POINTER(Opts), C.POINTER(Info), vp]
    L.jacobi_precond_noalloc.argtypes = [vp, vp, vp, i, i, vp]
    L.bbicggr_solve_batch.argtypes = [C.POINTER(Job), C.c_int, vp]
    L.bbicggr_solve_batch.restype = C.c_int
    L.bbicggr_default_opts.argtypes = [C.POINTER(Opts)]
    L.bbicggr_default_opts.restype = None
    L.wd_strerror.argtypes = [i]
    L.wd_strerror.restype = C.c_char_p
    L.wd_last_error.argtypes = []
    L.wd_last_error.restype = C.c_char_p
    L.wd_query.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_longlong), C.POINTER(d),
                           C.POINTER(d)]
    L.wd_net_create.argtypes = [C.POINTER(vp), i, i, vp]
    L.wd_net_destroy.argtypes = [vp]
    L.wd_net_destroy.restype = None
    L.wd_net_num_weights.argtypes = [vp]
    L.wd_net_num_weights.restype = C.c_longlong
    L.wd_net_set_weights.argtypes = [vp, vp]
    L.wd_net_get_weights.argtypes = [vp, vp]
    L.wd_net_apply.argtypes = [vp, vp, vp, vp, i, i, vp]
    L.wd_net_loss_grad.argtypes = [vp, vp, vp, vp, i, C.POINTER(d), vp, vp]
    L.wd_net_adam_step.argtypes = [vp, d, vp]
    for name in ("wd_net_create", "wd_net_set_weights", "wd_net_get_weights", "wd_net_apply",
                 "wd_net_loss_grad", "wd_net_adam_step"):
        getattr(L, name).restype = C.c_int
    L.wd_profile_enable.argtypes = [vp, i]
    L.wd_profile_reset.argtypes = [vp]
    L.wd_profile_read.argtypes = [vp, i, C.POINTER(C.c_longlong), C.POINTER(d)]
    L.wd_tuned_tile.argtypes = [vp, i, i, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.wd_tuned_tile.restype = C.c_int
    L.wd_set_tile.argtypes = [vp, i, i, i, i, i, i]
    L.wd_set_tile.restype = C.c_int
    L.wd_link_reals.argtypes = [vp, C.POINTER(C.c_int)]
    L.wd_link_reals.restype = C.c_int
    L.wd_set_link_reals.argtypes = [vp, i]
    L.wd_set_link_reals.restype = C.c_int
    L.wd_copy_residual.argtypes = [vp, vp, i, vp]
    L.wd_copy_residual.restype = C.c_int
    L.wd_set_apply_form.argtypes = [vp, i]
    L.wd_set_apply_form.restype = C.c_int
    L.wd_get_apply_form.argtypes = [vp]
    L.wd_get_apply_form.restype = C.c_int
    L.bb_update_u.argtypes = [vp, vp, vp, vp, i, vp, vp, i, vp]
    L.bb_update_xr.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, i, vp, vp, vp, i, vp]
    L.bb_update_pv.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, i, vp, vp, i, vp]
    for name in ("bb_update_u", "bb_update_xr", "bb_update_pv"):
        getattr(L, name).restype = C.c_int
    L.wd_set_domain.argtypes = [vp, C.POINTER(DomainStruct)]
    L.wd_set_domain.restype = C.c_int
    L.wd_profile_name.argtypes = [i]
    L.wd_profile_name.restype = C.c_char_p
    for name in ("wd_create", "wd_apply", "jacobi_precond", "jacobi_precond_noalloc",
                 "bbicggr_solve", "wd_query",
                 "wd_profile_enable", "wd_profile_reset", "wd_profile_read"):
        getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _raise(code: int):
    L = lib()
    raise WDError(code, L.wd_strerror(code).decode(), L.wd_last_error().decode())


def _check(code: int):
    if code != WD_OK:
        _raise(code)


# ---------------------------------------------------------------- buffer marshalling
def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr_and_L(x, what: str):
    """(pointer, L, keepalive) for a complex128 block vector on the device (torch) or host (numpy)."""
    if _is_torch(x):
        import torch
        if x.dtype != torch.complex128:
            raise TypeError(f"{what} must be complex128")
        if not x.is_contiguous():
            raise ValueError(f"{what} must be contiguous")
        return C.c_void_p(x.data_ptr()), int(x.shape[-1]), x
    a = np.ascontiguousarray(x, dtype=np.complex128) if not isinstance(x, np.ndarray) else x
    if a.dtype != np.complex128 or not a.flags.c_contiguous:
        raise TypeError(f"{what} must be a C-contiguous complex128 array")
    return C.c_void_p(a.ctypes.data), int(a.shape[-1]), a


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return C.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return C.c_void_p(0)
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


def _empty_like(x):
    if _is_torch(x):
        import torch
        return torch.empty_like(x)
    return np.empty_like(x)


class Context:
    """Owns a wd_ctx*; freed by wd_destroy (or when garbage collected)."""

    def __init__(self, handle: int, dims, kappa: float, csw: float):
        self.handle = C.c_void_p(handle)
        self.dims = tuple(dims)
        self.kappa = kappa
        self.csw = csw
        self.V = int(np.prod(dims))

    def close(self):
        if self.handle and self.handle.value:
            lib().wd_destroy(self.handle)
            self.handle = C.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- entry points
def wd_create(links, dims, kappa: float, csw: float, stream=None) -> Context:
    """Build A for ``links`` ([V][4][3][3] complex128, host numpy or device torch)."""
    p, _, keep = _ptr_and_L(links, "links")
    out = C.c_void_p()
    d = (C.c_int * 4)(*[int(v) for v in dims])
    _check(lib().wd_create(C.byref(out), p, d, float(kappa), float(csw), _stream(stream)))
    del keep
    return Context(out.value, dims, kappa, csw)


def wd_destroy(ctx: Context) -> None:
    ctx.close()


def wd_apply(ctx: Context, X, Y=None, stream=None):
    """Y = A X."""
    px, L, kx = _ptr_and_L(X, "X")
    if Y is None:
        Y = _empty_like(X)
    py, _, ky = _ptr_and_L(Y, "Y")
    _check(lib().wd_apply(ctx.handle, px, py, L, _stream(stream)))
    return Y


def jacobi_precond(ctx: Context, R, j: int, G=None, precision: int = 0, stream=None):
    """G = M R, j Jacobi sweeps from G = 0 (precision 0 = FP64, 1 = FP32 sweeps, 3 = FP32
    arithmetic on BF16-stored blocks, 4 = double-float sweeps)."""
    pr, L, kr = _ptr_and_L(R, "R")
    if G is None:
        G = _empty_like(R)
    pg, _, kg = _ptr_and_L(G, "G")
    _check(lib().jacobi_precond(ctx.handle, pr, pg, L, int(j), int(precision), _stream(stream)))
    return G


def jacobi_precond_noalloc(ctx: Context, R, G, j: int, stream=None):
    """G = M R like jacobi_precond, for device buffers, allocating nothing (a static 32 MiB
    scratch array in the library replaces the workspace block)."""
    pr, L, kr = _ptr_and_L(R, "R")
    pg, _, kg = _ptr_and_L(G, "G")
    _check(lib().jacobi_precond_noalloc(ctx.handle, pr, pg, L, int(j), _stream(stream)))
    return G


def bbicggr_solve(ctx: Context, B, X=None, j: int = 12, tol: float = 1e-12, maxit: int = 10000,
                  div_thresh: float = 1e2, max_restarts: int = 3, precision: int = 0,
                  history: int = 0, stall_window: int = 16, net=None, stream=None):
    """Solve A X = B by preconditioned block BiCGGR.  Returns (X, info dict).

    ``X`` (if given) holds X_0 and receives the solution; by default X_0 = 0.  ``precision``
    picks the preconditioner's arithmetic: 0 FP64 sweeps, 1 FP32 sweeps, 2 as 1 with the direction
    recurrences in double-float, 3 FP32 arithmetic on BF16 blocks, 4 double-float sweeps, 5 as 4
    with double-float direction recurrences; in 1-5 a stalled run starts over from X_0 with FP64
    sweeps (``info["fallbacks"]``).  Solver outcomes (WD_NOT_CONVERGED, WD_DIVERGED, WD_BREAKDOWN)
    are reported in ``info["status"]``; argument and CUDA errors raise WDError."""
    pb, L, kb = _ptr_and_L(B, "B")
    if X is None:
        if _is_torch(B):
            import torch
            X = torch.zeros_like(B)
        else:
            X = np.zeros_like(B)
    px, _, kx = _ptr_and_L(X, "X")
    o = Opts()
    lib().bbicggr_default_opts(C.byref(o))
    o.maxit, o.div_thresh, o.max_restarts, o.precision = int(maxit), float(div_thresh), \
        int(max_restarts), int(precision)
    o.stall_window = int(stall_window)
    if net is not None:
        o.net = net.handle
    hist = (C.c_double * max(history, 1))()
    if history:
        o.history = C.cast(hist, C.POINTER(C.c_double))
        o.history_len = int(history)
    rec = (C.c_double * L)()
    tru = (C.c_double * L)()
    info = Info()
    info.rec_resid = C.cast(rec, C.POINTER(C.c_double))
    info.true_resid = C.cast(tru, C.POINTER(C.c_double))
    rc = lib().bbicggr_solve(ctx.handle, pb, px, L, int(j), float(tol), C.byref(o),
                             C.byref(info), _stream(stream))
    if rc not in SOLVER_STATUSES:
        _raise(rc)
    out = dict(status=rc, status_name=lib().wd_strerror(rc).decode(), iters=info.iters,
               restarts=info.restarts, mvm_paper=info.mvm_paper, mvm_actual=info.mvm_actual,
               max_rec_resid=info.max_rec_resid, max_true_resid=info.max_true_resid,
               rec_resid=np.array(rec[:]), true_resid=np.array(tru[:]),
               history=np.array(hist[:info.history_count]), seconds=info.seconds,
               fallbacks=info.fallbacks)
    return X, out


def _host_c128(a, shape, what):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.complex128).reshape(shape))
    return a, C.c_void_p(a.ctypes.data)


def bb_update_u(ctx: Context, P, V, U, zeta: complex, alpha, precision: int = 0, stream=None):
    """U = (P - zeta V) alpha on device blocks (precision 1: double-float products)."""
    pp, L, k1 = _ptr_and_L(P, "P")
    pv, _, k2 = _ptr_and_L(V, "V")
    pu, _, k3 = _ptr_and_L(U, "U")
    z = np.array([complex(zeta)], dtype=np.complex128)
    al, pal = _host_c128(alpha, (L, L), "alpha")
    _check(lib().bb_update_u(ctx.handle, pp, pv, pu, L, C.c_void_p(z.ctypes.data), pal,
                             int(precision), _stream(stream)))
    return U


def bb_update_xr(ctx: Context, X, F, G, R, W, Y, Rt, zeta: complex, precision: int = 0,
                 stream=None):
    """X += zeta F + G, R -= zeta W + Y in place; returns (R~_0^H R, ||r_i||^2) of the new R."""
    ptrs, keep = [], []
    for name, b in (("X", X), ("F", F), ("G", G), ("R", R), ("W", W), ("Y", Y), ("Rt", Rt)):
        p, L, k = _ptr_and_L(b, name)
        ptrs.append(p)
        keep.append(k)
    z = np.array([complex(zeta)], dtype=np.complex128)
    rtr = np.empty((L, L), dtype=np.complex128)
    nrm = np.empty(L, dtype=np.float64)
    _check(lib().bb_update_xr(ctx.handle, *ptrs, L, C.c_void_p(z.ctypes.data),
                              C.c_void_p(rtr.ctypes.data), C.c_void_p(nrm.ctypes.data),
                              int(precision), _stream(stream)))
    return rtr, nrm


def bb_update_pv(ctx: Context, P, V, R, W, U, Y, Rt, gamma, precision: int = 0, stream=None):
    """P = R + U gamma, V = W + Y gamma (P, V written); returns R~_0^H V of the new V."""
    ptrs, keep = [], []
    for name, b in (("P", P), ("V", V), ("R", R), ("W", W), ("U", U), ("Y", Y), ("Rt", Rt)):
        p, L, k = _ptr_and_L(b, name)
        ptrs.append(p)
        keep.append(k)
    ga, pga = _host_c128(gamma, (L, L), "gamma")
    rtv = np.empty((L, L), dtype=np.complex128)
    _check(lib().bb_update_pv(ctx.handle, *ptrs, L, pga, C.c_void_p(rtv.ctypes.data),
                              int(precision), _stream(stream)))
    return rtv


def wd_set_domain(ctx: Context, exchange, allreduce) -> None:
    """Make ``ctx`` (built on a t-slab extended by one halo slice on each side) one rank of a
    domain-decomposed solve.  ``exchange(send_lo, send_hi, recv_lo, recv_hi)`` gets four uint8
    numpy views of the library's host staging buffers; ``allreduce(buf)`` a float64 view to sum
    over ranks in place.  An exception in either fails the library call.  ``exchange=None``
    clears the domain."""
    if exchange is None:
        _check(lib().wd_set_domain(ctx.handle, None))
        ctx._domain = None
        return

    def ex(a, b, c, d, nbytes, user):
        try:
            view = lambda p: np.ctypeslib.as_array((C.c_uint8 * nbytes).from_address(p))
            exchange(view(a), view(b), view(c), view(d))
            return 0
        except Exception:
            return 1

    def ar(buf, n, user):
        try:
            allreduce(np.ctypeslib.as_array(buf, shape=(n,)))
            return 0
        except Exception:
            return 1

    dom = DomainStruct(EXCHANGE_FN(ex), ALLREDUCE_FN(ar), None)
    _check(lib().wd_set_domain(ctx.handle, C.byref(dom)))
    ctx._domain = dom          # the callbacks live as long as the context uses them


WD_K_COUNT = 15


def wd_profile_enable(ctx: Context, timing_on: bool = True) -> None:
    """Count kernel launches per class; with timing_on also time them with CUDA events."""
    _check(lib().wd_profile_enable(ctx.handle, int(bool(timing_on))))


def wd_profile_reset(ctx: Context) -> None:
    _check(lib().wd_profile_reset(ctx.handle))


def wd_profile_read(ctx: Context) -> dict:
    """{kernel class name: (kernel launches, summed device ms)} since the last reset."""
    out = {}
    for k in range(WD_K_COUNT):
        n = C.c_longlong()
        ms = C.c_double()
        _check(lib().wd_profile_read(ctx.handle, k, C.byref(n), C.byref(ms)))
        out[lib().wd_profile_name(k).decode()] = (int(n.value), float(ms.value))
    return out


def wd_tuned_tile(ctx: Context, L: int, precision: int = 1):
    """(RHS per thread, threads per CTA, min CTAs per SM, staged) of the low-precision sweep for
    L (precision 1: FP32 blocks, 3: BF16 blocks, 4: double-float sweeps, where staged 1 is the
    packed FP32x2 variant), or None before the autotuner ran."""
    r, b, m, st = C.c_int(), C.c_int(), C.c_int(), C.c_int()
    if lib().wd_tuned_tile(ctx.handle, int(L), int(precision), C.byref(r), C.byref(b),
                           C.byref(m), C.byref(st)) != WD_OK:
        return None
    return int(r.value), int(b.value), int(m.value), int(st.value)


def wd_set_tile(ctx: Context, L: int, rhs_per_thread: int, block: int, min_blocks: int = 0,
                staged: int = 0, precision: int = 1) -> None:
    """Fix the low-precision sweep's tile for this L and storage instead of autotuning it."""
    _check(lib().wd_set_tile(ctx.handle, int(L), int(precision), int(rhs_per_thread), int(block),
                             int(min_blocks), int(staged)))


def wd_link_reals(ctx: Context) -> int:
    """12 when the low-precision sweeps rebuild row 2 of each link, 18 when they read it."""
    r = C.c_int()
    _check(lib().wd_link_reals(ctx.handle, C.byref(r)))
    return int(r.value)


def wd_set_link_reals(ctx: Context, reals: int) -> None:
    """Choose the link format of the low-precision sweeps (12 needs special unitary links)."""
    _check(lib().wd_set_link_reals(ctx.handle, int(reals)))


def wd_copy_residual(ctx: Context, R):
    """Copy the last solve's recursive residual block into R (a tensor shaped like B)."""
    pr, L, k = _ptr_and_L(R, "R")
    _check(lib().wd_copy_residual(ctx.handle, pr, L, _stream(None)))
    return R


def wd_set_apply_form(ctx: Context, form: int) -> None:
    """Form of the FP64 stencils: 1 = hopping sums exact on the FP32 lanes (unitary links), 0 = FP64 pipe."""
    _check(lib().wd_set_apply_form(ctx.handle, int(form)))


def wd_get_apply_form(ctx: Context) -> int:
    return int(lib().wd_get_apply_form(ctx.handle))


# ---------------------------------------------------------------- learned preconditioner
class Net:
    """Owns a wd_net*: weights, Adam state and workspace of one preconditioner network."""

    def __init__(self, handle: int, layers: int, hidden: int):
        self.handle = C.c_void_p(handle)
        self.layers = layers
        self.hidden = hidden
        self.channels = [1] + [hidden] * (layers - 1) + [1]

    def shapes(self):
        ch = self.channels
        return [(9, ch[i + 1], ch[i], 4, 4) for i in range(self.layers)]

    def close(self):
        if self.handle and self.handle.value:
            lib().wd_net_destroy(self.handle)
            self.handle = C.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _flat_weights(weights):
    return np.ascontiguousarray(np.concatenate([np.asarray(w, np.complex128).ravel()
                                                for w in weights]))


def wd_net_create(layers: int, hidden: int, weights) -> Net:
    """Network with the given initial weights (list of [9][C_out][C_in][4][4] arrays)."""
    flat = _flat_weights(weights)
    out = C.c_void_p()
    _check(lib().wd_net_create(C.byref(out), int(layers), int(hidden), C.c_void_p(flat.ctypes.data)))
    net = Net(out.value, layers, hidden)
    if lib().wd_net_num_weights(net.handle) != flat.size:
        raise ValueError("weights do not match the architecture")
    return net


def wd_net_destroy(net: Net) -> None:
    net.close()


def _unflatten(net: Net, flat):
    out, off = [], 0
    for shp in net.shapes():
        n = int(np.prod(shp))
        out.append(flat[off:off + n].reshape(shp))
        off += n
    return out


def wd_net_get_weights(net: Net):
    flat = np.empty(lib().wd_net_num_weights(net.handle), dtype=np.complex128)
    _check(lib().wd_net_get_weights(net.handle, C.c_void_p(flat.ctypes.data)))
    return _unflatten(net, flat)


def wd_net_set_weights(net: Net, weights) -> None:
    flat = _flat_weights(weights)
    _check(lib().wd_net_set_weights(net.handle, C.c_void_p(flat.ctypes.data)))


def wd_net_apply(ctx: Context, net: Net, R, G=None, bf16: bool = False, stream=None):
    """G = N(R) for device (torch) blocks; bf16 stores the activations in BF16."""
    pr, L, kr = _ptr_and_L(R, "R")
    if G is None:
        G = _empty_like(R)
    pg, _, kg = _ptr_and_L(G, "G")
    _check(lib().wd_net_apply(ctx.handle, net.handle, pr, pg, L, int(bool(bf16)), _stream(stream)))
    return G


def wd_net_loss_grad(ctx: Context, net: Net, R, E, want_grad: bool = True, stream=None):
    """(loss, gradient d loss / d conj(W) as a list of arrays or None) for device blocks R, E."""
    pr, L, kr = _ptr_and_L(R, "R")
    pe, _, ke = _ptr_and_L(E, "E")
    loss = C.c_double()
    flat = np.empty(lib().wd_net_num_weights(net.handle), dtype=np.complex128) if want_grad else None
    _check(lib().wd_net_loss_grad(ctx.handle, net.handle, pr, pe, L, C.byref(loss),
                                  C.c_void_p(flat.ctypes.data) if want_grad else None,
                                  _stream(stream)))
    return float(loss.value), (_unflatten(net, flat) if want_grad else None)


def wd_net_adam_step(net: Net, lr: float, stream=None) -> None:
    _check(lib().wd_net_adam_step(net.handle, float(lr), _stream(stream)))



def bbicggr_solve_batch(jobs, stream=None):
    """Solve several independent systems in one CUDA graph with device-side iteration control.

    ``jobs``: list of dicts with keys ctx, B, X (device torch tensors; X holds X_0), and optional
    j (12), tol (1e-12), maxit, div_thresh, max_restarts, precision, stall_window, net, history.
    Returns the list of info dicts (the keys of bbicggr_solve's; mvm_actual is not counted)."""
    n = len(jobs)
    arr = (Job * n)()
    keep = []
    for i, jb in enumerate(jobs):
        pb, L, kb = _ptr_and_L(jb["B"], "B")
        px, _, kx = _ptr_and_L(jb["X"], "X")
        o = Opts()
        lib().bbicggr_default_opts(C.byref(o))
        o.maxit = int(jb.get("maxit", 10000))
        o.div_thresh = float(jb.get("div_thresh", 1e2))
        o.precision = int(jb.get("precision", 0))
        o.stall_window = int(jb.get("stall_window", 16))
        o.max_restarts = int(jb.get("max_restarts", 3))
        if jb.get("net") is not None:
            o.net = jb["net"].handle
        hist = (C.c_double * max(int(jb.get("history", 0)), 1))()
        if jb.get("history", 0):
            o.history = C.cast(hist, C.POINTER(C.c_double))
            o.history_len = int(jb["history"])
        rec = (C.c_double * L)()
        tru = (C.c_double * L)()
        arr[i].ctx = jb["ctx"].handle
        arr[i].B = pb
        arr[i].X = px
        arr[i].L = L
        arr[i].j = int(jb.get("j", 12))
        arr[i].tol = float(jb.get("tol", 1e-12))
        arr[i].opts = o
        arr[i].info.rec_resid = C.cast(rec, C.POINTER(C.c_double))
        arr[i].info.true_resid = C.cast(tru, C.POINTER(C.c_double))
        keep.append((kb, kx, hist, rec, tru))
    rc = lib().bbicggr_solve_batch(arr, n, _stream(stream))
    if rc not in SOLVER_STATUSES:
        _raise(rc)
    out = []
    for i in range(n):
        info = arr[i].info
        hist, rec, tru = keep[i][2], keep[i][3], keep[i][4]
        out.append(dict(status=info.status, status_name=lib().wd_strerror(info.status).decode(),
                        iters=info.iters, restarts=info.restarts, fallbacks=info.fallbacks,
                        mvm_paper=info.mvm_paper,
                        max_rec_resid=info.max_rec_resid, max_true_resid=info.max_true_resid,
                        rec_resid=np.array(rec[:]), true_resid=np.array(tru[:]),
                        history=np.array(hist[:info.history_count]), seconds=info.seconds))
    return out
