"""The C-ABI library builds for sm_103a, loads, and exports every symbol include/bbicggr.h declares
(no GPU needed; no compute calls)."""
import ctypes

import pytest


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_0907_3261_gb300 import _lib
    return _lib


def test_every_declared_symbol_is_exported(lib):
    names = lib.declared_functions()
    assert {"wd_create", "wd_destroy", "wd_apply", "jacobi_precond", "bbicggr_solve",
            "wd_strerror", "bbicggr_default_opts"} <= set(names)
    so = ctypes.CDLL(lib.LIB_PATH)
    for n in names:
        assert hasattr(so, n), n


def test_host_only_entry_points(lib):
    L = lib.lib()
    assert L.wd_strerror(0) == b"WD_OK"
    assert L.wd_strerror(6) == b"WD_BREAKDOWN"
    o = lib.Opts()
    L.bbicggr_default_opts(ctypes.byref(o))
    assert o.maxit == 10000 and o.div_thresh == 1e2 and o.max_restarts == 3 and o.precision == 0
    assert o.stall_window == 16


def test_argument_errors_need_no_gpu(lib):
    """Invalid arguments are rejected before any CUDA call."""
    L = lib.lib()
    out = ctypes.c_void_p()
    dims = (ctypes.c_int * 4)(1, 4, 4, 4)
    assert L.wd_create(ctypes.byref(out), ctypes.c_void_p(16), dims, 0.1, 1.0, None) == 1
    assert out.value is None
    assert L.wd_apply(None, None, None, 4, None) == 1
    assert L.bbicggr_solve(None, None, None, 4, 2, 1e-12, None, None, None) == 1


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_0907_3261_gb300 import _lib
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        _lib.lib()
