"""The C-ABI library loads and exports every function include/pfgpu.h declares, and rejects
bad arguments before touching the GPU (these calls run on a machine without one)."""
import ctypes

import pytest

from paper_2109_02598_gb300 import _lib
from paper_2109_02598_gb300.build import build


@pytest.fixture(scope="module")
def lib():
    build()
    return _lib.load()


def test_exports_every_declared_symbol(lib):
    declared = _lib.header_functions()
    assert len(declared) >= 14
    for name in declared:
        assert hasattr(lib, name), name
    # and the binding declares a signature for each of them
    assert set(declared) <= set(_lib.SIGNATURES)


def test_version(lib):
    assert lib.pf_version() >= 10000


def _err(lib):
    return lib.pf_last_error().decode()


def test_create_grid_rejects_bad_arguments(lib):
    h = ctypes.c_void_p()
    n = (ctypes.c_int64 * 3)(16, 16, 16)
    assert lib.pf_create_grid(4, n, 1, 1.0, None, ctypes.byref(h)) == _lib.PF_ERR_INVALID_ARG
    assert "dim" in _err(lib)
    assert lib.pf_create_grid(2, n, 5, 1.0, None, ctypes.byref(h)) == _lib.PF_ERR_INVALID_ARG
    assert lib.pf_create_grid(2, n, 1, 0.0, None, ctypes.byref(h)) == _lib.PF_ERR_INVALID_ARG
    bad = (ctypes.c_int64 * 3)(0, 16, 16)
    assert lib.pf_create_grid(2, bad, 1, 1.0, None, ctypes.byref(h)) == _lib.PF_ERR_INVALID_ARG
    assert lib.pf_create_grid(2, n, 1, 1.0, None, None) == _lib.PF_ERR_INVALID_ARG
    assert lib.pf_create_grid(2, n, 1, float("inf"), None, ctypes.byref(h)) == _lib.PF_ERR_INVALID_ARG


def test_size_checks_do_not_overflow(lib):
    """2^30 x 2^30 x 16 floats is 2^64: a check that multiplies the sides wraps to 0 and passes.
    Both entry points must reject it (before any device work, so this runs without a GPU)."""
    h = ctypes.c_void_p()
    big = (ctypes.c_int64 * 3)(1 << 30, 1 << 30, 16)
    assert lib.pf_create_grid(3, big, 1, 1.0, None, ctypes.byref(h)) == _lib.PF_ERR_INVALID_ARG
    assert "2^36" in _err(lib)
    fake = ctypes.c_void_p(256)  # never dereferenced: the call fails validation first
    out = ctypes.c_void_p(512)
    rc = lib.pf_reduce_noalloc(_lib.PF_REDUCE_MASS, 3, big, 1 << 30, fake, 1.0, 0.0, 0.0, out, None)
    assert rc == _lib.PF_ERR_INVALID_ARG and "2^36" in _err(lib)
    ok = (ctypes.c_int64 * 3)(8, 8, 8)
    for bad_h in (float("inf"), float("nan"), 0.0, -1.0):
        rc = lib.pf_reduce_noalloc(_lib.PF_REDUCE_MASS, 3, ok, 8, fake, bad_h, 0.0, 0.0, out, None)
        assert rc == _lib.PF_ERR_INVALID_ARG and "h must be" in _err(lib)


def test_calls_on_null_handle_fail_cleanly(lib):
    c = (ctypes.c_double * 2)(1.0, 1.0)
    assert lib.pf_set_model(None, 1, c, 2, 0.05, 0) == _lib.PF_ERR_INVALID_ARG
    assert lib.pf_step(None, 1) == _lib.PF_ERR_INVALID_ARG
    out = ctypes.c_double()
    assert lib.pf_reduce(None, 1, 0, ctypes.byref(out)) == _lib.PF_ERR_INVALID_ARG
    lib.pf_destroy(None)  # no-op


def test_loader_fails_loudly_without_library(tmp_path):
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        saved = _lib._lib
        _lib._lib = None
        try:
            _lib.load(str(tmp_path / "missing.so"))
        finally:
            _lib._lib = saved


def test_spectral_and_structure_factor_reject_bad_arguments(lib):
    h = ctypes.c_void_p()
    n = (ctypes.c_int64 * 3)(16, 16, 16)
    c2 = (ctypes.c_double * 5)(1.0, 1.0, 1.0, 1.0, 1.0)
    INV = _lib.PF_ERR_INVALID_ARG
    assert lib.pf_spectral_create(2, n, 1.0, 3, c2, 4, 0.1, None, ctypes.byref(h)) == INV
    assert "Models A, B and C" in _err(lib)
    assert lib.pf_spectral_create(2, n, 1.0, 1, c2, 3, 0.1, None, ctypes.byref(h)) == INV
    assert lib.pf_spectral_create(2, n, 1.0, 1, c2, 2, 0.0, None, ctypes.byref(h)) == INV
    assert lib.pf_spectral_create(2, n, 0.0, 1, c2, 2, 0.1, None, ctypes.byref(h)) == INV
    assert lib.pf_spectral_create(4, n, 1.0, 1, c2, 2, 0.1, None, ctypes.byref(h)) == INV
    big = (ctypes.c_int64 * 3)(1 << 15, 1 << 15, 2)
    assert lib.pf_spectral_create(3, big, 1.0, 1, c2, 2, 0.1, None, ctypes.byref(h)) == INV
    thin = (ctypes.c_int64 * 3)(1, 16, 1)
    assert lib.pf_spectral_create(2, thin, 1.0, 1, c2, 2, 0.1, None, ctypes.byref(h)) == INV
    assert lib.pf_spectral_step(None, 1) == INV
    assert lib.pf_spectral_write_field(None, 0, None, 0) == INV
    assert lib.pf_spectral_read_field(None, 0, None, 0) == INV
    assert lib.pf_spectral_synchronize(None) == INV
    lib.pf_spectral_destroy(None)  # no-op
    cen = (ctypes.c_double * 8)()
    mean = (ctypes.c_double * 8)()
    cnt = (ctypes.c_int64 * 8)()
    fake = ctypes.c_void_p(256)  # never dereferenced: every call below fails validation
    assert lib.pf_structure_factor(2, n, 16, fake, 1.0, 0, cen, mean, cnt, None) == INV
    assert lib.pf_structure_factor(2, n, 16, fake, 1.0, 1025, cen, mean, cnt, None) == INV
    assert lib.pf_structure_factor(2, n, 15, fake, 1.0, 8, cen, mean, cnt, None) == INV
    assert lib.pf_structure_factor(2, n, 16, None, 1.0, 8, cen, mean, cnt, None) == INV
    assert lib.pf_structure_factor(2, n, 16, fake, -1.0, 8, cen, mean, cnt, None) == INV
