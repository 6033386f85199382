"""pf_reduce_noalloc: the mass / energy reduction for callers that cannot allocate device
memory (a host framework that owns the whole device through its own allocator, or a
latency-critical loop that cannot afford cudaMalloc's implicit synchronisation).  The
library keeps the reduction's partial sums in a fixed device array instead of allocating.

Checked through the C ABI against pf_reduce (which uses the grid's own scratch) on two
calls in a row, each on a different field and reduction, so a stale scratch array from the
first call would show up in the second.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

import synthetic
from paper_2109_02598_gb300 import _lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_02598_gb300.build import build
    build()
    import paper_2109_02598_gb300 as pf
    return pf


def _noalloc(lib, what, grid, c1, c2, out, stream):
    ptr = ctypes.c_void_p()
    pitch = ctypes.c_int64()
    plane = ctypes.c_int64()
    _lib.check(lib.pf_field_view(grid.handle, 0, ctypes.byref(ptr), ctypes.byref(pitch),
                                 ctypes.byref(plane)))
    nx, ny = grid.shape[-1], grid.shape[-2]
    nz = grid.shape[0] if grid.dim == 3 else 1
    n = (ctypes.c_int64 * 3)(nx, ny, nz)
    return lib.pf_reduce_noalloc(what, grid.dim, n, pitch.value, ptr, grid.h, c1, c2,
                                 ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))


def test_noalloc_matches_pf_reduce_on_consecutive_calls(pf):
    import torch
    lib = _lib.load()
    stream = torch.cuda.current_stream().cuda_stream
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    a = synthetic.allen_cahn_init((9, 30, 70), seed=41, lo=-0.9, hi=0.9)
    b = synthetic.cahn_hilliard_init((123, 77), seed=42, amp=0.4)
    ga = pf.Grid(a.shape, 1, 0.8).set_model("ac", (0.9, 1.1), 0.01)
    ga.write_field(0, a)
    gb = pf.Grid(b.shape, 1, 1.3).set_model("ch", (1.2, 0.7, 1.0), 0.001)
    gb.write_field(0, b)
    ref_first = ga.energy()
    ref_second = gb.mass()
    # two calls in a row through the shared scratch array
    assert _noalloc(lib, _lib.PF_REDUCE_ENERGY, ga, 0.9, 1.1, out[0:1], stream) == _lib.PF_OK
    assert _noalloc(lib, _lib.PF_REDUCE_MASS, gb, 0.0, 0.0, out[1:2], stream) == _lib.PF_OK
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert abs(got[0] - ref_first) <= 1e-12 * abs(ref_first)
    assert abs(got[1] - ref_second) <= 1e-12 * max(1.0, np.abs(b.astype(np.float64)).sum())
    # and again in the other order on the same arrays
    assert _noalloc(lib, _lib.PF_REDUCE_MASS, ga, 0.0, 0.0, out[0:1], stream) == _lib.PF_OK
    assert _noalloc(lib, _lib.PF_REDUCE_ENERGY, gb, 1.2, 0.7, out[1:2], stream) == _lib.PF_OK
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    ma, eb = ga.mass(), gb.energy()
    assert abs(got[0] - ma) <= 1e-12 * max(1.0, np.abs(a.astype(np.float64)).sum())
    assert abs(got[1] - eb) <= 1e-12 * abs(eb)
    # the property the entry point exists for: once the first call on the device has run,
    # further calls take no device memory
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    for _ in range(4):
        assert _noalloc(lib, _lib.PF_REDUCE_ENERGY, ga, 0.9, 1.1, out[0:1], stream) == _lib.PF_OK
        assert _noalloc(lib, _lib.PF_REDUCE_MASS, gb, 0.0, 0.0, out[1:2], stream) == _lib.PF_OK
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free_before
    ga.close()
    gb.close()


def test_noalloc_rejects_bad_sizes(pf):
    import torch
    lib = _lib.load()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    field = torch.zeros(64, dtype=torch.float32, device="cuda")
    big = (ctypes.c_int64 * 3)(1 << 31, 4, 1)
    rc = lib.pf_reduce_noalloc(_lib.PF_REDUCE_MASS, 2, big, 1 << 31,
                               ctypes.c_void_p(field.data_ptr()), 1.0, 0.0, 0.0,
                               ctypes.c_void_p(out.data_ptr()), None)
    assert rc == _lib.PF_ERR_INVALID_ARG and b"2^30" in lib.pf_last_error()
    n = (ctypes.c_int64 * 3)(8, 8, 1)
    rc = lib.pf_reduce_noalloc(_lib.PF_REDUCE_MASS, 2, n, 4, ctypes.c_void_p(field.data_ptr()),
                               1.0, 0.0, 0.0, ctypes.c_void_p(out.data_ptr()), None)
    assert rc == _lib.PF_ERR_INVALID_ARG and b"pitch" in lib.pf_last_error()
    rc = lib.pf_reduce_noalloc(_lib.PF_REDUCE_MASS, 2, n, 8, ctypes.c_void_p(field.data_ptr()),
                               float("inf"), 0.0, 0.0, ctypes.c_void_p(out.data_ptr()), None)
    assert rc == _lib.PF_ERR_INVALID_ARG and b"finite" in lib.pf_last_error()
