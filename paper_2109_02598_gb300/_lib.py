"""ctypes loader for libpfgpu.so (the C ABI of include/pfgpu.h).

Argument marshalling only: every step of the computation runs in the library's CUDA
kernels.  There is no fallback: if the library is missing, loading raises.
"""
from __future__ import annotations

import ctypes
import os
import re

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "_build", "libpfgpu.so")
# PFGPU_CHECKED=1 loads the checked variant (built with -DPF_CHECK: shared memory filled with
# NaN before every staging) instead; a process uses one or the other.
CHECKED_LIB_PATH = os.path.join(PKG, "_build", "checked", "libpfgpu_checked.so")
HEADER = os.path.join(os.path.dirname(PKG), "include", "pfgpu.h")

PF_OK = 0
PF_ERR_INVALID_ARG = -1
PF_ERR_OOM = -2
PF_ERR_CUDA = -3
PF_ERR_UNSTABLE_DT = -4
PF_ERR_NONFINITE = -5
PF_ERR_STATE = -6
PF_ERR_TIMEOUT = -7

PF_TILE_BANDS = -1  # tile_y of the band kernel (with tile_x = nx)
PF_TILE_STRIPS = -2  # tile_y of the strip kernel (with tile_x = 128 or 64)

PF_MODEL_AC = 1
PF_MODEL_CH = 2
PF_MODEL_GS = 3
PF_MODEL_C = 4
PF_MODEL_RD = 5
MODEL_IDS = {"ac": PF_MODEL_AC, "ch": PF_MODEL_CH, "gs": PF_MODEL_GS, "c": PF_MODEL_C,
             "rd": PF_MODEL_RD}
MODEL_FIELDS = {"ac": 1, "ch": 1, "gs": 2, "c": 2}

STENCIL_IDS = {"std": 0, "iso": 1, "4th": 2, "iso27": 3}

PF_REDUCE_MASS = 1
PF_REDUCE_ENERGY = 2

class GS2DSpec(ctypes.Structure):
    """pf_gs2d_spec: one batched 2D Gray-Scott instance."""
    _fields_ = [("nx", ctypes.c_int64), ("ny", ctypes.c_int64), ("Du", ctypes.c_double),
                ("Dv", ctypes.c_double), ("F", ctypes.c_double), ("k", ctypes.c_double)]


_c_int64_p = ctypes.POINTER(ctypes.c_int64)
_c_double_p = ctypes.POINTER(ctypes.c_double)
_c_int_p = ctypes.POINTER(ctypes.c_int)
_vp = ctypes.c_void_p

# name -> (restype, argtypes)
SIGNATURES = {
    "pf_version": (ctypes.c_int, []),
    "pf_last_error": (ctypes.c_char_p, []),
    "pf_create_grid": (ctypes.c_int, [ctypes.c_int, _c_int64_p, ctypes.c_int, ctypes.c_double,
                                      _vp, ctypes.POINTER(_vp)]),
    "pf_destroy": (None, [_vp]),
    "pf_set_model": (ctypes.c_int, [_vp, ctypes.c_int, _c_double_p, ctypes.c_int,
                                    ctypes.c_double, ctypes.c_int]),
    "pf_write_field": (ctypes.c_int, [_vp, ctypes.c_int, _vp, ctypes.c_int]),
    "pf_read_field": (ctypes.c_int, [_vp, ctypes.c_int, _vp, ctypes.c_int]),
    "pf_copy_planes": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int64, ctypes.c_int64, _vp,
                                      ctypes.c_int, ctypes.c_int]),
    "pf_step": (ctypes.c_int, [_vp, ctypes.c_int64]),
    "pf_write_field_host_async": (ctypes.c_int, [_vp, ctypes.c_int, _vp]),
    "pf_read_field_host_async": (ctypes.c_int, [_vp, ctypes.c_int, _vp]),
    "pf_reduce": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _c_double_p]),
    "pf_set_stencil": (ctypes.c_int, [_vp, ctypes.c_int]),
    "pf_set_tuning": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "pf_get_tuning": (ctypes.c_int, [_vp, _c_int_p, _c_int_p, _c_int_p]),
    "pf_autotune": (ctypes.c_int, [_vp, ctypes.c_int, _c_int_p, _c_int_p, _c_int_p]),
    "pf_synchronize": (ctypes.c_int, [_vp]),
    "pf_field_view": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(_vp), _c_int64_p,
                                     _c_int64_p]),
    "pf_batch_create": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(GS2DSpec), ctypes.c_double,
                                       ctypes.c_double, _vp, ctypes.POINTER(_vp)]),
    "pf_batch_destroy": (None, [_vp]),
    "pf_batch_write_field": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _vp, ctypes.c_int]),
    "pf_batch_read_field": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _vp, ctypes.c_int]),
    "pf_batch_set_tuning": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "pf_batch_get_tuning": (ctypes.c_int, [_vp, _c_int_p, _c_int_p, _c_int_p]),
    "pf_batch_autotune": (ctypes.c_int, [_vp, ctypes.c_int, _c_int_p, _c_int_p, _c_int_p]),
    "pf_batch_run": (ctypes.c_int, [_vp, ctypes.c_int64]),
    "pf_batch_synchronize": (ctypes.c_int, [_vp]),
    "pf_batch_info": (ctypes.c_int, [_vp, _c_int64_p, _c_int64_p]),
    "pf_adj_forward": (ctypes.c_int, [_vp, ctypes.c_int64, ctypes.c_int64]),
    "pf_adj_backward": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, _vp, _vp, _c_double_p]),
    "pf_spectral_create": (ctypes.c_int, [ctypes.c_int, _c_int64_p, ctypes.c_double, ctypes.c_int,
                                          _c_double_p, ctypes.c_int, ctypes.c_double, _vp,
                                          ctypes.POINTER(_vp)]),
    "pf_spectral_destroy": (None, [_vp]),
    "pf_spectral_write_field": (ctypes.c_int, [_vp, ctypes.c_int, _vp, ctypes.c_int]),
    "pf_spectral_read_field": (ctypes.c_int, [_vp, ctypes.c_int, _vp, ctypes.c_int]),
    "pf_spectral_step": (ctypes.c_int, [_vp, ctypes.c_int64]),
    "pf_spectral_synchronize": (ctypes.c_int, [_vp]),
    "pf_spectral_set_engine": (ctypes.c_int, [_vp, ctypes.c_int]),
    "pf_spectral_get_engine": (ctypes.c_int, [_vp, _c_int_p]),
    "pf_structure_factor": (ctypes.c_int, [ctypes.c_int, _c_int64_p, ctypes.c_int64, _vp,
                                           ctypes.c_double, ctypes.c_int, _c_double_p,
                                           _c_double_p, _c_int64_p, _vp]),
    "pf_porod_fit": (ctypes.c_int, [ctypes.c_int, _c_double_p, _c_double_p, _c_int64_p,
                                    ctypes.c_double, ctypes.c_double, _c_double_p, _c_double_p,
                                    _c_int_p]),
    "pf_selftest_wait_timeout": (ctypes.c_int, [ctypes.c_int64, _vp]),
    "pf_reduce_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _c_int64_p, ctypes.c_int64,
                                         _vp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                         _vp, _vp]),
}


class PfError(RuntimeError):
    """A libpfgpu call returned a negative status."""

    def __init__(self, code: int, message: str):
        super().__init__(f"[{code}] {message}")
        self.code = code


_lib = None


def load(path: str = None):
    """Load the library (once) and declare its signatures. Raises if it is not built."""
    global _lib
    if _lib is not None:
        return _lib
    if path is None:
        path = CHECKED_LIB_PATH if os.environ.get("PFGPU_CHECKED") == "1" else LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(
            f"libpfgpu.so not found at {path}: build it with __graft_entry__.build() "
            "(there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(rc: int) -> int:
    if rc != PF_OK:
        msg = load().pf_last_error()
        raise PfError(rc, msg.decode() if msg else "")
    return rc


def header_functions(path: str = HEADER):
    """Names of the functions include/pfgpu.h declares."""
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pf_[a-z0-9_]+)\s*\(", text)))
