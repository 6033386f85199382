"""Semi-implicit Fourier spectral solver, structure factor and Porod fit (argument marshalling
over include/pfgpu.h's pf_spectral_*, pf_structure_factor and pf_porod_fit calls).

``Spectral`` is the paper's second solver (Sec. 2.4.2) for Models A, B and C (Sec. 3): each
equation of motion split into a linear part, integrated exactly over a step in Fourier
space, and an explicit nonlinear part.  ``structure_factor`` is the radially averaged
S(|k|) of the phase indicator psi > 0.  Shapes follow numpy order, x fastest.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import MODEL_FIELDS, MODEL_IDS, check
from .grid import _stream_handle, _torch


def _dims(shape):
    shape = tuple(int(s) for s in shape)
    if len(shape) not in (2, 3):
        raise ValueError("shape must be (ny, nx) or (nz, ny, nx)")
    nx, ny = shape[-1], shape[-2]
    nz = shape[0] if len(shape) == 3 else 1
    return shape, (ctypes.c_int64 * 3)(nx, ny, nz)


class Spectral:
    """Spectral solver state (Fourier space, on the GPU) of one model on a periodic grid."""

    def __init__(self, shape, model: str, coeffs, dt: float, h: float = 1.0, stream=None):
        torch = _torch()
        self._lib = _lib.load()
        self.shape, n = _dims(shape)
        self.dim = len(self.shape)
        self.model = model
        self.n_fields = MODEL_FIELDS[model]
        self.coeffs = tuple(float(x) for x in coeffs)
        self.dt = float(dt)
        self.h = float(h)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        c = (ctypes.c_double * len(self.coeffs))(*self.coeffs)
        handle = ctypes.c_void_p()
        check(self._lib.pf_spectral_create(self.dim, n, self.h, MODEL_IDS[model], c,
                                           len(self.coeffs), self.dt,
                                           ctypes.c_void_p(_stream_handle(self.stream)),
                                           ctypes.byref(handle)))
        self._h = handle

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.pf_spectral_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def sites(self) -> int:
        return int(np.prod(self.shape))

    def write_field(self, field: int, data):
        """Copy in a dense float32 array of ``shape``: numpy (host) or torch (host/CUDA)."""
        if hasattr(data, "data_ptr"):
            torch = _torch()
            t = data.detach().to(torch.float32).contiguous()
            if tuple(t.shape) != self.shape:
                raise ValueError(f"field shape {tuple(t.shape)} != grid shape {self.shape}")
            check(self._lib.pf_spectral_write_field(self._h, field, ctypes.c_void_p(t.data_ptr()),
                                                    1 if t.is_cuda else 0))
            if t.is_cuda:
                self.synchronize()  # the copy reads t when the stream reaches it
            return self
        a = np.ascontiguousarray(data, dtype=np.float32)
        if a.shape != self.shape:
            raise ValueError(f"field shape {a.shape} != grid shape {self.shape}")
        check(self._lib.pf_spectral_write_field(self._h, field,
                                                a.ctypes.data_as(ctypes.c_void_p), 0))
        return self

    def write_fields(self, fields):
        for i, f in enumerate(fields):
            self.write_field(i, f)
        return self

    def read_field(self, field: int, device: bool = False, out=None):
        """Real-space field ``field`` as numpy (default) or a CUDA torch tensor."""
        if device or (out is not None and hasattr(out, "data_ptr")):
            torch = _torch()
            if out is None:
                out = torch.empty(self.shape, dtype=torch.float32, device="cuda")
            check(self._lib.pf_spectral_read_field(self._h, field, ctypes.c_void_p(out.data_ptr()),
                                                   1 if out.is_cuda else 0))
            return out
        a = np.empty(self.shape, dtype=np.float32) if out is None else out
        check(self._lib.pf_spectral_read_field(self._h, field, a.ctypes.data_as(ctypes.c_void_p),
                                               0))
        return a

    def read_fields(self, device: bool = False):
        return tuple(self.read_field(i, device=device) for i in range(self.n_fields))

    def step(self, n_steps: int = 1):
        check(self._lib.pf_spectral_step(self._h, int(n_steps)))
        return self

    ENGINES = {"auto": 0, "cufft": 1, "fused": 2}

    def set_engine(self, engine: str = "auto"):
        """"cufft", "fused" (power-of-two sides; in 3D a (y, z) slab that fits a CTA) or "auto"."""
        check(self._lib.pf_spectral_set_engine(self._h, self.ENGINES[engine]))
        return self

    @property
    def engine(self) -> str:
        e = ctypes.c_int()
        check(self._lib.pf_spectral_get_engine(self._h, ctypes.byref(e)))
        return {1: "cufft", 2: "fused"}[e.value]

    def synchronize(self):
        check(self._lib.pf_spectral_synchronize(self._h))


def structure_factor_view(dev_ptr: int, shape, pitch: int, h: float = 1.0, n_bins: int = 32,
                          stream=None):
    """S(|k|) of a float32 device field at ``dev_ptr`` laid out [nz][ny][pitch]."""
    lib = _lib.load()
    shape, n = _dims(shape)
    centres = np.empty(n_bins, dtype=np.float64)
    mean = np.empty(n_bins, dtype=np.float64)
    counts = np.empty(n_bins, dtype=np.int64)
    dp = ctypes.POINTER(ctypes.c_double)
    check(lib.pf_structure_factor(len(shape), n, int(pitch), ctypes.c_void_p(dev_ptr), float(h),
                                  int(n_bins), centres.ctypes.data_as(dp), mean.ctypes.data_as(dp),
                                  counts.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                  ctypes.c_void_p(_stream_handle(stream))))
    return centres, mean, counts


def structure_factor(psi, h: float = 1.0, n_bins: int = 32, stream=None):
    """Radially averaged S(|k|) of rho = [psi > 0] (Sec. 3): (bin centres, mean S, counts).

    ``psi`` is a numpy array or a torch tensor (copied to the GPU if it is not there)."""
    torch = _torch()
    t = psi if hasattr(psi, "data_ptr") else torch.from_numpy(np.ascontiguousarray(psi))
    t = t.detach().to(device="cuda", dtype=torch.float32).contiguous()
    if stream is None:
        stream = torch.cuda.current_stream()
    return structure_factor_view(t.data_ptr(), tuple(t.shape), t.shape[-1], h, n_bins, stream)


def porod_fit(centres, mean, counts, k_lo: float, k_hi: float):
    """Least-squares slope and intercept of log S against log k over the bins in
    [k_lo, k_hi] (Porod's law, Sec. 3: slope -(d+1) in the scaling regime); returns
    (slope, intercept, bins used)."""
    lib = _lib.load()
    c = np.ascontiguousarray(centres, dtype=np.float64)
    m = np.ascontiguousarray(mean, dtype=np.float64)
    n = np.ascontiguousarray(counts, dtype=np.int64)
    if not (len(c) == len(m) == len(n)):
        raise ValueError("centres, mean and counts must have the same length")
    dp = ctypes.POINTER(ctypes.c_double)
    slope, icpt, used = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
    check(lib.pf_porod_fit(len(c), c.ctypes.data_as(dp), m.ctypes.data_as(dp),
                           n.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), float(k_lo),
                           float(k_hi), ctypes.byref(slope), ctypes.byref(icpt),
                           ctypes.byref(used)))
    return slope.value, icpt.value, used.value
