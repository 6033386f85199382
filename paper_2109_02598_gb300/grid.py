"""Python face of a pfgpu grid (argument marshalling over the C ABI of include/pfgpu.h).

A ``Grid`` is the paper's Grid/System/Model triple (Sec. 2.2.1, 2.2.5): a periodic 2D or
3D grid of one or two float32 fields, an equation of motion with its coefficients
(Sec. 3) and the forward-Euler solver (Sec. 2.4.1).  Shapes follow numpy order,
``(ny, nx)`` or ``(nz, ny, nx)``, x fastest (Sec. 2.2.1).  PyTorch supplies the CUDA
stream and device tensors; all arithmetic runs in libpfgpu's kernels.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from . import checkpoint, tunecache
from ._lib import MODEL_FIELDS, MODEL_IDS, PfError, check


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("pfgpu needs a CUDA device (there is no CPU fallback)")
    return torch


def _stream_handle(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def _device_tag() -> str:
    """Name and compute capability of the current CUDA device (the tune cache's key)."""
    torch = _torch()
    d = torch.cuda.current_device()
    major, minor = torch.cuda.get_device_capability(d)
    return f"{torch.cuda.get_device_name(d)}|sm{major}{minor}"


def rd_coeffs(D, E, K):
    """The coefficient list of PF_MODEL_RD (N coupled species,
    du_i/dt = D_i lap u_i + sum_m K[i][m] prod_j u_j^E[m][j]): D (N), the exponents E (M rows
    of N integers in 0..3) and the rates K (N rows of M), flattened in that order after the
    monomial count M."""
    D = [float(x) for x in D]
    E = [[int(e) for e in row] for row in E]
    K = [[float(k) for k in row] for row in K]
    if any(len(row) != len(D) for row in E) or len(K) != len(D) or any(len(r) != len(E) for r in K):
        raise ValueError("E must be M x N and K N x M")
    return tuple(D) + (float(len(E)),) + tuple(float(e) for row in E for e in row) + \
        tuple(k for row in K for k in row)


class Grid:
    """A periodic grid with ``n_fields`` float32 fields living on the GPU."""

    def __init__(self, shape, n_fields: int = 1, h: float = 1.0, stream=None):
        torch = _torch()
        self._lib = _lib.load()
        self.shape = tuple(int(s) for s in shape)
        if len(self.shape) not in (2, 3):
            raise ValueError("shape must be (ny, nx) or (nz, ny, nx)")
        self.dim = len(self.shape)
        self.n_fields = int(n_fields)
        self.h = float(h)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        nx, ny = self.shape[-1], self.shape[-2]
        nz = self.shape[0] if self.dim == 3 else 1
        n = (ctypes.c_int64 * 3)(nx, ny, nz)
        handle = ctypes.c_void_p()
        check(self._lib.pf_create_grid(self.dim, n, self.n_fields, self.h,
                                       ctypes.c_void_p(_stream_handle(self.stream)),
                                       ctypes.byref(handle)))
        self._h = handle
        self.model = None
        self.coeffs = None
        self.dt = None
        self.stencil = "std"
        self.steps_done = 0  # steps taken through this object (or restored by load)

    # ---------------------------------------------------------------- lifecycle
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.pf_destroy(self._h)
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
    def handle(self):
        return self._h

    @property
    def sites(self) -> int:
        return int(np.prod(self.shape))

    # ---------------------------------------------------------------- model
    def set_model(self, model: str, coeffs, dt: float, force: bool = False):
        """model in {"ac", "ch", "gs", "c", "rd"}; coeffs AC (c1, c2), CH (c1, c2, M),
        GS (Du, Dv, F, k), Model C (c1, c2, c3, c4, c5), RD (N coupled species, any field
        count up to 4) the flat list of ``rd_coeffs(D, E, K)``."""
        c = (ctypes.c_double * len(coeffs))(*[float(x) for x in coeffs])
        check(self._lib.pf_set_model(self._h, MODEL_IDS[model], c, len(coeffs), float(dt),
                                     1 if force else 0))
        self.model = model
        self.coeffs = tuple(float(x) for x in coeffs)
        self.dt = float(dt)
        return self

    def set_stencil(self, stencil: str = "std"):
        """Laplacian stencil: "std" (5/7-point), "iso" (isotropic 9/19-point), "4th"
        (fourth-order 9-point, 2D) or "iso27" (isotropic 27-point, 3D)."""
        check(self._lib.pf_set_stencil(self._h, _lib.STENCIL_IDS[stencil]))
        self.stencil = stencil
        return self

    # ---------------------------------------------------------------- fields
    def write_field(self, field: int, data):
        """Copy in a dense float32 array of ``shape``: numpy (host) or torch (host/CUDA)."""
        if hasattr(data, "data_ptr"):
            t = data.detach()
            if tuple(t.shape) != self.shape:
                raise ValueError(f"field shape {tuple(t.shape)} != grid shape {self.shape}")
            torch = _torch()
            t = t.to(torch.float32).contiguous()
            check(self._lib.pf_write_field(self._h, field, ctypes.c_void_p(t.data_ptr()),
                                           1 if t.is_cuda else 0))
            if t.is_cuda:
                self._keep = t  # the copy is enqueued; keep the source alive until synced
                self.synchronize()
                self._keep = None
            return self
        a = np.ascontiguousarray(data, dtype=np.float32)
        if a.shape != self.shape:
            raise ValueError(f"field shape {a.shape} != grid shape {self.shape}")
        check(self._lib.pf_write_field(self._h, field, a.ctypes.data_as(ctypes.c_void_p), 0))
        return self

    def copy_planes(self, field: int, first: int, count: int, buf, to_buf: bool):
        """Copy planes [first, first + count) along the slowest axis (z in 3D, y in 2D) of a
        field to (``to_buf``) or from a dense float32 buffer: a numpy array, or a torch
        tensor on the host or the grid's device, of shape (count, ...) of the other axes."""
        if hasattr(buf, "data_ptr"):
            if not buf.is_contiguous() or buf.dtype != _torch().float32:
                raise ValueError("buf must be a contiguous float32 tensor")
            ptr, on_dev = buf.data_ptr(), 1 if buf.is_cuda else 0
        else:
            if not (buf.flags.c_contiguous and buf.dtype == np.float32):
                raise ValueError("buf must be a C-contiguous float32 array")
            ptr, on_dev = buf.ctypes.data, 0
        check(self._lib.pf_copy_planes(self._h, field, int(first), int(count),
                                       ctypes.c_void_p(ptr), 1 if to_buf else 0, on_dev))
        return buf

    def mass_planes(self, field: int, first: int, count: int) -> float:
        """h^d sum of a field over planes [first, first + count) along the slowest axis, by
        the library's reduction (pf_reduce_noalloc on that part of the field)."""
        torch = _torch()
        ptr, pitch, plane = ctypes.c_void_p(), ctypes.c_int64(), ctypes.c_int64()
        check(self._lib.pf_field_view(self._h, field, ctypes.byref(ptr), ctypes.byref(pitch),
                                      ctypes.byref(plane)))
        nslow = self.shape[0]
        if not (0 <= first and 0 < count and first + count <= nslow):
            raise ValueError("plane range outside the grid")
        step = plane.value if self.dim == 3 else pitch.value
        n = (ctypes.c_int64 * 3)(self.shape[-1], count if self.dim == 2 else self.shape[1],
                                 count if self.dim == 3 else 1)
        out = torch.empty(1, dtype=torch.float64, device="cuda")
        check(self._lib.pf_reduce_noalloc(_lib.PF_REDUCE_MASS, self.dim, n, pitch.value,
                                          ctypes.c_void_p(ptr.value + 4 * first * step), self.h,
                                          0.0, 0.0, ctypes.c_void_p(out.data_ptr()),
                                          ctypes.c_void_p(_stream_handle(self.stream))))
        self.synchronize()
        return float(out.item())

    def write_fields(self, fields):
        for i, f in enumerate(fields):
            self.write_field(i, f)
        return self

    def read_field(self, field: int, device: bool = False, out=None):
        """Field ``field`` as a numpy array (default) or a CUDA torch tensor."""
        if device or (out is not None and hasattr(out, "data_ptr")):
            torch = _torch()
            if out is None:
                out = torch.empty(self.shape, dtype=torch.float32, device="cuda")
            check(self._lib.pf_read_field(self._h, field, ctypes.c_void_p(out.data_ptr()),
                                          1 if out.is_cuda else 0))
            return out
        a = np.empty(self.shape, dtype=np.float32) if out is None else out
        check(self._lib.pf_read_field(self._h, field, a.ctypes.data_as(ctypes.c_void_p), 0))
        return a

    def read_fields(self, device: bool = False):
        return tuple(self.read_field(i, device=device) for i in range(self.n_fields))

    def write_field_async(self, field: int, pinned):
        """Enqueue the copy of a pinned host torch tensor of ``shape`` into ``field`` and
        return; ``pinned`` must stay untouched until ``synchronize``."""
        torch = _torch()
        if (tuple(pinned.shape) != self.shape or not pinned.is_contiguous() or pinned.is_cuda
                or pinned.dtype != torch.float32):
            raise ValueError("needs a contiguous float32 host tensor of the grid's shape")
        check(self._lib.pf_write_field_host_async(self._h, field,
                                                  ctypes.c_void_p(pinned.data_ptr())))
        return self

    def read_field_async(self, field: int, pinned):
        """Enqueue the copy of ``field`` into a pinned host torch tensor and return; its
        contents are valid after ``synchronize``."""
        torch = _torch()
        if (tuple(pinned.shape) != self.shape or not pinned.is_contiguous() or pinned.is_cuda
                or pinned.dtype != torch.float32):
            raise ValueError("needs a contiguous float32 host tensor of the grid's shape")
        check(self._lib.pf_read_field_host_async(self._h, field,
                                                 ctypes.c_void_p(pinned.data_ptr())))
        return pinned

    # ---------------------------------------------------------------- stepping
    def step(self, n_steps: int = 1):
        check(self._lib.pf_step(self._h, int(n_steps)))
        self.steps_done += int(n_steps)
        return self

    # ---------------------------------------------------------------- checkpoints
    def save(self, path: str, extra: dict | None = None):
        """Write a checkpoint: the fields and what is needed to continue the run (model,
        coefficients, dt, h, stencil, tuning, steps taken). `extra`: JSON-serialisable
        values stored alongside."""
        meta = {"shape": list(self.shape), "h": self.h, "model": self.model,
                "coeffs": list(self.coeffs) if self.coeffs is not None else None,
                "dt": self.dt, "stencil": self.stencil, "tuning": list(self.tuning),
                "steps": self.steps_done, "extra": extra or {}}
        checkpoint.save_state(path, meta, self.read_fields())
        return self

    @classmethod
    def load(cls, path: str, stream=None):
        """A grid restored from a checkpoint written by save(): same fields, model,
        coefficients, dt, h, stencil and step count, and the saved tuning where this build
        and device accept it. Stepping it on gives the bits of the run that did not stop."""
        meta, fields = checkpoint.load_state(path)
        g = cls(meta["shape"], len(fields), meta["h"], stream=stream)
        if meta["model"] is not None:
            g.set_model(meta["model"], meta["coeffs"], meta["dt"], force=True)
        if meta["stencil"] != "std":
            g.set_stencil(meta["stencil"])
        try:
            g.set_tuning(*meta["tuning"])
        except PfError:
            pass  # not available here: the default tuning gives the same bits
        g.write_fields(fields)
        g.steps_done = int(meta["steps"])
        g.checkpoint_extra = meta.get("extra", {})
        return g

    def synchronize(self):
        check(self._lib.pf_synchronize(self._h))

    # ---------------------------------------------------------------- reductions
    def mass(self, field: int = 0) -> float:
        out = ctypes.c_double()
        check(self._lib.pf_reduce(self._h, _lib.PF_REDUCE_MASS, field, ctypes.byref(out)))
        return out.value

    def energy(self) -> float:
        out = ctypes.c_double()
        check(self._lib.pf_reduce(self._h, _lib.PF_REDUCE_ENERGY, 0, ctypes.byref(out)))
        return out.value

    # ---------------------------------------------------------------- tuning
    def set_tuning(self, tile_x: int = 0, tile_y: int = 0, k: int = 0):
        """Tile and temporal-blocking depth (0 = default). (nx, ny / CS) selects the on-chip
        cluster kernel, (nx, PF_TILE_BANDS) the band kernel (one band of rows per SM)."""
        check(self._lib.pf_set_tuning(self._h, tile_x, tile_y, k))
        return self

    @property
    def tuning(self):
        a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        check(self._lib.pf_get_tuning(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return a.value, b.value, c.value

    def autotune(self, probe_launches: int = 5, cache: str | None = None):
        """Time every supported (tile, k) and keep the fastest (pf_autotune). With a cache
        file (`cache` or $PFGPU_TUNE_CACHE) a stored choice for this device, library version,
        shape, field count, model and stencil is applied without probing, and a new one is
        stored."""
        path = tunecache.cache_path(cache)
        key = None
        if path:
            key = tunecache.grid_key(_device_tag(), self._lib.pf_version(), self.shape,
                                     self.n_fields, str(self.model),
                                     getattr(self, "stencil", "std"))
            hit = tunecache.get(path, key)
            if hit is not None:
                try:
                    return self.set_tuning(*hit).tuning
                except PfError:
                    pass  # not valid for this build or device: tune again
        a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        check(self._lib.pf_autotune(self._h, probe_launches, ctypes.byref(a), ctypes.byref(b),
                                    ctypes.byref(c)))
        if path:
            tunecache.put(path, key, (a.value, b.value, c.value))
        return a.value, b.value, c.value

    def run_series(self, n_steps: int, every: int, energy: bool = False):
        """Advance n_steps in chunks of `every` and record the mass of every field (and the
        discrete free energy, for Models A, B and C) after each chunk: a list of dicts
        {"step", "mass": [...], "energy"}; the first entry is the state before stepping."""
        if every < 1:
            raise ValueError("every must be >= 1")

        def sample(step):
            rec = {"step": step, "mass": [self.mass(f) for f in range(self.n_fields)]}
            if energy:
                rec["energy"] = self.energy()
            return rec

        series = [sample(0)]
        done = 0
        while done < n_steps:
            k = min(every, n_steps - done)
            self.step(k)
            done += k
            series.append(sample(done))
        return series

    # ---------------------------------------------------------------- analysis
    def structure_factor(self, field: int = 0, n_bins: int = 32):
        """Radially averaged S(|k|) of [field > 0] (Sec. 3), read in place on the GPU."""
        from .spectral import structure_factor_view
        ptr, pitch, plane = ctypes.c_void_p(), ctypes.c_int64(), ctypes.c_int64()
        check(self._lib.pf_field_view(self._h, field, ctypes.byref(ptr), ctypes.byref(pitch),
                                      ctypes.byref(plane)))
        return structure_factor_view(ptr.value, self.shape, pitch.value, self.h, n_bins,
                                     self.stream)
