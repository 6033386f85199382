"""Batched 2D Gray-Scott (argument marshalling over include/pfgpu.h's pf_batch_* calls).

Many independent periodic grids of uneven sizes and coefficients advance together in one
CUDA-graph launch per ``run`` (the GPU form of the paper's driver that runs a list of models,
Sec. 2.4).  Each instance is bitwise identical to the same grid stepped alone with ``Grid``.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from . import tunecache
from ._lib import GS2DSpec, PfError, check
from .grid import _device_tag, _stream_handle, _torch


class Batch:
    """``specs``: iterable of dicts with keys nx, ny (or n for square), Du, Dv, F, k."""

    def __init__(self, specs, dt: float, h: float = 1.0, stream=None):
        torch = _torch()
        self._lib = _lib.load()
        specs = list(specs)
        arr = (GS2DSpec * len(specs))()
        self.shapes = []
        for i, s in enumerate(specs):
            nx = int(s.get("nx", s.get("n")))
            ny = int(s.get("ny", s.get("n")))
            arr[i] = GS2DSpec(nx, ny, float(s["Du"]), float(s["Dv"]), float(s["F"]), float(s["k"]))
            self.shapes.append((ny, nx))
        self.n = len(specs)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        handle = ctypes.c_void_p()
        check(self._lib.pf_batch_create(self.n, arr, float(dt), float(h),
                                        ctypes.c_void_p(_stream_handle(self.stream)),
                                        ctypes.byref(handle)))
        self._h = handle

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.pf_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def sites(self) -> int:
        s = ctypes.c_int64()
        check(self._lib.pf_batch_info(self._h, ctypes.byref(s), None))
        return s.value

    @property
    def bytes_per_copy(self) -> int:
        b = ctypes.c_int64()
        check(self._lib.pf_batch_info(self._h, None, ctypes.byref(b)))
        return b.value

    def write(self, inst: int, field: int, data):
        if hasattr(data, "data_ptr"):
            t = data.detach().contiguous()
            check(self._lib.pf_batch_write_field(self._h, inst, field,
                                                 ctypes.c_void_p(t.data_ptr()),
                                                 1 if t.is_cuda else 0))
            if t.is_cuda:
                self.synchronize()
            return self
        a = np.ascontiguousarray(data, dtype=np.float32)
        if a.shape != self.shapes[inst]:
            raise ValueError(f"instance {inst}: shape {a.shape} != {self.shapes[inst]}")
        check(self._lib.pf_batch_write_field(self._h, inst, field,
                                             a.ctypes.data_as(ctypes.c_void_p), 0))
        return self

    def read(self, inst: int, field: int, out=None):
        a = np.empty(self.shapes[inst], dtype=np.float32) if out is None else out
        check(self._lib.pf_batch_read_field(self._h, inst, field,
                                            a.ctypes.data_as(ctypes.c_void_p), 0))
        return a

    def run(self, n_steps: int):
        check(self._lib.pf_batch_run(self._h, int(n_steps)))
        return self

    def synchronize(self):
        check(self._lib.pf_batch_synchronize(self._h))

    def set_tuning(self, tile_x: int = 0, tile_y: int = 0, k: int = 0):
        check(self._lib.pf_batch_set_tuning(self._h, tile_x, tile_y, k))
        return self

    @property
    def tuning(self):
        a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        check(self._lib.pf_batch_get_tuning(self._h, ctypes.byref(a), ctypes.byref(b),
                                            ctypes.byref(c)))
        return a.value, b.value, c.value

    def autotune(self, probe_launches: int = 3, cache: str | None = None):
        """Time every (tile, k) on the whole batch and keep the fastest. With a cache file
        (`cache` or $PFGPU_TUNE_CACHE) a stored choice for this device, library version and
        list of instance sizes is applied without probing, and a new one is stored."""
        path = tunecache.cache_path(cache)
        key = None
        if path:
            key = tunecache.batch_key(_device_tag(), self._lib.pf_version(), self.shapes)
            hit = tunecache.get(path, key)
            if hit is not None:
                try:
                    return self.set_tuning(*hit).tuning
                except PfError:
                    pass  # not valid for this build or device: tune again
        a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        check(self._lib.pf_batch_autotune(self._h, probe_launches, ctypes.byref(a),
                                          ctypes.byref(b), ctypes.byref(c)))
        if path:
            tunecache.put(path, key, (a.value, b.value, c.value))
        return a.value, b.value, c.value


def shard_instances(sizes, rank: int, world: int):
    """Indices of the batch instances rank ``rank`` of ``world`` runs.

    The instances are independent, so ranks share no data: a deterministic greedy split
    (largest grid first, to the rank with the fewest sites so far; ties to the lowest rank)
    balances lattice sites across ranks.  ``sizes`` are sites per instance.
    """
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    order = sorted(range(len(sizes)), key=lambda i: (-int(sizes[i]), i))
    load = [0] * world
    mine = []
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        load[r] += int(sizes[i])
        if r == rank:
            mine.append(i)
    return sorted(mine)
