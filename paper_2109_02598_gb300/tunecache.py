"""Persistent autotune results.

The environment variable PFGPU_TUNE_CACHE (or an explicit path) names a JSON file. The file
maps a key to the (tile_x, tile_y, k) the autotuner chose. A key is made of the device, the
library version, the grid shape, the field count, the model and the stencil, or a digest of
a batch's instance sizes. A later run takes the stored tuning without probe launches. If
the library rejects a stored entry (another build, another device), the caller tunes again
and overwrites it. Writes go through a temporary file and a rename, so a reader never sees
a half-written file. A missing or unreadable file reads as empty.
"""
from __future__ import annotations

import hashlib
import json
import os
import tempfile

ENV = "PFGPU_TUNE_CACHE"


def cache_path(path: str | None = None) -> str | None:
    """The cache file to use: `path` if given, else $PFGPU_TUNE_CACHE, else None (no cache)."""
    if path:
        return path
    return os.environ.get(ENV) or None


def read(path: str) -> dict:
    try:
        with open(path) as f:
            data = json.load(f)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}


def get(path: str, key: str):
    """The stored (tile_x, tile_y, k) for `key`, or None."""
    v = read(path).get(key)
    if isinstance(v, list) and len(v) == 3 and all(isinstance(x, int) for x in v):
        return tuple(v)
    return None


def put(path: str, key: str, value) -> None:
    """Store (tile_x, tile_y, k) under `key` (read, update, write to a temporary file in the
    same directory, rename over the old file)."""
    data = read(path)
    data[key] = [int(x) for x in value]
    d = os.path.dirname(os.path.abspath(path))
    os.makedirs(d, exist_ok=True)
    fd, tmp = tempfile.mkstemp(prefix=".tune-", dir=d)
    try:
        with os.fdopen(fd, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except BaseException:
        if os.path.exists(tmp):
            os.unlink(tmp)
        raise


def grid_key(device: str, version: int, shape, n_fields: int, model: str, stencil: str) -> str:
    dims = "x".join(str(int(s)) for s in shape)
    return f"grid|{device}|v{version}|{dims}|f{n_fields}|{model}|{stencil}"


def batch_key(device: str, version: int, sizes) -> str:
    """Key of a batch: a digest of its instances' (ny, nx) in order."""
    h = hashlib.sha256(",".join(f"{int(a)}x{int(b)}" for a, b in sizes).encode()).hexdigest()
    return f"batch|{device}|v{version}|{len(sizes)}|{h[:16]}"
