"""Checkpoint files of a grid's state (the paper's data persistence for reading and writing
phase-field data and resuming a run, Sec. 2.3.5): an .npz holding the fields as float32
arrays and a JSON record of everything needed to continue the run. The record has the shape,
the field count, h, the model, coefficients, Δt, the stencil, the tuning and the steps taken.
Files are written to a temporary name and renamed, so a reader never sees a partial
checkpoint. A resumed run gives the same bits as one that did not stop, because the state is
the float32 fields and nothing else."""
from __future__ import annotations

import json
import os
import tempfile

import numpy as np

FORMAT = 1


def save_state(path: str, meta: dict, fields) -> None:
    """Write `fields` (float32 arrays) and `meta` (JSON-serialisable) to `path`."""
    rec = dict(meta)
    rec["format"] = FORMAT
    rec["n_fields"] = len(fields)
    arrays = {f"f{i}": np.ascontiguousarray(f, dtype=np.float32) for i, f in enumerate(fields)}
    d = os.path.dirname(os.path.abspath(path))
    os.makedirs(d, exist_ok=True)
    fd, tmp = tempfile.mkstemp(prefix=".ckpt-", suffix=".npz", dir=d)
    try:
        with os.fdopen(fd, "wb") as f:
            np.savez(f, meta=np.array(json.dumps(rec)), **arrays)
        os.replace(tmp, path)
    except BaseException:
        if os.path.exists(tmp):
            os.unlink(tmp)
        raise


def load_state(path: str):
    """(meta, [fields]) of a checkpoint written by save_state."""
    with np.load(path, allow_pickle=False) as z:
        meta = json.loads(str(z["meta"]))
        if meta.get("format") != FORMAT:
            raise ValueError(f"{path}: checkpoint format {meta.get('format')}, expected {FORMAT}")
        fields = [z[f"f{i}"].copy() for i in range(int(meta["n_fields"]))]
    for f in fields:
        if f.dtype != np.float32 or tuple(f.shape) != tuple(meta["shape"]):
            raise ValueError(f"{path}: field of dtype {f.dtype} and shape {f.shape} does not "
                             f"match {meta['shape']}")
    return meta, fields
