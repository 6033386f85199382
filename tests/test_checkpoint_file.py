"""Checkpoint file format (host logic, no GPU)."""
import json

import numpy as np
import pytest

from paper_2109_02598_gb300 import checkpoint


def test_roundtrip(tmp_path):
    rng = np.random.default_rng(3)
    f = [rng.standard_normal((5, 7)).astype(np.float32) for _ in range(2)]
    meta = {"shape": [5, 7], "h": 0.5, "model": "gs", "coeffs": [0.2, 0.1, 0.04, 0.06],
            "dt": 0.5, "stencil": "std", "tuning": [64, 16, 4], "steps": 123, "extra": {"a": 1}}
    path = str(tmp_path / "d" / "c.npz")
    checkpoint.save_state(path, meta, f)
    m, g = checkpoint.load_state(path)
    assert m["steps"] == 123 and m["coeffs"] == meta["coeffs"] and m["n_fields"] == 2
    assert m["format"] == checkpoint.FORMAT and m["extra"] == {"a": 1}
    assert all(np.array_equal(a, b) and b.dtype == np.float32 for a, b in zip(f, g))
    assert sorted(p.name for p in (tmp_path / "d").iterdir()) == ["c.npz"]  # no temporary


def test_rejects_other_formats_and_shapes(tmp_path):
    path = tmp_path / "c.npz"
    np.savez(path, meta=np.array(json.dumps({"format": 99, "n_fields": 0, "shape": [1]})))
    with pytest.raises(ValueError, match="format"):
        checkpoint.load_state(str(path))
    np.savez(path, meta=np.array(json.dumps({"format": checkpoint.FORMAT, "n_fields": 1,
                                             "shape": [4, 4]})),
             f0=np.zeros((4, 5), np.float32))
    with pytest.raises(ValueError, match="shape"):
        checkpoint.load_state(str(path))
