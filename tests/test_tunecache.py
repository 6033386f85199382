"""The autotune cache file (host logic, no GPU)."""
import json
import os

from paper_2109_02598_gb300 import tunecache


def test_roundtrip_and_keys(tmp_path):
    path = str(tmp_path / "sub" / "tune.json")
    k1 = tunecache.grid_key("GB300|sm103", 3, (2048, 2048), 1, "ch", "std")
    k2 = tunecache.grid_key("GB300|sm103", 3, (2048, 2048), 1, "ac", "std")
    k3 = tunecache.grid_key("GB300|sm103", 4, (2048, 2048), 1, "ch", "std")
    assert len({k1, k2, k3}) == 3
    assert tunecache.get(path, k1) is None  # no file yet
    tunecache.put(path, k1, (2048, -1, 1))
    tunecache.put(path, k2, (128, 32, 4))
    assert tunecache.get(path, k1) == (2048, -1, 1)
    assert tunecache.get(path, k2) == (128, 32, 4)
    tunecache.put(path, k1, (128, 16, 2))  # overwrite
    assert tunecache.get(path, k1) == (128, 16, 2)
    assert sorted(os.listdir(tmp_path / "sub")) == ["tune.json"]  # no temporary left
    assert json.load(open(path))[k2] == [128, 32, 4]


def test_bad_files_and_entries_read_as_missing(tmp_path):
    path = tmp_path / "tune.json"
    path.write_text("{ not json")
    assert tunecache.read(str(path)) == {}
    assert tunecache.get(str(path), "x") is None
    path.write_text(json.dumps({"x": [1, 2], "y": "z", "w": [1, 2, 3.5]}))
    assert tunecache.get(str(path), "x") is None
    assert tunecache.get(str(path), "y") is None
    assert tunecache.get(str(path), "w") is None
    tunecache.put(str(path), "x", (64, 16, 4))  # a corrupt file is replaced, not an error
    assert tunecache.get(str(path), "x") == (64, 16, 4)


def test_cache_path_and_batch_key(tmp_path, monkeypatch):
    monkeypatch.delenv(tunecache.ENV, raising=False)
    assert tunecache.cache_path() is None
    monkeypatch.setenv(tunecache.ENV, str(tmp_path / "env.json"))
    assert tunecache.cache_path() == str(tmp_path / "env.json")
    assert tunecache.cache_path(str(tmp_path / "arg.json")) == str(tmp_path / "arg.json")
    a = tunecache.batch_key("d", 1, [(64, 64), (97, 130)])
    b = tunecache.batch_key("d", 1, [(97, 130), (64, 64)])
    c = tunecache.batch_key("d", 1, [(64, 64), (97, 131)])
    assert len({a, b, c}) == 3
