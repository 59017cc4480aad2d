"""The autotuner's cache (CPU): winners are stored per key in a JSON file,
read back, and other keys survive an update."""
import json

from paper_1407_8142_gb300 import autotune


def test_store_and_load(tmp_path, monkeypatch):
    path = tmp_path / "sub" / "autotune.json"
    monkeypatch.setenv("WT_AUTOTUNE_CACHE", str(path))
    assert autotune.cache_path() == str(path)
    assert autotune._load() == {}                       # no file yet
    autotune._store("gpu|single|n2^30|L8|b1", {"tile_threads": 512, "ms": {"512": 5.5}})
    autotune._store("gpu|single|n2^28|L20|b4|tree|levels_per_pass", {"levels_per_pass": 4})
    data = json.loads(path.read_text())
    assert data["gpu|single|n2^30|L8|b1"]["tile_threads"] == 512
    assert autotune._load()["gpu|single|n2^28|L20|b4|tree|levels_per_pass"]["levels_per_pass"] == 4
    autotune._store("gpu|single|n2^30|L8|b1", {"tile_threads": 256})
    assert autotune._load()["gpu|single|n2^30|L8|b1"]["tile_threads"] == 256
    assert "gpu|single|n2^28|L20|b4|tree|levels_per_pass" in autotune._load()


def test_corrupt_cache_reads_as_empty(tmp_path, monkeypatch):
    path = tmp_path / "autotune.json"
    path.write_text("{not json")
    monkeypatch.setenv("WT_AUTOTUNE_CACHE", str(path))
    assert autotune._load() == {}
