"""Autotuner bookkeeping that needs no GPU: cache keys and the JSON cache."""
import json


def test_cache_key_buckets_by_log2_n(monkeypatch, tmp_path):
    from paper_1908_11807_b300 import autotune
    assert autotune.cache_key(1_000_000, 10, "cube") == "n2^20/k10/cube"
    assert autotune.cache_key(1_048_576, 10, "cube") == autotune.cache_key(1_000_000, 10, "cube")
    assert autotune.cache_key(10_000_000, 50, "mix") == "n2^23/k50/mix"


def test_cache_roundtrip(monkeypatch, tmp_path):
    from paper_1908_11807_b300 import autotune
    path = tmp_path / "sub" / "tune.json"
    monkeypatch.setenv("ARBORX_TUNE_CACHE", str(path))
    assert autotune._load() == {}
    autotune._store("a", {"block_size": 64})
    autotune._store("b", {"block_size": 128})
    assert json.loads(path.read_text()) == {"a": {"block_size": 64}, "b": {"block_size": 128}}
    assert autotune._load()["a"]["block_size"] == 64
