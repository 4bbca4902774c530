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


def test_anchor_pick_keeps_the_default_on_near_ties():
    from paper_1908_11807_b300 import autotune as at
    assert at.pick_anchor({1: 0.965, 2: 0.99, 3: 0.964}) == 3
    assert at.pick_anchor({1: 0.960, 2: 0.99, 3: 0.964}) == 3   # 0.4% faster: within the margin
    assert at.pick_anchor({1: 0.900, 2: 0.99, 3: 0.964}) == 1   # 6.6% faster: taken
    assert at.pick_anchor({1: 1.2, 2: 1.0}) == 2                # no default among the candidates
