"""The batched autotuner's cache (the one state the library keeps across
processes): a miss runs the tuner and stores its result, a hit returns it
without tuning, other keys are kept, and the file is replaced whole."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_cache_miss_then_hit(tmp_path):
    import pytest
    pytest.importorskip("torch")
    from paper_1211_4896_gb300.api import cached_tuning
    calls = []

    def tune():
        calls.append(1)
        return {"tile_w": 16, "tile_h": 2, "ctas_per_sm": 3}

    path = str(tmp_path / "tune.json")
    assert cached_tuning("k1", tune, path) == {"tile_w": 16, "tile_h": 2, "ctas_per_sm": 3}
    assert cached_tuning("k1", tune, path) == {"tile_w": 16, "tile_h": 2, "ctas_per_sm": 3}
    assert len(calls) == 1
    cached_tuning("k2", lambda: {"tile_w": 8, "tile_h": 4, "ctas_per_sm": 0}, path)
    table = json.load(open(path))
    assert set(table) == {"k1", "k2"} and table["k2"]["tile_w"] == 8
    assert not [f for f in os.listdir(tmp_path) if ".tmp" in f]


def test_no_cache_without_a_path(tmp_path, monkeypatch):
    import pytest
    pytest.importorskip("torch")
    from paper_1211_4896_gb300.api import cached_tuning
    monkeypatch.delenv("VR_AUTOTUNE_CACHE", raising=False)
    n = []
    for _ in range(2):
        cached_tuning("k", lambda: n.append(1) or {"tile_w": 8, "tile_h": 4, "ctas_per_sm": 0})
    assert len(n) == 2
    monkeypatch.setenv("VR_AUTOTUNE_CACHE", str(tmp_path / "env.json"))
    for _ in range(2):
        cached_tuning("k", lambda: n.append(1) or {"tile_w": 8, "tile_h": 4, "ctas_per_sm": 0})
    assert len(n) == 3 and os.path.exists(tmp_path / "env.json")
