"""Autotuner bookkeeping on the host: size buckets and the JSON cache."""
import json

import numpy as np

from paper_1807_00399_gb300 import autotune


def test_bucket_rounds_shape():
    n = np.array([1000, 3000, 5000])
    assert autotune.bucket(n, n, 10, 30) == "B4-n4096-k10-i30"
    assert autotune.bucket(np.array([2000] * 256), np.array([2000] * 256), 16, 5) == \
        "B256-n2048-k16-i5"


def test_cache_roundtrip(tmp_path, monkeypatch):
    path = tmp_path / "t.json"
    monkeypatch.setenv("CIL_TUNE_CACHE", str(path))
    assert autotune.cache_path() == str(path)
    assert autotune._load(str(path)) == {}
    autotune._store(str(path), {"k": {"cell_scale": 1.0, "block": 128, "ms": 1.5}})
    assert json.loads(path.read_text())["k"]["block"] == 128
    path.write_text("not json")
    assert autotune._load(str(path)) == {}
