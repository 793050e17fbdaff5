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


def test_descent_brackets_the_best_scale_and_picks_each_axis():
    # cost minimal at scale 6 (beyond the listed range), block 64, heap layout
    def cost(sc, bl, tk):
        return (np.log(sc / 6.0)) ** 2 + (0.0 if bl == 64 else 0.1) + (0.0 if tk == 2 else 0.05)
    (sc, bl, tk), table, interior = autotune.coordinate_descent(cost)
    assert interior and bl == 64 and tk == 2
    assert abs(np.log(sc / 6.0)) <= np.log(1.5) / 2 + 1e-12  # nearest tried point to 6
    assert max(r["cell_scale"] for r in table) > 4.0        # the range was extended
    assert len({(r["cell_scale"], r["block"], r["topk"]) for r in table}) == len(table)
    # minimum below the range: extended downwards
    (sc, _, _), table, interior = autotune.coordinate_descent(
        lambda s, b, t: abs(np.log(s / 0.3)))
    assert interior and min(r["cell_scale"] for r in table) < 0.5 and abs(sc - 1 / 3) < 1e-9
    # a flat cost keeps the defaults (block 128, layout by k) and the first scale tried
    (sc, bl, tk), _, interior = autotune.coordinate_descent(lambda s, b, t: 1.0)
    assert (bl, tk) == (128, 0) and not interior
