"""Autotuner on the GPU: every configuration it tries registers the batch to
bitwise the same transforms (the searches are exact whatever the cell size
or block shape), the winner is one of them, and it is cached."""
import numpy as np
import pytest
import torch

import paper_1807_00399_gb300 as cil
from paper_1807_00399_gb300 import autotune, synth

pytestmark = pytest.mark.gpu


def test_tuned_configurations_agree_and_cache(tmp_path, monkeypatch):
    monkeypatch.setenv("CIL_TUNE_CACHE", str(tmp_path / "tune.json"))
    sizes = np.array([2000, 3500, 5000, 8000, 2500, 6000], np.int64)
    src, dst, _ = synth.surface_batch_torch(77, sizes)
    res = autotune.tune_batch(src, dst, sizes, sizes, k=10, iters=8, reps=1)
    assert not res["cached"] and len(res["table"]) >= len(autotune.SCALES) + 2
    assert {r["topk"] for r in res["table"]} >= {0, 1, 2}
    assert {r["block"] for r in res["table"]} == set(autotune.BLOCKS)
    again = autotune.tune_batch(src, dst, sizes, sizes, k=10, iters=8, reps=1)
    assert again["cached"] and again["cell_scale"] == res["cell_scale"]
    assert again["topk"] == res["topk"] and again["block"] == res["block"]
    Ts = []
    for r in res["table"]:
        h = cil.Batch(sizes, sizes, k=10, iters=8, max_corr_dist=0.1, viewpoint=(0.0, 0.0, 10.0),
                      cell_scale=r["cell_scale"], block=r["block"], topk=r["topk"])
        T, _ = h.run(src, dst)
        torch.cuda.synchronize()
        Ts.append(T.cpu().numpy())
        h.close()
    for T in Ts[1:]:
        assert np.array_equal(T, Ts[0])
