"""Host-side checks of the learned warm start: parameter layout, seeded
initialisation and the shipped checkpoint (no GPU)."""
import json
import os

import numpy as np

from paper_1807_00399_gb300 import learned


def test_layout_matches_network_shape():
    # shared MLP 3 -> 64 -> 128 -> 256, head 512 -> 256 -> 9 (weights + biases)
    n = 3 * 64 + 64 + 64 * 128 + 128 + 128 * 256 + 256 + 512 * 256 + 256 + 256 * 9 + 9
    assert sum(int(np.prod(s)) for _, s in learned.LAYOUT) == n == 175241


def test_init_is_seeded_and_starts_at_identity():
    a, b = learned.init_params(5), learned.init_params(5)
    assert a.dtype == np.float32 and a.shape == (175241,)
    np.testing.assert_array_equal(a, b)
    assert not np.array_equal(a, learned.init_params(6))
    # last bias: 6-D rotation (e1, e2) and zero translation
    np.testing.assert_array_equal(a[-9:], [1, 0, 0, 0, 1, 0, 0, 0, 0])


def test_shipped_checkpoint():
    with open(learned.CHECKPOINT + ".json") as fh:
        meta = json.load(fh)
    params = np.fromfile(learned.CHECKPOINT + ".bin", dtype="<f4")
    assert params.size == meta["n_params"] == 175241
    assert np.all(np.isfinite(params))
    assert meta["extra"]["pairs_seen"] >= 200_000
    hist = meta["extra"]["loss_history"]
    assert hist[-1][1] < 0.5 * hist[0][1]
    # the generator labels survive plain ICP started from them
    assert meta["extra"]["label_check"]["icp_from_label_rot_change_deg_max"] < 0.1
    assert os.path.getsize(learned.CHECKPOINT + ".bin") == 4 * 175241
