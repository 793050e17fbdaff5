"""Pins for the oracle's voxel-grid downsampling (Sec. 3 GridAccumulator):
hand-computed lattice groupings, conservation of points, one voxel holding
everything, membership of every mean in its voxel, permutation invariance."""
import numpy as np

import oracle
from paper_1807_00399_gb300 import synth


def test_lattice_groups_of_eight():
    pts = synth.lattice_points((4, 4, 4), spacing=0.5)  # coordinates 0, .5, 1, 1.5
    out, cnt = oracle.voxel_downsample(pts, 1.0)
    # voxel size 1 groups each 2x2x2 block; its mean sits at the block centre
    assert len(out) == 8 and np.all(cnt == 8)
    expect = np.array([[a, b, c] for a in (0.25, 1.25) for b in (0.25, 1.25) for c in (0.25, 1.25)])
    np.testing.assert_array_equal(out, expect)


def test_conservation_membership_and_order():
    p = synth.surface_pair(3, n=20_000).target
    v = np.float32(0.03)
    out, cnt = oracle.voxel_downsample(p, v)
    assert cnt.sum() == len(p)
    ijk = np.floor(out / np.float64(v))
    # the mean of points of one voxel lies in that voxel
    lo = ijk * np.float64(v)
    assert np.all(out >= lo - 1e-12) and np.all(out <= lo + np.float64(v) + 1e-12)
    keys = [tuple(r) for r in ijk.astype(np.int64)]
    assert keys == sorted(keys) and len(set(keys)) == len(keys)


def test_single_voxel_gives_centroid():
    p = synth.surface_pair(4, n=1000).target
    q = (p + np.float32(10.0)).astype(np.float32)
    out, cnt = oracle.voxel_downsample(q, 100.0)
    assert len(out) == 1 and cnt[0] == 1000
    np.testing.assert_allclose(out[0], q.astype(np.float64).mean(0), rtol=1e-12)


def test_permutation_invariance():
    p = synth.surface_pair(5, n=5000).target
    perm = np.random.default_rng(0).permutation(len(p))
    a, ca = oracle.voxel_downsample(p, 0.05)
    b, cb = oracle.voxel_downsample(p[perm], 0.05)
    assert np.array_equal(ca, cb)
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-15)
