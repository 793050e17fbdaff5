"""Voxel-grid downsampling: libcil (cil_voxel_downsample) against the oracle.
The voxel of each point is an integer decision from floating point, taken on
both sides in FP32 (correctly rounded division), so the voxel sets and counts
must match exactly; the means agree within 1e-6 of the coordinate magnitude
(compensated FP32 sums vs FP64)."""
import numpy as np
import pytest
import torch

import oracle
import paper_1807_00399_gb300 as cil
from paper_1807_00399_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("v", [0.01, 0.03, 0.2, 5.0])
def test_surface_voxels(v):
    p = synth.surface_pair(6, n=30_000).target
    g, gc = cil.voxel_downsample(torch.from_numpy(p).cuda(), v)
    torch.cuda.synchronize()
    o, oc = oracle.voxel_downsample(p, v)
    assert np.array_equal(gc.cpu().numpy(), oc)
    mag = np.abs(p).max()
    np.testing.assert_allclose(g.cpu().numpy(), o, rtol=0, atol=1e-6 * mag)


def test_depth_frame_1cm():
    p = synth.depth_frame_pair(0)
    g, gc = cil.voxel_downsample(torch.from_numpy(p.target).cuda(), 0.01)
    torch.cuda.synchronize()
    o, oc = oracle.voxel_downsample(p.target, 0.01)
    assert np.array_equal(gc.cpu().numpy(), oc)
    np.testing.assert_allclose(g.cpu().numpy(), o, rtol=0, atol=1e-6 * np.abs(p.target).max())


def test_lattice_and_single_voxel():
    pts = synth.lattice_points((4, 4, 4), spacing=0.5)
    g, gc = cil.voxel_downsample(torch.from_numpy(pts).cuda(), 1.0)
    torch.cuda.synchronize()
    assert np.all(gc.cpu().numpy() == 8) and len(gc) == 8
    g, gc = cil.voxel_downsample(torch.from_numpy(pts).cuda(), 1000.0)
    torch.cuda.synchronize()
    assert gc.cpu().tolist() == [64]
    np.testing.assert_allclose(g.cpu().numpy()[0], [0.75, 0.75, 0.75], atol=1e-7)


def test_wide_and_flat_spans():
    """Keys packed in the bits the occupied span needs: x spans the whole
    21-bit coordinate range, y a small one, z one voxel (no bits)."""
    rng = np.random.default_rng(11)
    xs = np.array([-1048575.5, -4.5, 0.5, 7.5, 1048574.5], np.float32)
    n = 4000
    pts = np.stack([rng.choice(xs, n), rng.uniform(-100.0, 100.0, n),
                    np.full(n, 0.25)], axis=1).astype(np.float32)
    g, gc = cil.voxel_downsample(torch.from_numpy(pts).cuda(), 1.0)
    torch.cuda.synchronize()
    o, oc = oracle.voxel_downsample(pts, 1.0)
    assert np.array_equal(gc.cpu().numpy(), oc)
    assert np.all(np.abs(g.cpu().numpy() - o) <= 1e-6 * np.abs(pts).max(axis=0))
