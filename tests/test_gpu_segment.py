"""Connected-component segmentation (cil_segment) against the oracle: the
partition must lie between the oracle's bounds (every edge the definition
leaves open -- k-th-rank distance ties, similarity values at the threshold --
removed / added), and equal the oracle's labels where those bounds agree."""
import numpy as np
import pytest
import torch

import oracle
import paper_1807_00399_gb300 as cil
from oracle import segment as sg
from paper_1807_00399_gb300 import synth

pytestmark = pytest.mark.gpu
GATE = 1e-2  # eigen-gap gate of the normal parity bar: (l1 - l0) >= GATE l2
TOL_ANGLE = 1e-4  # normal parity bar (rad) where the gap clears the gate


def _normal_eps(P, on, oev, vp):
    """Per-point bound on the angle between the library's normal and the
    oracle's: the normal parity bar where the eigenvector is well conditioned
    and the orientation clear of the viewpoint plane, else unbounded."""
    good = (oev[:, 1] - oev[:, 0]) >= GATE * oev[:, 2]
    v = np.asarray(vp, np.float64) - P.astype(np.float64)
    clear = np.abs((on * v).sum(1)) / np.linalg.norm(v, axis=1) > 1e-3
    return np.where(good & clear & np.isfinite(on).all(1), TOL_ANGLE, 3.0)


def _check(P, N, k, theta, radius=0.0):
    lab, nc = cil.segment(torch.from_numpy(P).cuda(), torch.from_numpy(N).cuda(), k=k, theta=theta,
                          radius=radius)
    lab = lab.cpu().numpy()
    lo, hi = sg.bounds(P, N, k=k, theta=theta, radius=radius)
    assert sg.consistent(lab, lo, hi)
    assert nc == int(np.sum(lab == np.arange(len(P))))
    if np.array_equal(lo, hi):
        np.testing.assert_array_equal(lab, lo)
    return lab, nc


def test_random_normals():
    rng = np.random.default_rng(0)
    P = rng.uniform(-1, 1, (20_000, 3)).astype(np.float32)
    N = rng.normal(size=(20_000, 3))
    N = (N / np.linalg.norm(N, axis=1, keepdims=True)).astype(np.float32)
    _check(P, N, 10, 1.0)
    _check(P, N, 30, 2.8)
    _check(P, N, 16, 2.0, radius=0.08)


def test_depth_frame_smooth_segments():
    p = synth.depth_frame_pair(0)
    on, _, _ = oracle.normals(p.target, 30, p.viewpoint, method="kdtree")
    lab, nc = _check(p.target, on.astype(np.float32), 30, 2.8)
    assert 1 <= nc < len(p.target)


def test_smooth_segment_equals_the_two_step_path():
    p = synth.depth_frame_pair(0)
    x = torch.from_numpy(p.target).cuda()
    nrm, lab, nc = cil.smooth_segment(x, 30, p.viewpoint, theta=2.8)
    gn, _ = cil.estimate_normals(x, 30, p.viewpoint)
    assert torch.equal(nrm, gn)
    lab2, nc2 = cil.segment(x, gn, k=30, theta=2.8)
    assert torch.equal(lab, lab2) and nc == nc2


@pytest.mark.parametrize("k,theta", [(10, 0.2), (30, 2.8)])
def test_smooth_segment_oracle_bounds(k, theta):
    p = synth.depth_frame_pair(1)
    on, _, oev = oracle.normals(p.target, k, p.viewpoint, method="kdtree")
    nrm, lab, nc = cil.smooth_segment(torch.from_numpy(p.target).cuda(), k, p.viewpoint, theta=theta)
    lab = lab.cpu().numpy()
    eps = _normal_eps(p.target, on, oev, p.viewpoint)
    lo, hi = sg.bounds(p.target, on.astype(np.float32), k=k, theta=theta, eps=eps)
    assert sg.consistent(lab, lo, hi)
    assert nc == int(np.sum(lab == np.arange(len(lab))))
    if theta < 1:
        assert nc > 10  # box faces meeting at right angles are cut


def test_empty_and_invalid():
    lab, nc = cil.segment(torch.empty(0, 3, device="cuda"), torch.empty(0, 3, device="cuda"))
    assert lab.numel() == 0 and nc == 0
    x = torch.zeros(10, 3, device="cuda")
    with pytest.raises(Exception):
        cil.segment(x, x, k=0)
    with pytest.raises(Exception):
        cil.segment(x, x, k=8, theta=-1.0)


def test_single_point_and_duplicates():
    lab, nc = cil.segment(torch.zeros(1, 3, device="cuda"), torch.tensor([[0.0, 0, 1]], device="cuda"))
    assert nc == 1 and lab.item() == 0
    P = np.zeros((50, 3), np.float32)
    N = np.tile(np.float32([0, 0, 1]), (50, 1))
    lab, nc = _check(P, N, 8, 0.1)


def test_separated_clusters_and_determinism():
    rng = np.random.default_rng(1)
    P = np.concatenate([rng.normal(0, 0.05, (3000, 3)),
                        rng.normal(0, 0.05, (2000, 3)) + [4.0, 0, 0]]).astype(np.float32)
    N = np.tile(np.float32([0, 0, 1]), (5000, 1))
    a, na = cil.segment(torch.from_numpy(P).cuda(), torch.from_numpy(N).cuda(), k=12, theta=0.3)
    b, nb = cil.segment(torch.from_numpy(P).cuda(), torch.from_numpy(N).cuda(), k=12, theta=0.3)
    assert na == nb == 2 and torch.equal(a, b)
    a = a.cpu().numpy()
    assert (a[:3000] == 0).all() and (a[3000:] == 3000).all()


def test_nan_normals_isolate_points():
    rng = np.random.default_rng(2)
    P = rng.uniform(-1, 1, (2000, 3)).astype(np.float32)
    N = np.tile(np.float32([0, 0, 1]), (2000, 1))
    N[::7] = np.nan
    lab, nc = _check(P, N, 8, 0.5)
    isolated = np.arange(0, 2000, 7)
    assert (lab[isolated] == isolated).all()


def test_apartment_scale_smooth_segmentation():
    """Sec. 4's smooth-segmentation workload at full size (7.8M-point scan
    stand-in, 5 mm voxel grid -> 4.49M points, k = 30, 2.8 rad), voxel
    centroids and normals from the oracle on both sides; the library's
    partition must lie between the oracle's bounds."""
    P = synth.apartment_scene(0)
    V, _ = oracle.voxel_downsample(P, 0.005)
    V = V.astype(np.float32)
    N, _, oev = oracle.normals(V, 30, synth.APARTMENT_VIEWPOINT, method="kdtree")
    N = N.astype(np.float32)
    lab, nc = cil.segment(torch.from_numpy(V).cuda(), torch.from_numpy(N).cuda(), k=30, theta=2.8)
    lab = lab.cpu().numpy()
    idx = np.arange(len(V))
    assert (lab <= idx).all() and (lab[lab] == lab).all()
    assert nc == int(np.sum(lab == idx))
    lo, hi = sg.bounds(V, N, k=30, theta=2.8)
    assert sg.consistent(lab, lo, hi)
    assert len(np.unique(lo)) >= nc >= len(np.unique(hi))
    # one search for normals and graph, against bounds widened by the normals'
    # parity bar
    _, lab, nc = cil.smooth_segment(torch.from_numpy(V).cuda(), 30, synth.APARTMENT_VIEWPOINT,
                                    theta=2.8)
    lab = lab.cpu().numpy()
    eps = _normal_eps(V, N.astype(np.float64), oev, synth.APARTMENT_VIEWPOINT)
    lo, hi = sg.bounds(V, N, k=30, theta=2.8, eps=eps)
    assert sg.consistent(lab, lo, hi)
