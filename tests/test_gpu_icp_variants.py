"""ICP variants (cil_icp) against the FP64 variant oracle: point-to-point
(closed form), weighted point/plane combination, projective association.
Bar as for point-to-plane: rotation within 1e-5 rad, translation within 1e-6
of the target's bounding-box diagonal; inlier counts within a few (FP32
versus FP64 decisions at the rejection boundary)."""
import numpy as np
import pytest
import torch

import oracle
import paper_1807_00399_gb300 as cil
from oracle import icp_variants as iv
from paper_1807_00399_gb300 import synth
from parity import extent, rot_angle

pytestmark = pytest.mark.gpu


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _same(Tg, To, dst, rot_tol=1e-5, trans_rel=1e-6):
    ang = rot_angle(Tg[:3, :3], To[:3, :3])
    dt = np.abs(Tg[:3, 3] - To[:3, 3]).max()
    assert ang <= rot_tol, f"rotation differs by {ang:.3g} rad"
    assert dt <= trans_rel * extent(dst), f"translation differs by {dt:.3g}"


@pytest.fixture(scope="module")
def surface():
    p = synth.surface_pair(21, n=10_000)
    on, _, _ = oracle.normals(p.target, 10, p.viewpoint)
    return p, on.astype(np.float32)


@pytest.mark.parametrize("iters", [1, 20])
def test_point_to_point(surface, iters):
    p, _ = surface
    Tg, rg = cil.icp(_cuda(p.source), _cuda(p.target), None, iters=iters, max_corr_dist=0.1,
                     metric="point_to_point")
    o = iv.icp(p.source, p.target, iters=iters, max_corr_dist=0.1, metric="point_to_point")
    _same(Tg, o["T"], p.target)
    assert abs(rg["n_inliers"] - o["n_inliers"]) <= 2 and rg["status"] == 0
    assert rg["rmse"] == pytest.approx(o["rmse"], rel=1e-4)


def test_point_to_point_exact_motion():
    rng = np.random.default_rng(2)
    tgt = rng.uniform(-1, 1, (5000, 3)).astype(np.float32)
    R = iv.so3_exp(np.radians(3.0) * np.array([0.6, -0.8, 0.0]))
    t = np.array([0.02, 0.01, -0.03])
    src = ((tgt.astype(np.float64) - t) @ R).astype(np.float32)
    Tg, rg = cil.icp(_cuda(src), _cuda(tgt), None, iters=25, max_corr_dist=0.5,
                     metric="point_to_point")
    np.testing.assert_allclose(Tg[:3, :3], R, atol=2e-6)
    np.testing.assert_allclose(Tg[:3, 3], t, atol=2e-6)
    assert rg["n_inliers"] == len(src)


@pytest.mark.parametrize("wp,wl", [(0.3, 1.0), (1.0, 0.2)])
def test_combined(surface, wp, wl):
    # a rejection distance no correspondence comes near: with a point term,
    # one correspondence accepted on one side only (FP32 vs FP64 distance at
    # d_max) moves the translation by ~d_max / n, which is about the bar
    p, nrm = surface
    Tg, rg = cil.icp(_cuda(p.source), _cuda(p.target), _cuda(nrm), iters=15, max_corr_dist=0.5,
                     metric="combined", w_point=wp, w_plane=wl)
    o = iv.icp(p.source, p.target, nrm, iters=15, max_corr_dist=0.5, metric="combined",
               w_point=wp, w_plane=wl)
    _same(Tg, o["T"], p.target)
    assert abs(rg["n_inliers"] - o["n_inliers"]) <= 2
    assert rg["rmse"] == pytest.approx(o["rmse"], rel=1e-4)


def test_combined_without_point_term_is_point_to_plane(surface):
    p, nrm = surface
    args = (_cuda(p.source), _cuda(p.target), _cuda(nrm))
    Ta, ra = cil.icp(*args, iters=10, max_corr_dist=0.1, metric="combined", w_point=0.0, w_plane=1.0)
    Tb, rb = cil.icp_point_to_plane(*args, iters=10, max_corr_dist=0.1)
    assert np.array_equal(Ta, Tb) and ra == rb


def _projective_setup():
    p = synth.depth_frame_pair(0)
    m = p.meta
    pm = np.full(m["w"] * m["h"], -1, np.int32)
    pm[m["target_pixels"]] = np.arange(len(p.target), dtype=np.int32)
    on, _, _ = oracle.normals(p.target, 10, p.viewpoint, method="kdtree")
    return p, m, _cuda(pm.reshape(m["h"], m["w"])), on.astype(np.float32)


@pytest.mark.parametrize("metric", ["point_to_plane", "point_to_point"])
def test_projective(metric):
    p, m, pm, nrm = _projective_setup()
    kw = dict(iters=15, max_corr_dist=0.05, metric=metric)
    Tg, rg = cil.icp(_cuda(p.source), _cuda(p.target), _cuda(nrm), association="projective",
                     pixel_map=pm, intrinsics=m["intrinsics"], **kw)
    o = iv.icp(p.source, p.target, nrm, association="projective", pixels=m["target_pixels"],
               width=m["w"], height=m["h"], intrinsics=m["intrinsics"], **kw)
    _same(Tg, o["T"], p.target)
    assert abs(rg["n_inliers"] - o["n_inliers"]) <= 10
    if metric == "point_to_plane":
        # and the frame pair is registered (projective point-to-point, like
        # the oracle, is still ~0.03 rad away after 15 rounds)
        assert rot_angle(Tg[:3, :3], p.T_gt[:3, :3]) < 3e-3


def test_invalid_options_are_rejected(surface):
    p, nrm = surface
    with pytest.raises(cil.CilError):
        cil.icp(_cuda(p.source), _cuda(p.target), _cuda(nrm), metric="combined", w_point=-1.0)
    with pytest.raises(cil.CilError):  # plane metrics need normals
        cil.icp(_cuda(p.source), _cuda(p.target), None, metric="combined", w_point=1.0)
