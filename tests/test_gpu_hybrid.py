"""Hybrid query (k nearest within r) and radius-neighbourhood normals:
libcil against the FP64 oracle, with the kNN and normals bars of
test_gpu_knn.py / test_gpu_normals.py (points on the ball's boundary,
|d2 - r^2| <= 1e-6 r^2, may go either way)."""
import numpy as np
import pytest
import torch

import oracle
import paper_1807_00399_gb300 as cil
from paper_1807_00399_gb300 import synth
from parity import angle_unsigned, check_knn_rows

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("k,r", [(10, 0.05), (16, 0.02), (32, 0.2), (4, 0.0)])
def test_hybrid_matches_oracle(k, r):
    p = synth.surface_pair(0, n=10_000)
    ref = p.target
    qry = np.concatenate([p.source[:3000], p.source[:50] + np.float32(5.0)])  # far queries too
    R = torch.from_numpy(ref).cuda()
    gi, gd = cil.knn_hybrid(R, torch.from_numpy(qry).cuda(), k, r)
    torch.cuda.synchronize()
    gi, gd = gi.cpu().numpy(), gd.cpu().numpy()
    oi, od = oracle.knn_hybrid(ref, qry, k + 1, r)
    rr = float(np.float32(r)) ** 2
    # drop rows with a neighbour on the ball's boundary (FP32 vs FP64 membership)
    bnd = (np.abs(od - rr) <= 1e-6 * rr).any(1) | (np.abs(gd.astype(np.float64) - rr) <= 1e-6 * rr).any(1)
    keep = ~bnd
    check_knn_rows(ref, qry[keep], gi[keep], gd[keep], oi[keep], od[keep], k)
    assert np.all(gi[-50:] == -1)


def test_hybrid_self_query_depth_frame_sampled():
    p = synth.depth_frame_pair(0)
    R = torch.from_numpy(p.target).cuda()
    gi, gd = cil.knn_hybrid(R, R, 10, 0.01)
    torch.cuda.synchronize()
    rows = np.random.default_rng(1).choice(len(p.target), 1500, replace=False)
    oi, od = oracle.knn_hybrid(p.target, p.target[rows], 11, 0.01)
    rr = float(np.float32(0.01)) ** 2
    gi, gd = gi.cpu().numpy()[rows], gd.cpu().numpy()[rows]
    keep = ~((np.abs(od - rr) <= 1e-6 * rr).any(1) | (np.abs(gd - rr) <= 1e-6 * rr).any(1))
    check_knn_rows(p.target, p.target[rows][keep], gi[keep], gd[keep], oi[keep], od[keep], 10)


@pytest.mark.parametrize("r", [0.04, 0.08])
def test_radius_normals_match_oracle(r):
    p = synth.surface_pair(1, n=8000)
    X = torch.from_numpy(p.target).cuda()
    gn, gc, cnt = cil.estimate_normals_radius(X, r, p.viewpoint)
    torch.cuda.synchronize()
    on, oc, oev, ocnt = oracle.normals_radius(p.target, r, p.viewpoint)
    cnt = cnt.cpu().numpy()
    # counts may differ only through boundary points
    assert np.abs(cnt - ocnt).max() <= 2 and (cnt == ocnt).mean() > 0.99
    same = (cnt == ocnt) & (ocnt >= 3)
    good = same & ((oev[:, 1] - oev[:, 0]) >= 1e-2 * oev[:, 2])
    gn = gn.cpu().numpy().astype(np.float64)
    ang = angle_unsigned(gn[good], on[good])
    assert ang.max() <= 1e-4, f"max angle {ang.max():.3g}"
    np.testing.assert_allclose(gc.cpu().numpy()[good], oc[good], atol=1e-5)
    assert np.all((gn[good] * on[good]).sum(1) > 0)
    assert np.isnan(gn[ocnt < 3]).all()


def test_radius_normals_depth_frame_1cm_sampled():
    # the paper's second normals experiment uses 1 cm balls on VGA depth frames
    p = synth.depth_frame_pair(0)
    X = torch.from_numpy(p.target).cuda()
    gn, gc, cnt = cil.estimate_normals_radius(X, 0.01, p.viewpoint)
    torch.cuda.synchronize()
    sel = np.random.default_rng(2).choice(len(p.target), 400, replace=False)
    on, oc, oev, ocnt = oracle.normals_radius(p.target, 0.01, p.viewpoint, sel=sel)
    cnt = cnt.cpu().numpy()[sel]
    assert (cnt == ocnt).mean() > 0.98
    same = (cnt == ocnt) & (ocnt >= 3)
    good = same & ((oev[:, 1] - oev[:, 0]) >= 1e-2 * oev[:, 2])
    ang = angle_unsigned(gn.cpu().numpy()[sel][good], on[good])
    assert good.sum() > 200 and ang.max() <= 1e-4
