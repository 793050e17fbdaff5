"""Hybrid query (k nearest within r) and radius-neighbourhood normals:
libcil against the FP64 oracle, with the kNN and normals bars of
test_gpu_knn.py / test_gpu_normals.py (points on the ball's boundary,
|d2 - r^2| <= 1e-6 r^2, may go either way; every other point's membership
must agree, so a neighbourhood's size may differ from the oracle's only by
boundary points)."""
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


def _count_bounds(ref, qry, r):
    """Per query, the neighbourhood sizes the membership rule allows: the
    oracle's count without its boundary members (lo) up to the count with
    every boundary point just outside the ball as well (hi); the boundary is
    |d2 - r^2| <= 1e-6 r^2 in FP64."""
    r2 = float(np.float32(r)) ** 2
    # a float32 radius whose square exceeds r^2 (1 + 1e-6): every outside
    # boundary point is a member of this larger ball
    r_out = np.nextafter(np.float32(np.float32(r) * np.float32(1 + 1e-6)), np.float32(np.inf))
    assert float(r_out) ** 2 >= r2 * (1 + 1e-6)
    off, _, d2 = oracle.radius(ref, qry, float(r_out))
    row = np.repeat(np.arange(len(qry)), np.diff(off))
    inside = d2 <= r2
    bnd = np.abs(d2 - r2) <= 1e-6 * r2
    n_in = np.bincount(row, weights=inside, minlength=len(qry)).astype(np.int64)
    n_bnd_in = np.bincount(row, weights=inside & bnd, minlength=len(qry)).astype(np.int64)
    n_bnd_out = np.bincount(row, weights=~inside & bnd, minlength=len(qry)).astype(np.int64)
    return n_in, n_in - n_bnd_in, n_in + n_bnd_out


@pytest.mark.parametrize("r", [0.04, 0.08])
def test_radius_normals_match_oracle(r):
    p = synth.surface_pair(1, n=8000)
    X = torch.from_numpy(p.target).cuda()
    gn, gc, cnt = cil.estimate_normals_radius(X, r, p.viewpoint)
    torch.cuda.synchronize()
    on, oc, oev, ocnt = oracle.normals_radius(p.target, r, p.viewpoint)
    cnt = cnt.cpu().numpy()
    # counts may differ only through boundary points
    n_in, lo, hi = _count_bounds(p.target, p.target, r)
    assert np.array_equal(n_in, ocnt)
    bad = (cnt < lo) | (cnt > hi)
    assert not bad.any(), f"{bad.sum()} neighbourhood sizes differ beyond the boundary points"
    print(f"r={r}: sizes differing from the oracle's (boundary points only): "
          f"{int((cnt != ocnt).sum())} of {len(cnt)}")
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
    n_in, lo, hi = _count_bounds(p.target, p.target[sel], 0.01)
    assert np.array_equal(n_in, ocnt)
    bad = (cnt < lo) | (cnt > hi)
    assert not bad.any(), f"{bad.sum()} neighbourhood sizes differ beyond the boundary points"
    same = (cnt == ocnt) & (ocnt >= 3)
    good = same & ((oev[:, 1] - oev[:, 0]) >= 1e-2 * oev[:, 2])
    ang = angle_unsigned(gn.cpu().numpy()[sel][good], on[good])
    assert good.sum() > 200 and ang.max() <= 1e-4
