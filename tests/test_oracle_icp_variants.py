"""Pins of the ICP-variant oracle (oracle/icp_variants.py) against things other
than itself: exact motions, an independent closed form (Horn's quaternion
method), the C point-to-plane oracle, least squares on independently built
rows, and self-correspondence of an organised frame."""
import numpy as np
import pytest

import oracle
from oracle import icp_variants as iv
from paper_1807_00399_gb300 import synth


def _rot(axis, deg):
    a = np.asarray(axis, np.float64)
    a /= np.linalg.norm(a)
    t = np.radians(deg)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + np.sin(t) * K + (1 - np.cos(t)) * K @ K


def _horn(P, Q):
    """Horn's closed form (unit quaternion = top eigenvector of the 4x4
    matrix built from the cross-covariance) -- a different derivation from
    the SVD route the oracle takes."""
    cp, cq = P.mean(0), Q.mean(0)
    S = (P - cp).T @ (Q - cq)
    Sxx, Sxy, Sxz, Syx, Syy, Syz, Szx, Szy, Szz = S.ravel()
    N = np.array([
        [Sxx + Syy + Szz, Syz - Szy, Szx - Sxz, Sxy - Syx],
        [Syz - Szy, Sxx - Syy - Szz, Sxy + Syx, Szx + Sxz],
        [Szx - Sxz, Sxy + Syx, -Sxx + Syy - Szz, Syz + Szy],
        [Sxy - Syx, Szx + Sxz, Syz + Szy, -Sxx - Syy + Szz]])
    w, V = np.linalg.eigh(N)
    q0, qx, qy, qz = V[:, -1]
    R = np.array([
        [q0 * q0 + qx * qx - qy * qy - qz * qz, 2 * (qx * qy - q0 * qz), 2 * (qx * qz + q0 * qy)],
        [2 * (qy * qx + q0 * qz), q0 * q0 - qx * qx + qy * qy - qz * qz, 2 * (qy * qz - q0 * qx)],
        [2 * (qz * qx - q0 * qy), 2 * (qz * qy + q0 * qx), q0 * q0 - qx * qx - qy * qy + qz * qz]])
    return R, cq - R @ cp


def test_kabsch_exact_and_proper():
    rng = np.random.default_rng(0)
    P = rng.normal(size=(50, 3))
    R = _rot([1, 2, 3], 37.0)
    t = np.array([0.3, -1.2, 2.0])
    Rk, tk = iv.kabsch(P, P @ R.T + t)
    np.testing.assert_allclose(Rk, R, atol=1e-12)
    np.testing.assert_allclose(tk, t, atol=1e-12)
    # a mirrored target still yields a proper rotation
    M = np.diag([1.0, 1.0, -1.0])
    Rm, _ = iv.kabsch(P, P @ M.T)
    assert np.linalg.det(Rm) == pytest.approx(1.0, abs=1e-12)


def test_point_to_point_round_equals_horn():
    p = synth.surface_pair(3, n=3000, max_angle_deg=8.0, max_trans=0.04)
    out = iv.icp(p.source, p.target, iters=1, max_corr_dist=0.1, metric="point_to_point")
    idx = iv.nn_correspondences(iv.transform(p.source, np.eye(4)), p.target.astype(np.float64),
                                float(np.float32(0.1)))
    m = idx >= 0
    R, t = _horn(p.source.astype(np.float64)[m], p.target.astype(np.float64)[idx[m]])
    np.testing.assert_allclose(out["T"][:3, :3], R, atol=1e-10)
    np.testing.assert_allclose(out["T"][:3, 3], t, atol=1e-10)


def test_point_to_point_recovers_exact_motion():
    rng = np.random.default_rng(1)
    tgt = rng.uniform(-1, 1, (2000, 3)).astype(np.float32)
    R = _rot([0.3, -1, 0.5], 4.0)
    t = np.array([0.02, -0.01, 0.015])
    # source = target moved by the inverse motion, so T_gt = [R t]
    src = ((tgt.astype(np.float64) - t) @ R).astype(np.float32)
    out = iv.icp(src, tgt, iters=30, max_corr_dist=0.5, metric="point_to_point")
    T = out["T"]
    Rs = src.astype(np.float64) @ T[:3, :3].T + T[:3, 3]
    assert np.abs(Rs - tgt).max() < 1e-6
    assert out["n_inliers"] == 2000 and out["rmse"] < 1e-6


def test_combined_with_zero_point_weight_is_the_plane_oracle():
    p = synth.surface_pair(4, n=4000)
    on, _, _ = oracle.normals(p.target, 10, p.viewpoint)
    nrm = on.astype(np.float32)
    a = iv.icp(p.source, p.target, nrm, iters=6, max_corr_dist=0.1, metric="combined",
               w_point=0.0, w_plane=1.0)
    b = oracle.icp(p.source, p.target, nrm, iters=6, max_corr_dist=0.1)
    np.testing.assert_allclose(a["T"], b["T"], atol=1e-9)
    assert a["n_inliers"] == b["n_inliers"]
    assert a["rmse"] == pytest.approx(b["rmse"], rel=1e-9)


def test_combined_round_equals_lstsq_on_stacked_rows():
    p = synth.surface_pair(5, n=2000)
    on, _, _ = oracle.normals(p.target, 10, p.viewpoint)
    nrm = on.astype(np.float32)
    wp, wl = 0.3, 1.7
    out = iv.icp(p.source, p.target, nrm, iters=1, max_corr_dist=0.1, metric="combined",
                 w_point=wp, w_plane=wl)
    P = p.source.astype(np.float64)
    idx = iv.nn_correspondences(P, p.target.astype(np.float64), float(np.float32(0.1)))
    m = idx >= 0
    P, Q, N = P[m], p.target.astype(np.float64)[idx[m]], nrm.astype(np.float64)[idx[m]]
    # rows built here from the definitions: d/dw (R p) = -[p]x at w = 0
    rows, rhs = [], []
    for i in range(len(P)):
        px, py, pz = P[i]
        Jpt = np.array([[0, pz, -py, 1, 0, 0], [-pz, 0, px, 0, 1, 0], [py, -px, 0, 0, 0, 1.0]])
        rows.append(np.sqrt(wp) * Jpt)
        rhs.append(-np.sqrt(wp) * (P[i] - Q[i]))
        rows.append(np.sqrt(wl) * np.concatenate([np.cross(P[i], N[i]), N[i]])[None])
        rhs.append(-np.sqrt(wl) * np.array([N[i] @ (P[i] - Q[i])]))
    xi = np.linalg.lstsq(np.vstack(rows), np.concatenate(rhs), rcond=None)[0]
    np.testing.assert_allclose(out["T"][:3, 3], xi[3:], atol=1e-10)
    np.testing.assert_allclose(out["T"][:3, :3], iv.so3_exp(xi[:3]), atol=1e-10)


def test_combined_recovers_exact_motion():
    p = synth.surface_pair(6, n=4000)
    on, _, _ = oracle.normals(p.target, 10, p.viewpoint)
    R = _rot([1, 1, 0], 3.0)
    t = np.array([0.01, 0.02, -0.01])
    src = ((p.target.astype(np.float64) - t) @ R).astype(np.float32)
    out = iv.icp(src, p.target, on.astype(np.float32), iters=30, max_corr_dist=0.2,
                 metric="combined", w_point=0.5, w_plane=1.0)
    np.testing.assert_allclose(out["T"][:3, :3], R, atol=1e-6)
    np.testing.assert_allclose(out["T"][:3, 3], t, atol=1e-6)


def test_projective_self_association_and_registration():
    p = synth.depth_frame_pair(0)
    m = p.meta
    kw = dict(association="projective", pixels=m["target_pixels"], width=m["w"], height=m["h"],
              intrinsics=m["intrinsics"])
    # every target point projects onto its own pixel
    idx = iv.projective_correspondences(p.target.astype(np.float64), p.target, m["target_pixels"],
                                        m["w"], m["h"], m["intrinsics"], 0.05)
    np.testing.assert_array_equal(idx, np.arange(len(p.target)))
    # and projective point-to-plane ICP registers the frame pair
    on, _, _ = oracle.normals(p.target, 10, p.viewpoint, method="kdtree")
    out = iv.icp(p.source, p.target, on.astype(np.float32), iters=15, max_corr_dist=0.05,
                 metric="point_to_plane", **kw)
    M = out["T"][:3, :3] @ p.T_gt[:3, :3].T
    ang = np.arccos(np.clip((np.trace(M) - 1) / 2, -1, 1))
    assert ang < 2e-3 and out["status"] == 0


def test_degenerate_rounds_keep_the_transform():
    tgt = np.zeros((2, 3), np.float32)
    out = iv.icp(tgt, tgt, iters=2, metric="point_to_point")
    assert out["status"] == iv.DEGENERATE
    np.testing.assert_array_equal(out["T"], np.eye(4))
