"""Pins for the oracle's rigid point-to-plane ICP (Sec. 2 ICP base loop,
Sec. 3 point-to-plane estimator after Low 2004, Sec. 4 fixed iterations and
rejection distance).  References: the exact transform of a noiseless moved
copy, a Gauss-Newton step rebuilt with scipy's kd-tree, numpy's least squares
and scipy's rotation-vector exponential, and exact symmetries."""
import numpy as np
import pytest
from scipy.spatial import cKDTree
from scipy.spatial.transform import Rotation

import oracle
from paper_1807_00399_gb300 import synth


def rot_angle(Ra, Rb):
    M = Ra @ Rb.T
    w = np.array([M[2, 1] - M[1, 2], M[0, 2] - M[2, 0], M[1, 0] - M[0, 1]]) / 2
    return np.arctan2(np.linalg.norm(w), (np.trace(M) - 1) / 2)


@pytest.fixture(scope="module")
def pair():
    p = synth.surface_pair(0, n=4000)
    nrm, _, _ = oracle.normals(p.target, 10, p.viewpoint)
    return p, nrm.astype(np.float32)


def test_noiseless_copy_recovers_exact_transform():
    rng = np.random.default_rng(1)
    tgt = synth.surface_points(rng, 3000, noise=0.0).astype(np.float32)
    nrm, _, _ = oracle.normals(tgt, 10, [0, 0, 10])
    T_gen = synth.random_rigid(rng, 8.0, 0.05)
    src = synth.apply_rigid(T_gen, tgt).astype(np.float32)
    out = oracle.icp(src, tgt, nrm.astype(np.float32), iters=30, max_corr_dist=0.2)
    T_inv = np.linalg.inv(T_gen)
    assert rot_angle(out["T"][:3, :3], T_inv[:3, :3]) < 1e-6
    assert np.abs(out["T"][:3, 3] - T_inv[:3, 3]).max() < 1e-6
    assert out["rmse"] < 1e-6 and out["n_inliers"] == 3000
    # closed-form cross-check: Kabsch on the known correspondences
    P = src.astype(np.float64)
    Q = tgt.astype(np.float64)
    pc, qc = P.mean(0), Q.mean(0)
    U, S, Vt = np.linalg.svd((P - pc).T @ (Q - qc))
    D = np.diag([1, 1, np.sign(np.linalg.det(Vt.T @ U.T))])
    Rk = Vt.T @ D @ U.T
    assert rot_angle(out["T"][:3, :3], Rk) < 1e-6
    assert np.abs(out["T"][:3, 3] - (qc - Rk @ pc)).max() < 1e-6


def _gn_step_reference(src, dst, nrm, T, dmax):
    """One linearised point-to-plane step built independently: scipy kd-tree
    correspondences, stacked Jacobian rows, numpy least squares and scipy's
    rotation-vector exponential."""
    P = src.astype(np.float64) @ T[:3, :3].T + T[:3, 3]
    dist, j = cKDTree(dst.astype(np.float64)).query(P, 1)
    keep = dist <= dmax
    P, j = P[keep], j[keep]
    N = nrm[j].astype(np.float64)
    Q = dst[j].astype(np.float64)
    r = ((P - Q) * N).sum(1)
    J = np.column_stack([np.cross(P, N), N])
    xi = np.linalg.lstsq(J, -r, rcond=None)[0]
    D = np.eye(4)
    D[:3, :3] = Rotation.from_rotvec(xi[:3]).as_matrix()
    D[:3, 3] = xi[3:]
    return D @ T, J.T @ J, J.T @ r


def test_one_step_equals_least_squares(pair):
    p, nrm = pair
    T0 = np.eye(4)
    T0[:3, :3] = synth.rotation_from_axis_angle([0.2, -1.0, 0.4], 0.05)
    T0[:3, 3] = [0.01, -0.02, 0.005]
    out = oracle.icp(p.source, p.target, nrm, T_init=T0, iters=1, max_corr_dist=0.1,
                     want_trace=True)
    T_ref, H_ref, g_ref = _gn_step_reference(p.source, p.target, nrm, T0, float(np.float32(0.1)))
    np.testing.assert_allclose(out["H"][0], H_ref, rtol=1e-10, atol=1e-9)
    np.testing.assert_allclose(out["g"][0], g_ref, rtol=1e-9, atol=1e-11)
    np.testing.assert_allclose(out["trace"][0], T_ref, atol=1e-11)


def test_converges_to_generator_transform(pair):
    p, nrm = pair
    out = oracle.icp(p.source, p.target, nrm, iters=20, max_corr_dist=0.1)
    assert out["status"] == 0
    assert rot_angle(out["T"][:3, :3], p.T_gt[:3, :3]) < 2e-3
    assert np.abs(out["T"][:3, 3] - p.T_gt[:3, 3]).max() < 2e-3
    # point-to-plane noise of two independent N(0, 0.002) samples
    assert 0.0015 < out["rmse"] < 0.004


def test_last_step_is_a_fixed_point():
    # with every source point owning an exact counterpart, the correspondences
    # settle and the Gauss-Newton step vanishes (g = 0 at the solution)
    rng = np.random.default_rng(9)
    tgt = synth.surface_points(rng, 3000, noise=0.0).astype(np.float32)
    nrm, _, _ = oracle.normals(tgt, 10, [0, 0, 10])
    src = synth.apply_rigid(synth.random_rigid(rng, 5.0, 0.03), tgt).astype(np.float32)
    out = oracle.icp(src, tgt, nrm.astype(np.float32), iters=30, max_corr_dist=0.2,
                     want_trace=True)
    d = out["trace"][-1] @ np.linalg.inv(out["trace"][-2])
    assert rot_angle(d[:3, :3], np.eye(3)) < 1e-12 and np.abs(d[:3, 3]).max() < 1e-12
    assert np.abs(out["g"][-1]).max() < 1e-9 * np.abs(out["H"][-1]).max()


@pytest.mark.parametrize("axes,signs", [((1, 2, 0), (1, 1, 1)), ((0, 1, 2), (-1, 1, -1))])
def test_rigid_motion_equivariance(pair, axes, signs):
    p, nrm = pair
    G = np.zeros((4, 4))
    for i, (a, s) in enumerate(zip(axes, signs)):
        G[i, a] = s
    G[3, 3] = 1
    g = lambda x: (x @ G[:3, :3].T).astype(np.float32)
    a = oracle.icp(p.source, p.target, nrm, iters=10, max_corr_dist=0.1)
    b = oracle.icp(g(p.source), g(p.target), g(nrm), iters=10, max_corr_dist=0.1)
    np.testing.assert_allclose(b["T"], G @ a["T"] @ np.linalg.inv(G), atol=1e-10)


def test_normal_sign_and_permutation_invariance(pair):
    p, nrm = pair
    a = oracle.icp(p.source, p.target, nrm, iters=10, max_corr_dist=0.1)
    flip = nrm.copy()
    flip[::3] *= -1
    b = oracle.icp(p.source, p.target, flip, iters=10, max_corr_dist=0.1)
    np.testing.assert_allclose(b["T"], a["T"], atol=1e-12)
    rng = np.random.default_rng(7)
    ps = rng.permutation(len(p.source))
    pt = rng.permutation(len(p.target))
    c = oracle.icp(p.source[ps], p.target[pt], nrm[pt], iters=10, max_corr_dist=0.1)
    np.testing.assert_allclose(c["T"], a["T"], atol=1e-11)


def test_kdtree_route_equals_exhaustive(pair):
    p, nrm = pair
    a = oracle.icp(p.source, p.target, nrm, iters=8, max_corr_dist=0.1, method="brute")
    b = oracle.icp(p.source, p.target, nrm, iters=8, max_corr_dist=0.1, method="kdtree")
    np.testing.assert_allclose(b["T"], a["T"], atol=1e-13)
    assert a["n_inliers"] == b["n_inliers"]


def test_planar_target_is_degenerate():
    rng = np.random.default_rng(8)
    xy = rng.uniform(-1, 1, size=(2000, 2))
    tgt = np.column_stack([xy, np.zeros(len(xy))]).astype(np.float32)
    nrm = np.tile(np.float32([0, 0, 1]), (len(tgt), 1))
    src = (tgt + np.float32([0, 0, 0.01])).astype(np.float32)
    out = oracle.icp(src, tgt, nrm, iters=3, max_corr_dist=0.1)
    assert out["status"] == oracle.ICP_DEGENERATE
    np.testing.assert_array_equal(out["T"], np.eye(4))


def test_rejection_distance_and_no_inliers(pair):
    p, nrm = pair
    far = (p.source + np.float32(5.0)).astype(np.float32)
    out = oracle.icp(far, p.target, nrm, iters=2, max_corr_dist=0.1)
    assert out["n_inliers"] == 0 and out["status"] == oracle.ICP_DEGENERATE
    assert np.isnan(out["rmse"])
    # rejection is inclusive on the point-to-point distance
    tgt = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0]], np.float32)
    n4 = np.tile(np.float32([0, 0, 1]), (4, 1))
    src = tgt + np.float32([0, 0, 0.5])
    out = oracle.icp(src, tgt, n4, iters=0, max_corr_dist=0.5)
    assert out["n_inliers"] == 4 and abs(out["rmse"] - 0.5) < 1e-15
    out = oracle.icp(src, tgt, n4, iters=0, max_corr_dist=0.4999)
    assert out["n_inliers"] == 0
