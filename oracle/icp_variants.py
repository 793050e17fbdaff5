"""FP64 oracle for the ICP variants of Sec. 3: the point-to-point metric (closed
form, after Besl & McKay), a weighted combination of the point-to-point and
point-to-plane metrics (both linearised, one Gauss-Newton step per round, after
Low 2004), and correspondences by projective data association on an organised
target frame.

TEST INFRASTRUCTURE.  Only the test-suite and the bench's CPU legs use this
module; the product library never imports it, and it imports nothing from the
product library.

Each round follows the ICP loop of Sec. 2/3 in its order: correspondences at
the current transform, then the estimator, then T <- dT T.  numpy FP64 on the
FP32 inputs promoted exactly; scipy's cKDTree (a library routine, validated
against exhaustive search in the tests) finds nearest neighbours.

Readings (where the paper names the variant but not its details):

* point-to-point estimator: the closed-form minimiser of sum |R p' + t - q|^2
  over the round's correspondences, from the SVD of the centred
  cross-covariance with the determinant sign fixed to a proper rotation;
* weighted combination: minimise w_point * sum |p' - q|^2 +
  w_plane * sum (n . (p' - q))^2, linearised about the current pose with
  T <- [exp(w^), tau; 0 1] T (rows [-[p']x | I] per coordinate and
  [p' x n, n] per plane residual);
* projective association: the target is the organised image of the camera
  it was captured with (target coordinates = that camera's frame; pinhole
  fx, fy, cx, cy; pixel = round-half-even of the projection); p' with z <= 0
  or outside the image has no correspondence, and one is kept only if
  |p' - q| <= d_max (inclusive), like the nearest-neighbour rejection;
* degenerate rounds (fewer than 3 correspondences for the closed form, fewer
  than 6 or a Cholesky pivot <= 1e-12 tr(H) for the linearised metrics) keep
  the transform and report status 5;
* the final RMSE is the metric's own residual after one more association
  pass: sqrt(mean |p' - q|^2) (point-to-point), sqrt(mean (n.(p' - q))^2)
  (point-to-plane), sqrt(mean(w_point |p' - q|^2 + w_plane (n.(p' - q))^2))
  (combination).
"""
from __future__ import annotations

import numpy as np

DEGENERATE = 5


def transform(P, T):
    T = np.asarray(T, np.float64)
    return np.asarray(P, np.float64) @ T[:3, :3].T + T[:3, 3]


def nn_correspondences(src_t, tgt, dmax):
    """Nearest target point of each transformed source point, kept when its
    distance is <= dmax.  Returns target indices (-1: none)."""
    from scipy.spatial import cKDTree
    tree = cKDTree(np.asarray(tgt, np.float64))
    # cKDTree's bound is exclusive; the rejection test is inclusive
    d, idx = tree.query(src_t, k=1, distance_upper_bound=np.nextafter(dmax, np.inf))
    idx = np.where(np.isfinite(d) & (d <= dmax), idx, -1)
    return idx.astype(np.int64)


def projective_correspondences(src_t, tgt, pixels, width, height, intrinsics, dmax):
    """Target point seen at the pixel each transformed source point projects
    to (pixels: flat pixel index v * width + u of every target point)."""
    fx, fy, cx, cy = intrinsics
    pix_map = np.full(width * height, -1, np.int64)
    pix_map[np.asarray(pixels, np.int64)] = np.arange(len(pixels))
    x, y, z = src_t[:, 0], src_t[:, 1], src_t[:, 2]
    with np.errstate(divide="ignore", invalid="ignore"):
        u = np.rint(fx * x / z + cx)
        v = np.rint(fy * y / z + cy)
    ok = (z > 0) & np.isfinite(u) & np.isfinite(v) & (u >= 0) & (u < width) & (v >= 0) & (v < height)
    idx = np.full(len(src_t), -1, np.int64)
    flat = (v[ok] * width + u[ok]).astype(np.int64)
    idx[ok] = pix_map[flat]
    has = idx >= 0
    d2 = np.full(len(src_t), np.inf)
    d2[has] = np.sum((src_t[has] - np.asarray(tgt, np.float64)[idx[has]]) ** 2, axis=1)
    return np.where(has & (d2 <= dmax * dmax), idx, -1)


def kabsch(P, Q):
    """Closed-form rigid (R, t) minimising sum |R p + t - q|^2 (SVD of the
    centred cross-covariance, proper rotation)."""
    cp = P.mean(axis=0)
    cq = Q.mean(axis=0)
    H = (P - cp).T @ (Q - cq)
    U, _, Vt = np.linalg.svd(H)
    d = np.sign(np.linalg.det(Vt.T @ U.T))
    D = np.diag([1.0, 1.0, d if d != 0 else 1.0])
    R = Vt.T @ D @ U.T
    return R, cq - R @ cp


def _skew(w):
    return np.array([[0.0, -w[2], w[1]], [w[2], 0.0, -w[0]], [-w[1], w[0], 0.0]])


def so3_exp(w):
    """Rodrigues' formula."""
    t = np.linalg.norm(w)
    K = _skew(w)
    if t < 1e-12:
        return np.eye(3) + K + 0.5 * K @ K
    return np.eye(3) + np.sin(t) / t * K + (1 - np.cos(t)) / (t * t) * K @ K


def cholesky_solve(H, g):
    """H x = -g by a plain Cholesky; None when a pivot is <= 1e-12 tr(H)."""
    n = H.shape[0]
    tr = np.trace(H)
    if not tr > 0:
        return None
    L = np.zeros_like(H)
    for j in range(n):
        d = H[j, j] - L[j, :j] @ L[j, :j]
        if not d > 1e-12 * tr:
            return None
        L[j, j] = np.sqrt(d)
        for i in range(j + 1, n):
            L[i, j] = (H[i, j] - L[i, :j] @ L[j, :j]) / L[j, j]
    y = np.zeros(n)
    for i in range(n):
        y[i] = (-g[i] - L[i, :i] @ y[:i]) / L[i, i]
    x = np.zeros(n)
    for i in reversed(range(n)):
        x[i] = (y[i] - L[i + 1:, i] @ x[i + 1:]) / L[i, i]
    return x


def point_rows(p):
    """Jacobian rows of the three point-to-point residual coordinates of a
    transformed point p w.r.t. (w, tau): [-[p]x | I]."""
    J = np.zeros((3, 6))
    J[:, :3] = -_skew(p)
    J[:, 3:] = np.eye(3)
    return J


def normal_equations(P, Q, N, w_point, w_plane):
    """H (6x6), g (6) of the weighted combination at the current pose."""
    H = np.zeros((6, 6))
    g = np.zeros(6)
    if w_plane:
        r = np.sum(N * (P - Q), axis=1)
        Jp = np.hstack([np.cross(P, N), N])
        H += w_plane * Jp.T @ Jp
        g += w_plane * Jp.T @ r
    if w_point:
        D = P - Q
        for i in range(len(P)):
            J = point_rows(P[i])
            H += w_point * J.T @ J
            g += w_point * J.T @ D[i]
    return H, g


def metric_rmse(P, Q, N, metric, w_point, w_plane):
    if len(P) == 0:
        return float("nan")
    if metric == "point_to_point":
        e = np.sum((P - Q) ** 2, axis=1)
    elif metric == "point_to_plane":
        e = np.sum(N * (P - Q), axis=1) ** 2
    else:
        e = w_point * np.sum((P - Q) ** 2, axis=1) + w_plane * np.sum(N * (P - Q), axis=1) ** 2
    return float(np.sqrt(e.mean()))


def icp(src, tgt, tgt_normals=None, T_init=None, iters: int = 20, max_corr_dist: float = 0.1,
        metric: str = "point_to_point", w_point: float = 1.0, w_plane: float = 1.0,
        association: str = "nn", pixels=None, width: int = 0, height: int = 0,
        intrinsics=None, want_trace: bool = False):
    """Rigid ICP.  metric: point_to_point | point_to_plane | combined;
    association: nn | projective (needs pixels, width, height, intrinsics).
    Returns a dict with T (source -> target), rmse, n_inliers, status."""
    src = np.asarray(src, np.float32).astype(np.float64)
    tgt = np.asarray(tgt, np.float32).astype(np.float64)
    nrm = None if tgt_normals is None else np.asarray(tgt_normals, np.float32).astype(np.float64)
    dmax = float(np.float32(max_corr_dist))
    T = np.eye(4) if T_init is None else np.asarray(T_init, np.float64).copy()
    if metric == "point_to_plane":
        w_point, w_plane = 0.0, 1.0
    elif metric == "point_to_point":
        w_point, w_plane = 1.0, 0.0
    status = 0
    trace = []

    def associate(T):
        P = transform(src, T)
        if association == "nn":
            idx = nn_correspondences(P, tgt, dmax)
        else:
            idx = projective_correspondences(P, tgt, pixels, width, height, intrinsics, dmax)
        m = idx >= 0
        if nrm is not None and w_plane:
            m &= np.all(np.isfinite(nrm[np.maximum(idx, 0)]), axis=1)
        return P[m], tgt[idx[m]], (nrm[idx[m]] if nrm is not None else None)

    for _ in range(iters):
        P, Q, N = associate(T)
        if metric == "point_to_point":
            if len(P) < 3:
                status = DEGENERATE
            else:
                R, t = kabsch(P, Q)
                dT = np.eye(4)
                dT[:3, :3] = R
                dT[:3, 3] = t
                T = dT @ T
        else:
            H, g = normal_equations(P, Q, N, w_point, w_plane)
            xi = cholesky_solve(H, g) if len(P) >= 6 else None
            if xi is None:
                status = DEGENERATE
            else:
                dT = np.eye(4)
                dT[:3, :3] = so3_exp(xi[:3])
                dT[:3, 3] = xi[3:]
                T = dT @ T
        trace.append(T.copy())
    P, Q, N = associate(T)
    out = {"T": T, "rmse": metric_rmse(P, Q, N, metric, w_point, w_plane), "n_inliers": len(P),
           "status": status}
    if want_trace:
        out["trace"] = np.array(trace)
    return out
