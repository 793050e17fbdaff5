"""PCA normal parity: libcil (cil_estimate_normals) against the FP64 Jacobi
oracle.

Bar: normals within 1e-4 rad up to sign where the eigenvector is well
conditioned.  The library builds the covariance in FP32 from exactly rounded
offsets, so its entries err by ~eps32 * R^2 (R = neighbourhood radius); the
smallest eigenvector then moves by about that error over the gap l1 - l0.
With l2 ~ R^2 / 4 the angle is ~1e-6 / ((l1 - l0) / l2), so the 1e-4 rad bar
is asserted where (l1 - l0) / l2 >= 1e-2; points below that gate (edges,
corners, isotropic blobs) are counted, not failed.  Curvature l0 / sum(l)
carries an absolute error of a few eps32: we allow 1e-5.  Orientation must
agree wherever |n . (v - p)| / |v - p| > 1e-3."""
import numpy as np
import pytest
import torch

import oracle
import paper_1807_00399_gb300 as cil
from paper_1807_00399_gb300 import synth
from parity import angle_unsigned

pytestmark = pytest.mark.gpu
GATE = 1e-2
TOL_ANGLE = 1e-4
TOL_CURV = 1e-5


def _gpu_normals(pts, k, vp, **kw):
    x = torch.from_numpy(np.ascontiguousarray(pts)).cuda()
    n, c = cil.estimate_normals(x, k, vp, **kw)
    torch.cuda.synchronize()
    assert cil.sync_status() == 0
    return n.cpu().numpy().astype(np.float64), c.cpu().numpy().astype(np.float64)


def _compare(pts, k, vp, gn, gc, on, oc, oev, sel=None):
    """Asserts the bars; returns the figures to report: points compared,
    points below the eigen-gap gate, the largest and 99th-percentile angle
    above the gate and the largest angle below it (finite normals)."""
    P = pts if sel is None else pts[sel]
    good = (oev[:, 1] - oev[:, 0]) >= GATE * oev[:, 2]
    ang = angle_unsigned(gn, on)
    fin = np.isfinite(ang)
    below = ~good & fin
    figs = {"points": int(len(ang)), "below_gate": int((~good).sum()),
            "max_rad": float(ang[good].max()) if good.any() else 0.0,
            "p99_rad": float(np.percentile(ang[good], 99)) if good.any() else 0.0,
            "max_rad_below_gate": float(ang[below].max()) if below.any() else 0.0}
    assert np.all(ang[good] <= TOL_ANGLE), f"max angle {ang[good].max():.3g} rad"
    np.testing.assert_allclose(gc[good], oc[good], atol=TOL_CURV, rtol=0)
    assert np.allclose(np.linalg.norm(gn[good], axis=1), 1.0, atol=1e-5)
    v = np.asarray(vp, np.float64) - P.astype(np.float64)
    s_o = (on * v).sum(1) / np.linalg.norm(v, axis=1)
    clear = good & (np.abs(s_o) > 1e-3)
    assert np.all((gn[clear] * on[clear]).sum(1) > 0), "orientation differs"
    return figs


@pytest.mark.parametrize("k", [3, 10, 16, 32])
def test_surface_normals(k, parity_report):
    p = synth.surface_pair(0, n=10_000)
    gn, gc = _gpu_normals(p.target, k, p.viewpoint)
    on, oc, oev = oracle.normals(p.target, k, p.viewpoint)
    parity_report(f"normals, wavy surface 10k, k={k}",
                  **_compare(p.target, k, p.viewpoint, gn, gc, on, oc, oev))


def test_plane_exact_normal():
    rng = np.random.default_rng(1)
    m = np.array([0.3, -0.5, 0.8])
    m /= np.linalg.norm(m)
    u = np.cross(m, [1.0, 0, 0])
    u /= np.linalg.norm(u)
    v = np.cross(m, u)
    ab = rng.uniform(-1, 1, (6000, 2))
    pts = (ab[:, :1] * u + ab[:, 1:] * v).astype(np.float32)
    gn, gc = _gpu_normals(pts, 10, 10 * m)
    assert angle_unsigned(gn, m).max() < 1e-4
    assert np.all(gn @ m > 0)
    assert np.all(gc < 1e-5)


def test_degenerate_inputs_give_nan():
    gn, gc = _gpu_normals(np.array([[0, 0, 0], [1, 0, 0]], np.float32), 10, [0, 0, 1])
    assert np.isnan(gn).all() and np.isnan(gc).all()
    gn, gc = _gpu_normals(np.zeros((20, 3), np.float32), 5, [0, 0, 1])
    assert np.isnan(gn).all() and np.isnan(gc).all()


def test_depth_frame_sampled(parity_report):
    p = synth.depth_frame_pair(0)
    sel = np.random.default_rng(2).choice(len(p.target), 3000, replace=False)
    gn, gc = _gpu_normals(p.target, 10, p.viewpoint)
    on, oc, oev = oracle.normals_subset(p.target, sel, 10, p.viewpoint, method="kdtree")
    parity_report("normals, depth frame (3000 sampled points), k=10",
                  **_compare(p.target, 10, p.viewpoint, gn[sel], gc[sel], on, oc, oev, sel))


def test_lidar_sampled(parity_report):
    p = synth.lidar_sweep_pair(0)
    sel = np.random.default_rng(3).choice(len(p.target), 3000, replace=False)
    gn, gc = _gpu_normals(p.target, 16, p.viewpoint)
    on, oc, oev = oracle.normals_subset(p.target, sel, 16, p.viewpoint, method="kdtree")
    parity_report("normals, LiDAR sweep (3000 sampled points), k=16",
                  **_compare(p.target, 16, p.viewpoint, gn[sel], gc[sel], on, oc, oev, sel))


def test_deterministic():
    p = synth.surface_pair(4, n=30_000)
    a = _gpu_normals(p.target, 10, p.viewpoint)
    b = _gpu_normals(p.target, 10, p.viewpoint)
    assert np.array_equal(a[0], b[0], equal_nan=True) and np.array_equal(a[1], b[1], equal_nan=True)


def test_permutation_equivariant():
    """Normals of permuted points are the permuted normals (the neighbourhood
    of each point does not depend on the order the points come in)."""
    p = synth.surface_pair(31, n=20_000).target
    perm = np.random.default_rng(32).permutation(len(p))
    vp = (0.0, 0.0, 10.0)
    gn, gc = _gpu_normals(p, 10, vp)
    pn, pc = _gpu_normals(p[perm], 10, vp)
    fin = np.isfinite(gn).all(axis=1)
    assert np.all(angle_unsigned(pn[fin], gn[perm][fin]) <= 1e-6)
    np.testing.assert_allclose(pc, gc[perm], atol=1e-7, rtol=0)
