"""Pins for the oracle's PCA normals and curvature (Sec. 3 surface normal and
curvature estimation; Sec. 4 kNN neighbourhoods and viewpoint-consistent
orientation).  The references are numpy's symmetric eigensolver, exact plane
and sphere geometry, closed-form covariances and exact symmetries."""
import numpy as np
import pytest

import oracle
from paper_1807_00399_gb300 import synth


def angle_unsigned(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    cr = np.linalg.norm(np.cross(a, b), axis=-1)
    dt = np.abs((a * b).sum(-1))
    return np.arctan2(cr, dt)


def test_jacobi_matches_numpy_eigh():
    rng = np.random.default_rng(0)
    mats = []
    for _ in range(300):
        A = rng.normal(size=(3, 3))
        mats.append(A @ A.T)
    mats.append(np.diag([3.0, 1.0, 2.0]))
    mats.append(np.diag([1.0, 1.0, 5.0]))          # repeated eigenvalue
    Q = np.linalg.qr(rng.normal(size=(3, 3)))[0]
    mats.append(Q @ np.diag([1e-8, 1.0, 1.0]) @ Q.T)  # flat + repeated
    mats.append(Q @ np.diag([0.0, 2.0, 7.0]) @ Q.T)   # singular
    for C in mats:
        ev, V = oracle.sym3_eigen(C)
        w, U = np.linalg.eigh(C)
        np.testing.assert_allclose(ev, w, rtol=0, atol=1e-13 * max(1.0, np.abs(w).max()))
        # eigen-equation and orthonormality (vectors of repeated values are not unique)
        np.testing.assert_allclose(C @ V, V * ev, atol=1e-12 * max(1.0, np.abs(w).max()))
        np.testing.assert_allclose(V.T @ V, np.eye(3), atol=1e-13)
        if w[1] - w[0] > 1e-6 * max(1.0, w[2]):
            assert angle_unsigned(V[:, 0], U[:, 0]) < 1e-10


def test_plane_gives_exact_normal_and_zero_curvature():
    rng = np.random.default_rng(1)
    xy = rng.uniform(-1, 1, size=(3000, 2))
    pts = np.column_stack([xy, np.zeros(len(xy))]).astype(np.float32)
    n, c, ev = oracle.normals(pts, 10, [0.3, -0.2, 10.0])
    assert np.all(n[:, 2] == 1.0) and np.all(n[:, :2] == 0.0)  # oriented to +z
    assert np.all(c == 0.0)
    n2, _, _ = oracle.normals(pts, 10, [0.0, 0.0, -10.0])
    assert np.all(n2[:, 2] == -1.0)


def test_tilted_plane_normal():
    rng = np.random.default_rng(2)
    m = np.array([0.3, -0.5, 0.8])
    m /= np.linalg.norm(m)
    u = np.cross(m, [1.0, 0, 0])
    u /= np.linalg.norm(u)
    v = np.cross(m, u)
    ab = rng.uniform(-1, 1, size=(4000, 2))
    pts = (ab[:, :1] * u + ab[:, 1:] * v).astype(np.float32)
    n, c, _ = oracle.normals(pts, 12, m * 10)
    # float32 rounding of the samples moves them ~1e-7 off the plane
    assert angle_unsigned(n, m).max() < 2e-5
    assert np.all((n @ m) > 0)
    assert c.max() < 1e-9


def test_sphere_normals_are_radial_and_oriented():
    rng = np.random.default_rng(3)
    d = rng.normal(size=(20000, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    pts = (2.0 * d).astype(np.float32)
    n, c, _ = oracle.normals(pts, 10, [0.0, 0.0, 0.0])  # viewpoint at the centre
    # the PCA plane of a curved patch is tilted by O(R_k / radius) for
    # lopsided random neighbourhoods: bound the mean tightly, the worst loosely
    a = angle_unsigned(n, d)
    assert a.mean() < 0.01 and a.max() < 0.08
    assert np.all((n * d).sum(1) < 0)  # inward, towards the viewpoint


def test_isotropic_star_curvature_one_third():
    # self + 6 face neighbours of a lattice point: covariance (2/7) I
    pts = synth.lattice_points((3, 3, 3))
    centre = 13
    n, c, ev = oracle.normals(pts, 7, [0, 0, 10])
    np.testing.assert_allclose(ev[centre], [2 / 7] * 3, rtol=1e-14)
    assert abs(c[centre] - 1.0 / 3.0) < 1e-15


def test_closed_form_covariance_of_a_square():
    # 4 corners of a unit square in the xy plane + its centre: covariance
    # diag(0.2, 0.2, 0) (mean at the centre, sum x^2 = 4 * 0.25)
    pts = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0], [0.5, 0.5, 0]], np.float32)
    n, c, ev = oracle.normals(pts, 5, [0, 0, 1])
    np.testing.assert_allclose(ev[4], [0.0, 0.2, 0.2], atol=1e-15)
    assert n[4].tolist() == [0.0, 0.0, 1.0]


@pytest.mark.parametrize("axes,signs", [((1, 2, 0), (1, 1, 1)), ((0, 1, 2), (-1, 1, -1))])
def test_exact_rotation_equivariance(axes, signs):
    pts = synth.surface_pair(4, n=3000).target
    vp = np.array([0.2, 0.1, 10.0])
    g = lambda p: p[:, list(axes)] * np.asarray(signs, p.dtype)
    n, c, ev = oracle.normals(pts, 10, vp)
    ng, cg, evg = oracle.normals(g(pts).astype(np.float32), 10, g(vp[None])[0])
    np.testing.assert_allclose(ng, g(n), atol=1e-12)
    np.testing.assert_allclose(cg, c, atol=1e-15)


def test_wavy_surface_close_to_analytic_normal():
    # noise-free samples of z = 0.1 sin 4x cos 4y; the PCA normal carries an
    # O(h^2 * curvature) bias, so this is a sanity bound, not parity
    rng = np.random.default_rng(5)
    pts = synth.surface_points(rng, 20000, noise=0.0).astype(np.float32)
    n, c, _ = oracle.normals(pts, 10, [0, 0, 10])
    x, y = pts[:, 0].astype(np.float64), pts[:, 1].astype(np.float64)
    fx = 0.4 * np.cos(4 * x) * np.cos(4 * y)
    fy = -0.4 * np.sin(4 * x) * np.sin(4 * y)
    a = np.column_stack([-fx, -fy, np.ones_like(fx)])
    a /= np.linalg.norm(a, axis=1, keepdims=True)
    interior = (np.abs(x) < 0.95) & (np.abs(y) < 0.95)
    assert angle_unsigned(n[interior], a[interior]).max() < 0.05
    assert np.all(n[:, 2] > 0)


def test_degenerate_neighbourhoods_give_nan():
    two = np.array([[0, 0, 0], [1, 0, 0]], np.float32)
    n, c, _ = oracle.normals(two, 10, [0, 0, 1])
    assert np.isnan(n).all() and np.isnan(c).all()
    same = np.zeros((6, 3), np.float32)
    n, c, _ = oracle.normals(same, 4, [0, 0, 1])
    assert np.isnan(n).all() and np.isnan(c).all()


def test_subset_route_equals_full():
    pts = synth.surface_pair(6, n=3000).target
    sel = np.arange(0, 3000, 37)
    n, c, ev = oracle.normals(pts, 10, [0, 0, 10])
    ns, cs, evs = oracle.normals_subset(pts, sel, 10, [0, 0, 10])
    np.testing.assert_allclose(ns, n[sel], atol=1e-14)
    np.testing.assert_allclose(cs, c[sel], atol=1e-15)


def test_radius_normals_plane_and_star():
    rng = np.random.default_rng(7)
    xy = rng.uniform(-1, 1, size=(2000, 2))
    pts = np.column_stack([xy, np.zeros(len(xy))]).astype(np.float32)
    n, c, ev, cnt = oracle.normals_radius(pts, 0.1, [0, 0, 10])
    ok = cnt >= 3
    assert ok.mean() > 0.99
    assert np.all(n[ok] == [0.0, 0.0, 1.0]) and np.all(c[ok] == 0.0)
    assert np.isnan(n[~ok]).all()
    # on the integer lattice a radius-1 ball is the 7-point star (covariance (2/7) I)
    lat = synth.lattice_points((3, 3, 3))
    n, c, ev, cnt = oracle.normals_radius(lat, 1.0, [0, 0, 10])
    assert cnt[13] == 7 and abs(c[13] - 1.0 / 3.0) < 1e-15


def test_radius_normals_equal_knn_normals_when_the_sets_coincide():
    # when the radius ball holds exactly the k nearest points, both routes agree
    pts = synth.surface_pair(8, n=3000).target
    k = 10
    idx, d2 = oracle.knn(pts, pts, k + 1)
    # a radius strictly between the k-th and (k+1)-th distance of every point
    # is not available globally, so compare per point with its own radius
    sel = np.arange(0, 3000, 97)
    nk, ck, _ = oracle.normals(pts, k, [0, 0, 10])
    for i in sel:
        r = float(np.sqrt(0.5 * (d2[i, k - 1] + d2[i, k])))
        if not (np.float32(r) ** 2 > d2[i, k - 1] and np.float32(r) ** 2 < d2[i, k]):
            continue
        nr, cr, _, cnt = oracle.normals_radius(pts, r, [0, 0, 10])
        assert cnt[i] == k
        np.testing.assert_allclose(nr[i], nk[i], atol=1e-12)
        assert abs(cr[i] - ck[i]) < 1e-15


def test_radius_normals_subset_route_equals_full():
    pts = synth.surface_pair(9, n=2000).target
    sel = np.arange(0, 2000, 13)
    n, c, ev, cnt = oracle.normals_radius(pts, 0.07, [0, 0, 10])
    ns, cs, evs, cnts = oracle.normals_radius(pts, 0.07, [0, 0, 10], sel=sel)
    np.testing.assert_array_equal(cnts, cnt[sel])
    np.testing.assert_allclose(ns, n[sel], atol=0)
