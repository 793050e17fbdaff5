"""Pins for the oracle's kNN and radius search (Sec. 3, KDTree k-NN and radius
queries).  Each check compares against something other than the oracle: a
library kd-tree (scipy cKDTree), neighbour sets of an integer lattice counted
by hand, or an exact symmetry of the data."""
import numpy as np
import pytest
from scipy.spatial import cKDTree

import oracle
from paper_1807_00399_gb300 import synth


def _cloud(seed, n):
    return np.random.default_rng(seed).uniform(-1, 1, size=(n, 3)).astype(np.float32)


@pytest.mark.parametrize("k", [1, 4, 10, 16, 32])
def test_knn_matches_library_kdtree(k):
    ref = _cloud(0, 3000)
    qry = _cloud(1, 500)
    idx, d2 = oracle.knn(ref, qry, k)
    dd, ii = cKDTree(ref.astype(np.float64)).query(qry.astype(np.float64), k)
    dd = dd.reshape(len(qry), k)
    ii = ii.reshape(len(qry), k)
    assert np.array_equal(idx, ii)
    np.testing.assert_allclose(d2, dd**2, rtol=1e-12, atol=0)


def test_knn_distances_ascending_and_self_first():
    pts = synth.surface_pair(3, n=2000).target
    idx, d2 = oracle.knn(pts, pts, 10)
    assert np.all(np.diff(d2, axis=1) >= 0)
    assert np.array_equal(idx[:, 0], np.arange(len(pts)))  # distinct points: self at d2 = 0
    assert np.all(d2[:, 0] == 0)


def test_lattice_ties_broken_by_index():
    # 5x5x5 integer lattice, index = 25 i + 5 j + l.  Around the centre (2,2,2)
    # (index 62): 6 face neighbours at d2 = 1, 12 edge neighbours at d2 = 2,
    # 8 corner neighbours at d2 = 3.  Each tie group must come out in
    # ascending index order.
    pts = synth.lattice_points((5, 5, 5))
    lin = lambda i, j, l: 25 * i + 5 * j + l
    offs = [(a, b, c) for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)]
    groups = {}
    for o in offs:
        groups.setdefault(sum(x * x for x in o), []).append(lin(2 + o[0], 2 + o[1], 2 + o[2]))
    expect = [62] + sorted(groups[1]) + sorted(groups[2]) + sorted(groups[3])
    idx, d2 = oracle.knn(pts, pts[62:63], 27)
    assert idx[0].tolist() == expect
    assert d2[0].tolist() == [0.0] + [1.0] * 6 + [2.0] * 12 + [3.0] * 8
    # cutting inside a tie group keeps the smallest indices
    idx7, _ = oracle.knn(pts, pts[62:63], 10)
    assert idx7[0].tolist() == expect[:10]


def test_k_larger_than_reference_pads():
    ref = _cloud(2, 5)
    idx, d2 = oracle.knn(ref, ref[:2], 8)
    assert (idx[:, 5:] == -1).all() and np.isinf(d2[:, 5:]).all()
    assert sorted(idx[0, :5].tolist()) == list(range(5))


def test_empty_reference():
    idx, d2 = oracle.knn(np.zeros((0, 3), np.float32), _cloud(3, 4), 3)
    assert (idx == -1).all() and np.isinf(d2).all()


def test_permutation_equivariance():
    ref = _cloud(4, 2000)
    qry = _cloud(5, 300)
    perm = np.random.default_rng(6).permutation(len(ref))
    idx, d2 = oracle.knn(ref, qry, 10)
    idx_p, d2_p = oracle.knn(ref[perm], qry, 10)
    assert np.array_equal(perm[idx_p], idx)
    assert np.array_equal(d2_p, d2)


@pytest.mark.parametrize("axes,signs", [((1, 2, 0), (1, 1, 1)), ((0, 1, 2), (-1, 1, -1)),
                                        ((2, 0, 1), (-1, -1, 1))])
def test_exact_rigid_motion_invariance(axes, signs):
    # axis permutations and sign flips are exact in float32
    ref = _cloud(7, 2000)
    qry = _cloud(8, 300)
    g = lambda p: (p[:, list(axes)] * np.asarray(signs, np.float32)).astype(np.float32)
    idx, d2 = oracle.knn(ref, qry, 12)
    idx_g, d2_g = oracle.knn(g(ref), g(qry), 12)
    assert np.array_equal(idx, idx_g)
    # permuting the axes reorders the three squared terms of the FP64 sum
    np.testing.assert_allclose(d2_g, d2, rtol=4e-16, atol=0)


@pytest.mark.parametrize("case", ["random", "lattice", "duplicates", "surface"])
def test_kdtree_route_equals_exhaustive(case):
    if case == "random":
        ref, qry = _cloud(9, 5000), _cloud(10, 700)
    elif case == "lattice":
        ref = synth.lattice_points((9, 8, 7))
        qry = ref[::3]
    elif case == "duplicates":
        base = _cloud(11, 300)
        ref = np.concatenate([base, base, base[:50]])
        qry = base[:100]
    else:
        ref = synth.surface_pair(12, n=6000).target
        qry = ref[::7]
    for k in (1, 10, 27):
        a = oracle.knn(ref, qry, k)
        b = oracle.knn(ref, qry, k, method="kdtree")
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_radius_matches_library_and_is_sorted():
    ref = _cloud(13, 4000)
    qry = _cloud(14, 300)
    r = 0.15
    off, idx, d2 = oracle.radius(ref, qry, r)
    tree = cKDTree(ref.astype(np.float64))
    rr = float(np.float32(r))
    for q in range(len(qry)):
        row = idx[off[q]:off[q + 1]]
        rd = d2[off[q]:off[q + 1]]
        lib = tree.query_ball_point(qry[q].astype(np.float64), rr)
        # membership may differ only for points on the sphere boundary
        dl = ((ref[lib].astype(np.float64) - qry[q]) ** 2).sum(1)
        strict = set(np.asarray(lib)[np.abs(dl - rr * rr) > 1e-12])
        assert strict <= set(row.tolist())
        keys = list(zip(rd.tolist(), row.tolist()))
        assert keys == sorted(keys)
        assert np.all(rd <= rr * rr)


def test_radius_lattice_exact_counts():
    pts = synth.lattice_points((5, 5, 5))
    # inclusive boundary: r = 1 around the centre gives self + 6 face neighbours
    off, idx, d2 = oracle.radius(pts, pts[62:63], 1.0)
    assert idx.tolist() == [62, 37, 57, 61, 63, 67, 87]
    off, idx, d2 = oracle.radius(pts, pts[62:63], 0.999)
    assert idx.tolist() == [62]
    off, idx, d2 = oracle.radius(pts, pts[62:63], 0.0)
    assert idx.tolist() == [62]


def test_radius_empty_rows():
    ref = _cloud(15, 100)
    qry = ref[:5] + 10.0
    off, idx, d2 = oracle.radius(ref, qry, 0.5)
    assert off.tolist() == [0] * 6 and idx.size == 0


def test_hybrid_query_matches_library_bounded_search():
    ref = _cloud(20, 4000)
    qry = _cloud(21, 300)
    k, r = 12, 0.12
    idx, d2 = oracle.knn_hybrid(ref, qry, k, r)
    rr = float(np.float32(r))
    dd, ii = cKDTree(ref.astype(np.float64)).query(qry.astype(np.float64), k,
                                                    distance_upper_bound=rr * (1 + 1e-12))
    found = np.isfinite(dd)
    assert np.array_equal(idx[found], ii[found])
    assert np.all(idx[~found] == -1) and np.all(np.isinf(d2[~found]))
    np.testing.assert_allclose(d2[found], dd[found] ** 2, rtol=1e-12)


def test_hybrid_query_is_knn_truncated_by_radius():
    pts = synth.lattice_points((5, 5, 5))
    idx, d2 = oracle.knn_hybrid(pts, pts[62:63], 27, 1.0)
    full, fd = oracle.knn(pts, pts[62:63], 27)
    assert idx[0, :7].tolist() == full[0, :7].tolist()  # self + 6 face neighbours at d2 <= 1
    assert np.all(idx[0, 7:] == -1)
