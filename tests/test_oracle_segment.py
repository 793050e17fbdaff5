"""Pins of the segmentation oracle (oracle/segment.py): breadth-first search
over brute-force k-NN edges on small inputs, separated clusters, a normal
flip that must cut, permutation equivariance and the ambiguity bounds."""
import numpy as np

from oracle import segment as sg


def _bfs_labels(P, N, k, theta, radius):
    P64 = P.astype(np.float64)
    n = len(P)
    D = ((P64[:, None, :] - P64[None, :, :]) ** 2).sum(-1)
    order = np.lexsort((np.tile(np.arange(n), (n, 1)), D), axis=1)[:, :k]
    cos_t = np.float32(np.cos(np.float64(np.float32(theta))))
    r2 = np.float32(float(np.float32(radius)) ** 2) if radius > 0 else np.float32(0)
    adj = [set() for _ in range(n)]
    for i in range(n):
        for j in order[i]:
            if j == i:
                continue
            a, b = N[i].astype(np.float32), N[j].astype(np.float32)
            dot = (a[0] * b[0] + a[1] * b[1]) + a[2] * b[2]
            dv = (P[i] - P[j]).astype(np.float32)
            d2 = (dv[0] * dv[0] + dv[1] * dv[1]) + dv[2] * dv[2]
            if np.isfinite(dot) and dot >= cos_t and (radius <= 0 or d2 <= r2):
                adj[i].add(int(j))
                adj[int(j)].add(i)
    lab = np.full(n, -1, np.int64)
    for s in range(n):
        if lab[s] >= 0:
            continue
        stack, comp = [s], []
        lab[s] = s
        while stack:
            u = stack.pop()
            comp.append(u)
            for v in adj[u]:
                if lab[v] < 0:
                    lab[v] = s
                    stack.append(v)
        lab[comp] = min(comp)
    return lab.astype(np.int32)


def _cloud(seed, n=300):
    rng = np.random.default_rng(seed)
    P = rng.uniform(-1, 1, (n, 3)).astype(np.float32)
    N = rng.normal(size=(n, 3))
    N /= np.linalg.norm(N, axis=1, keepdims=True)
    return P, N.astype(np.float32)


def test_matches_breadth_first_search():
    for seed, k, theta, r in [(0, 6, 1.2, 0.0), (1, 8, 2.8, 0.0), (2, 5, 2.0, 0.35)]:
        P, N = _cloud(seed)
        lab, nc = sg.segment(P, N, k=k, theta=theta, radius=r, method="brute")
        ref = _bfs_labels(P, N, k, theta, r)
        np.testing.assert_array_equal(lab, ref)
        assert nc == len(np.unique(ref))


def test_separated_clusters():
    rng = np.random.default_rng(3)
    A = rng.normal(0, 0.05, (200, 3))
    B = rng.normal(0, 0.05, (150, 3)) + np.array([5.0, 0, 0])
    P = np.concatenate([A, B]).astype(np.float32)
    N = np.tile(np.float32([0, 0, 1]), (350, 1))
    lab, nc = sg.segment(P, N, k=10, theta=0.5)
    assert nc == 2
    np.testing.assert_array_equal(lab[:200], 0)
    np.testing.assert_array_equal(lab[200:], 200)


def test_normal_flip_cuts_a_plane():
    g = np.stack(np.meshgrid(np.arange(20), np.arange(20)), -1).reshape(-1, 2).astype(np.float32)
    P = np.column_stack([g, np.zeros(len(g), np.float32)]) * np.float32(0.1)
    N = np.tile(np.float32([0, 0, 1]), (len(P), 1))
    N[P[:, 0] > 0.95] *= -1  # right half points the other way
    lab, nc = sg.segment(P, N, k=9, theta=1.0)
    assert nc == 2
    assert len(np.unique(lab[P[:, 0] > 0.95])) == 1 and len(np.unique(lab[P[:, 0] < 0.95])) == 1


def test_permutation_equivariance():
    P, N = _cloud(4, 400)
    lab, _ = sg.segment(P, N, k=7, theta=1.5)
    perm = np.random.default_rng(5).permutation(len(P))
    lab2, _ = sg.segment(P[perm], N[perm], k=7, theta=1.5)
    # same partition: points together before are together after
    same = lab[:, None] == lab[None, :]
    same2 = lab2[:, None] == lab2[None, :]
    np.testing.assert_array_equal(same[np.ix_(perm, perm)], same2)


def test_bounds_bracket_the_definition():
    P, N = _cloud(6, 500)
    lab, _ = sg.segment(P, N, k=8, theta=1.8)
    lo, hi = sg.bounds(P, N, k=8, theta=1.8)
    assert sg.consistent(lab, lo, hi)
    # a partition merging two upper components is rejected
    if len(np.unique(hi)) > 1:
        bad = hi.copy()
        u = np.unique(hi)
        bad[bad == u[1]] = u[0]
        assert not sg.consistent(bad, lo, hi)


def test_bounds_with_uncertain_normals():
    P, _ = _cloud(7, 400)
    N = np.tile(np.float32([0, 0, 1]), (400, 1))
    # every normal fully uncertain: nothing is certain to join, everything may
    lo, hi = sg.bounds(P, N, k=6, theta=0.5, eps=np.full(400, 3.0))
    np.testing.assert_array_equal(lo, np.arange(400))
    np.testing.assert_array_equal(hi, _bfs_labels(P, N, 6, 0.5, 0.0))
    # no uncertainty: the plain bounds
    a = sg.bounds(P, N, k=6, theta=0.5)
    b = sg.bounds(P, N, k=6, theta=0.5, eps=np.zeros(400))
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])
