"""FP64 oracle for connected-component segmentation on the k-NN graph (Sec. 3:
connected components under a point-wise similarity; smooth segments as in
Sec. 4's apartment-scale test, k = 30 and a normal-angle threshold).

TEST INFRASTRUCTURE.  Only the test-suite and the bench's CPU leg use this
module; the product library never imports it, and it imports nothing from the
product library.

Steps, in the order of the method:
1. the k nearest neighbours of every point (the oracle's exhaustive / kd-tree
   k-NN, FP64 distances, (d^2, index) order, the point itself included);
2. an undirected edge {i, j} for every j among the k nearest of i (so the
   graph is the symmetric closure of the directed k-NN relation), kept when
   the similarity holds: the normals' angle is at most theta (oriented
   normals, n_i . n_j >= cos theta) and, when a radius r > 0 is given, the
   points are at most r apart;
3. connected components (scipy.sparse.csgraph.connected_components, a
   library routine), each labelled by its smallest point index.

Readings: the similarity tests are integer decisions taken from floating
point, so they are evaluated in FP32 with a fixed operation order, the same
one the library uses: dot = (nx mx + ny my) + nz mz and d^2 = (dx dx + dy dy)
+ dz dz, each product and sum rounded to nearest (no fused multiply-add), on
the FP32 inputs; cos theta and r^2 are rounded to FP32 first.  A point whose
normal is not finite has no edge.  Where the k-th neighbour ties (within
1e-6 relative) with the (k+1)-th, or a similarity value lies within 1e-6 of
its threshold, the graph is not fixed by the definition alone; `bounds`
returns the two partitions with every such edge removed and added, between
which any correct result lies.
"""
from __future__ import annotations

import numpy as np


def _f32(x):
    return np.asarray(x, np.float32)


def similarity(P, N, i, j, cos_t, r2):
    """FP32 similarity values and the boolean decision for edges (i, j)."""
    P = _f32(P)
    N = _f32(N)
    ni, nj = N[i], N[j]
    dot = (ni[:, 0] * nj[:, 0] + ni[:, 1] * nj[:, 1]) + ni[:, 2] * nj[:, 2]
    ok = np.isfinite(dot) & (dot >= np.float32(cos_t))
    d = P[i] - P[j]
    d2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
    if r2 > 0:
        ok &= d2 <= np.float32(r2)
    return dot, d2, ok


def canonical(labels):
    """Relabel components by their smallest member index."""
    n = len(labels)
    first = np.full(labels.max() + 1 if n else 0, n, np.int64)
    np.minimum.at(first, labels, np.arange(n))
    return first[labels].astype(np.int32)


def components(n, i, j):
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components
    A = coo_matrix((np.ones(len(i), np.int8), (i, j)), shape=(n, n))
    _, lab = connected_components(A, directed=False)
    return canonical(lab)


def knn_edges(P, k, method="kdtree"):
    import oracle
    idx, d2 = oracle.knn(_f32(P), _f32(P), k + 1, method=method)
    return idx, d2


def segment(P, N, k: int = 30, theta: float = 2.8, radius: float = 0.0, method: str = "kdtree"):
    """Labels (int32, smallest index of the component) and the number of
    components."""
    P = _f32(P)
    n = len(P)
    idx, _ = knn_edges(P, k, method)
    idx = idx[:, :k]
    i = np.repeat(np.arange(n), k)
    j = idx.ravel().astype(np.int64)
    keep = (j >= 0) & (j != i)
    i, j = i[keep], j[keep]
    cos_t = np.float32(np.cos(np.float64(np.float32(theta))))
    r2 = float(np.float32(radius)) ** 2 if radius > 0 else 0.0
    _, _, ok = similarity(P, N, i, j, cos_t, np.float32(r2))
    lab = components(n, i[ok], j[ok])
    return lab, int(np.sum(lab == np.arange(n)))


def bounds(P, N, k: int = 30, theta: float = 2.8, radius: float = 0.0, rel: float = 1e-6,
           eps=None):
    """(lower, upper) partitions: without / with every edge the definition
    leaves open (k-th-rank distance ties and similarity values within `rel` of
    their thresholds).  `eps` (optional, per point, radians): how far the
    normal a compared result used may lie from N; since unit vectors turned by
    angles a and b change their dot product by at most a + b, an edge is also
    open where |n_i . n_j - cos theta| <= rel + eps_i + eps_j, and wherever
    eps_i + eps_j >= 2 (the dot product of unit vectors spans [-1, 1], so the
    edge is then undecided whatever N holds, a non-finite normal included)."""
    P = _f32(P)
    n = len(P)
    idx, d2 = knn_edges(P, k)
    i = np.repeat(np.arange(n), k + 1).reshape(n, k + 1)
    # rank-k candidates tied with rank k+1 (either may be chosen)
    tie = np.abs(d2[:, k - 1] - d2[:, k]) <= rel * np.maximum(d2[:, k], 1e-300)
    cand_i = i.ravel()
    cand_j = idx.ravel().astype(np.int64)
    rank = np.tile(np.arange(k + 1), n)
    tied_row = np.repeat(tie, k + 1)
    # rows: ranks < k are edges; rank k-1 and k are open where tied; rank k
    # (the (k+1)-th) is not an edge otherwise
    sure = (rank < k) & ~(tied_row & (rank == k - 1))
    maybe = tied_row & (rank >= k - 1)
    valid = (cand_j >= 0) & (cand_j != cand_i)
    cos_t = np.float32(np.cos(np.float64(np.float32(theta))))
    r2 = np.float32(float(np.float32(radius)) ** 2) if radius > 0 else np.float32(0)
    dot, dd2, ok = similarity(P, N, cand_i, cand_j, cos_t, r2)
    slack = rel if eps is None else rel + np.asarray(eps, np.float64)[cand_i] + \
        np.asarray(eps, np.float64)[np.maximum(cand_j, 0)]
    near = (np.abs(dot.astype(np.float64) - float(cos_t)) <= slack) | (slack >= 2.0 + rel)
    if radius > 0:
        near |= np.abs(dd2.astype(np.float64) - float(r2)) <= rel * float(r2)
    lo = valid & sure & ok & ~near
    hi = valid & (sure | maybe) & (ok | near)
    return (components(n, cand_i[lo], cand_j[lo]), components(n, cand_i[hi], cand_j[hi]))


def consistent(labels, lower, upper) -> bool:
    """True when `labels` is a partition between `lower` (finer) and `upper`
    (coarser): every lower component lies inside one labels component, and
    every labels component inside one upper component."""
    labels = np.asarray(labels)
    # each lower component maps to one label
    a = np.unique(np.stack([lower, labels], 1), axis=0)
    if len(np.unique(a[:, 0])) != len(a):
        return False
    b = np.unique(np.stack([labels, upper], 1), axis=0)
    return len(np.unique(b[:, 0])) == len(b)
