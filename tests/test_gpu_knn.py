"""kNN parity: libcil (cil_knn, sm_103a) against the FP64 exhaustive oracle.

Bar: squared distances within 1e-6 relative (FP32 d2 from exactly rounded
differences errs by < 2.4e-7); indices bit-exact outside oracle tie groups
(distances within 1e-6 relative), inside them the distances agree and every
index is a genuine point at that distance (see tests/parity.py)."""
import numpy as np
import pytest
import torch

import oracle
import paper_1807_00399_gb300 as cil
from paper_1807_00399_gb300 import synth
from parity import check_knn_rows

pytestmark = pytest.mark.gpu


def _gpu_knn(ref, qry, k, self_query=False, **kw):
    r = torch.from_numpy(np.ascontiguousarray(ref)).cuda()
    q = r if self_query else torch.from_numpy(np.ascontiguousarray(qry)).cuda()
    idx, d2 = cil.knn(r, q, k, **kw)
    torch.cuda.synchronize()
    assert cil.sync_status() == 0
    return idx.cpu().numpy(), d2.cpu().numpy()


def _check(ref, qry, k, self_query=False, rows=None, **kw):
    gi, gd = _gpu_knn(ref, qry, k, self_query, **kw)
    q = ref if self_query else qry
    if rows is not None:
        gi, gd, q = gi[rows], gd[rows], q[rows]
    oi, od = oracle.knn(ref, q, k + 1, method="kdtree" if len(ref) > 50000 else "brute")
    return check_knn_rows(ref, q, gi, gd, oi, od, k)


def _cube(seed, n, scale=1.0):
    return (np.random.default_rng(seed).uniform(-1, 1, (n, 3)) * scale).astype(np.float32)


@pytest.mark.parametrize("k", [1, 4, 10, 16, 32])
def test_surface_self_query(k):
    p = synth.surface_pair(0, n=10_000)
    _check(p.target, None, k, self_query=True)


def test_external_queries_ragged_sizes():
    ref = _cube(1, 3001)
    qry = _cube(2, 777, 1.2)  # some queries outside the reference box
    _check(ref, qry, 10)
    _check(ref, qry, 7)


def test_lattice_exact_ties():
    ref = synth.lattice_points((9, 8, 7))
    gi, gd = _gpu_knn(ref, None, 27, self_query=True)
    oi, od = oracle.knn(ref, ref, 27)
    # integer lattice: FP32 and FP64 distances are exact, so ties are exact
    # and the (d2, index) order must match bit for bit
    assert np.array_equal(gi, oi)
    assert np.array_equal(gd.astype(np.float64), od)


@pytest.mark.parametrize("k", [10, 24])  # register list / shared-memory heap
def test_duplicates_and_coincident_points(k):
    base = _cube(3, 400)
    ref = np.concatenate([base, base, base[:123]])
    _check(ref, None, k, self_query=True)
    same = np.zeros((50, 3), np.float32)
    gi, gd = _gpu_knn(same, None, k, self_query=True)
    assert np.all(gd == 0) and np.array_equal(np.sort(gi, 1), np.tile(np.arange(k), (50, 1)))
    assert np.array_equal(gi, np.tile(np.arange(k), (50, 1)))


@pytest.mark.parametrize("k", [8, 20])
def test_k_larger_than_reference_pads(k):
    ref = _cube(4, 5)
    gi, gd = _gpu_knn(ref, _cube(5, 9), k)
    oi, od = oracle.knn(ref, _cube(5, 9), k)
    assert np.array_equal(gi, oi)
    assert np.all(np.isinf(gd[:, 5:])) and np.all(gi[:, 5:] == -1)


def test_single_point_and_empty_reference():
    ref = _cube(6, 1)
    gi, gd = _gpu_knn(ref, _cube(7, 33), 3)
    assert np.all(gi[:, 0] == 0) and np.all(gi[:, 1:] == -1)
    empty = np.zeros((0, 3), np.float32)
    r = torch.zeros((0, 3), dtype=torch.float32, device="cuda")
    q = torch.from_numpy(_cube(8, 17)).cuda()
    idx, d2 = cil.knn(r, q, 4)
    torch.cuda.synchronize()
    assert (idx.cpu().numpy() == -1).all() and np.isinf(d2.cpu().numpy()).all()
    assert empty.shape[0] == 0


def test_far_outliers_and_mixed_density():
    rng = np.random.default_rng(9)
    dense = rng.normal(0, 0.01, (4000, 3))
    sparse = rng.uniform(-50, 50, (200, 3))
    ref = np.concatenate([dense, sparse]).astype(np.float32)
    qry = np.concatenate([rng.normal(0, 0.02, (300, 3)), rng.uniform(-200, 200, (100, 3))]).astype(
        np.float32)
    _check(ref, qry, 10)
    _check(ref, None, 10, self_query=True)
    _check(ref, qry, 32)
    _check(ref, None, 32, self_query=True)


@pytest.mark.parametrize("kw", [{"cell_scale": 0.25}, {"cell_scale": 4.0}, {"cell_size": 1e-4},
                                {"cell_size": 10.0}, {"block": 64}, {"block": 256}])
def test_cell_size_and_block_do_not_change_results(kw):
    p = synth.surface_pair(10, n=5003)
    _check(p.target, None, 10, self_query=True, **kw)
    _check(p.target, p.source, 10, **kw)
    _check(p.target, p.source, 30, **kw)


def test_deterministic():
    p = synth.surface_pair(11, n=20_000)
    a = _gpu_knn(p.target, p.source, 10)
    b = _gpu_knn(p.target, p.source, 10)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_depth_frame_full_size_sampled():
    p = synth.depth_frame_pair(0)
    rows = np.random.default_rng(12).choice(len(p.target), 2000, replace=False)
    _check(p.target, None, 10, self_query=True, rows=rows)
    _check(p.target, p.source, 10, rows=rows[:1000])


def test_lidar_full_size_sampled():
    p = synth.lidar_sweep_pair(0)
    rows = np.random.default_rng(13).choice(len(p.target), 2000, replace=False)
    _check(p.target, None, 16, self_query=True, rows=rows)


@pytest.mark.parametrize("topk", [1, 2, 3])
def test_topk_layouts_give_bitwise_equal_results(topk):
    """The top-k layout (per-query register list, per-query shared-memory
    heap, or the warp-staged search that scans a shared set of points per 32
    queries and falls back to the per-query search where it cannot prove the
    k-th distance) changes the speed only: results are bitwise those of the
    default, on clustered and outlier-heavy clouds, with exact ties."""
    rng = np.random.default_rng(31)
    dense = rng.normal(0, 0.01, (6000, 3))
    sparse = rng.uniform(-50, 50, (300, 3))
    clouds = [synth.surface_pair(12, n=20_000).target,
              np.concatenate([dense, sparse]).astype(np.float32),
              synth.lattice_points((20, 20, 20))]
    for ref in clouds:
        qry = np.concatenate([ref[::3] + np.float32(1e-3), ref[:50] + np.float32(70.0)])
        for k in (1, 4, 10, 16, 32):
            for q, self_query in ((None, True), (qry, False)):
                a = _gpu_knn(ref, q, k, self_query)
                b = _gpu_knn(ref, q, k, self_query, topk=topk)
                assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]), (k, self_query)
    _check(clouds[0], None, 10, self_query=True, topk=topk)
    _check(clouds[1], qry, 10, topk=topk)


def test_staged_normals_and_batch_bitwise_equal():
    p = synth.surface_pair(13, n=30_000)
    x = torch.from_numpy(p.target).cuda()
    for k in (3, 10, 30):
        n0, c0 = cil.estimate_normals(x, k, p.viewpoint)
        n3, c3 = cil.estimate_normals(x, k, p.viewpoint, topk=3)
        torch.cuda.synchronize()
        assert torch.equal(n0, n3) and torch.equal(c0, c3)
    sizes = np.array([2000, 3500, 9000, 700, 12000], np.int64)
    src, dst, _ = synth.surface_batch_torch(5, sizes)
    out = []
    for topk in (0, 3):
        h = cil.Batch(sizes, sizes, k=10, iters=5, max_corr_dist=0.1, topk=topk)
        nrm = torch.empty_like(dst)
        T, _ = h.run(src, dst, normals_out=nrm)
        torch.cuda.synchronize()
        out.append((T.clone(), nrm.clone()))
        h.close()
    assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])


def test_reference_permutation_equivariant():
    """Permuting the reference points permutes the returned indices and
    leaves the distances unchanged: with the reference points in another
    order (another Morton-sort tie order inside each cell, another index
    tie-break), every row's d2 is the same bit for bit and, in rows without
    equal distances, the indices map through the permutation."""
    ref = synth.surface_pair(21, n=20_000).target
    qry = _cube(22, 3_000, scale=1.2)
    perm = np.random.default_rng(23).permutation(len(ref))
    gi, gd = _gpu_knn(ref, qry, 10)
    pi, pd = _gpu_knn(ref[perm], qry, 10)
    assert np.array_equal(gd, pd)
    no_ties = np.all(np.diff(gd, axis=1) > 0, axis=1)
    assert no_ties.mean() > 0.9
    assert np.array_equal(perm[pi[no_ties]], gi[no_ties])
