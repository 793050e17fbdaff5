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
