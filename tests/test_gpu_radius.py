"""Radius search parity: libcil (cil_radius_search) against the FP64
exhaustive oracle.  Membership must match except for points within 1e-6
relative of the sphere (|d2 - r^2| <= 1e-6 r^2: FP32 vs FP64 rounding); rows
ascend by (d2, index); d2 within 1e-6 relative."""
import numpy as np
import pytest
import torch

import oracle
import paper_1807_00399_gb300 as cil
from paper_1807_00399_gb300 import synth
from parity import rel_close

pytestmark = pytest.mark.gpu


def _gpu_radius(ref, qry, r, capacity=None):
    R = torch.from_numpy(np.ascontiguousarray(ref)).cuda()
    Q = R if qry is None else torch.from_numpy(np.ascontiguousarray(qry)).cuda()
    off, idx, d2 = cil.radius_search(R, Q, r, capacity=capacity)
    return off.cpu().numpy(), idx.cpu().numpy(), d2.cpu().numpy()


def _check(ref, qry, r, rows=None):
    go, gi, gd = _gpu_radius(ref, qry, r)
    q = ref if qry is None else qry
    sel = np.arange(len(q)) if rows is None else rows
    oo, oi, od = oracle.radius(ref, q[sel], r)
    r2 = float(np.float32(r)) ** 2
    for t, row in enumerate(sel):
        g_idx = gi[go[row]:go[row + 1]]
        g_d2 = gd[go[row]:go[row + 1]].astype(np.float64)
        o_idx = oi[oo[t]:oo[t + 1]]
        o_d2 = od[oo[t]:oo[t + 1]]
        keys = list(zip(g_d2.tolist(), g_idx.tolist()))
        assert keys == sorted(keys), f"row {row} not sorted"
        assert len(set(g_idx.tolist())) == len(g_idx)
        P = ref[g_idx].astype(np.float64)
        true = ((P - q[row].astype(np.float64)) ** 2).sum(1)
        assert rel_close(g_d2, true).all()
        bnd_o = np.abs(o_d2 - r2) <= 1e-6 * r2
        bnd_g = np.abs(true - r2) <= 1e-6 * r2
        a = set(o_idx[~bnd_o].tolist())
        b = set(g_idx[~bnd_g].tolist())
        assert a == b, f"row {row}: membership differs ({len(a ^ b)} points)"


def test_random_cube():
    rng = np.random.default_rng(0)
    ref = rng.uniform(-1, 1, (5000, 3)).astype(np.float32)
    qry = rng.uniform(-1.2, 1.2, (613, 3)).astype(np.float32)
    _check(ref, qry, 0.15)
    _check(ref, None, 0.1, rows=np.arange(0, 5000, 7))


def test_lattice_exact():
    pts = synth.lattice_points((5, 5, 5))
    go, gi, gd = _gpu_radius(pts, pts[62:63], 1.0)
    assert gi.tolist() == [62, 37, 57, 61, 63, 67, 87] and go.tolist() == [0, 7]
    go, gi, gd = _gpu_radius(pts, pts[62:63], 0.0)
    assert gi.tolist() == [62]


def test_capacity_and_empty_rows():
    rng = np.random.default_rng(1)
    ref = rng.uniform(-1, 1, (2000, 3)).astype(np.float32)
    R = torch.from_numpy(ref).cuda()
    with pytest.raises(cil.CilError) as e:
        cil.radius_search(R, R, 0.3, capacity=10)
    assert e.value.status == 4
    far = torch.from_numpy(ref[:50] + 100).cuda()
    off, idx, d2 = cil.radius_search(R, far, 0.5)
    assert off.cpu().numpy().tolist() == [0] * 51 and idx.numel() == 0


def test_long_rows_sorted_in_global_memory():
    # a dense blob puts > 4096 neighbours in one row (the global-memory sort)
    rng = np.random.default_rng(2)
    ref = rng.normal(0, 0.05, (20000, 3)).astype(np.float32)
    _check(ref, ref[:40], 0.2)


def test_lidar_sampled():
    p = synth.lidar_sweep_pair(0)
    rows = np.random.default_rng(3).choice(len(p.target), 300, replace=False)
    _check(p.target, None, 0.5, rows=rows)


@pytest.mark.parametrize("r", [1.0, 2.9, 4.0, 5.0, 6.0, 7.0, 8.5])
def test_lattice_rows_across_sort_paths(r):
    """Integer lattice (exact distances, many exact ties, so the index order
    inside equal distances is checked bit for bit) with row lengths from a
    few to about three thousand: rows up to 1024 keys are sorted by their
    warp in shared memory (bucket sort), longer ones by a block each (bitonic
    network in shared memory)."""
    pts = synth.lattice_points((16, 16, 16))
    go, gi, gd = _gpu_radius(pts, None, r)
    oo, oi, od = oracle.radius(pts, pts, r)
    assert np.array_equal(go, oo) and np.array_equal(gi, oi)
    assert np.array_equal(gd.astype(np.float64), od)
    lengths = np.diff(go)
    assert lengths.max() >= 7
    if r >= 7.0:
        assert lengths.max() > 1024


@pytest.mark.parametrize("scale", [0.5, 0.7, 2.0])
def test_cell_size_does_not_change_results(scale):
    """The cell edge of the search (r by default) is a speed knob only."""
    p = synth.lidar_sweep_pair(1)
    R = torch.from_numpy(p.target).cuda()
    a = cil.radius_search(R, R, 0.5)
    b = cil.radius_search(R, R, 0.5, cell_scale=scale)
    torch.cuda.synchronize()
    for x, y in zip(a, b):
        assert torch.equal(x, y)
