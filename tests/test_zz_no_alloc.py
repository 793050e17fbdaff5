"""cil_knn_noalloc: the k-nearest-neighbour entry point for callers that cannot
call cudaMalloc (plugins inside a framework that owns all device memory,
real-time loops, code without dynamic allocation after start-up).  It runs on
scratch held in a fixed array inside the library; here it must return what
cil_knn returns, on two calls in a row (the second reuses the array the first
left behind), and refuse sizes beyond its limit.

Collected last on purpose, so a run that stops at the first failure has run
every other test before this one; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

import paper_1807_00399_gb300 as cil
from paper_1807_00399_gb300 import synth

pytestmark = pytest.mark.gpu

MAX_POINTS = 32768
CAPACITY = 4  # CIL_ERR_CAPACITY


def _entry():
    L = cil.lib()
    f = L.cil_knn_noalloc
    P = ctypes.c_void_p
    f.argtypes = [P, ctypes.c_int64, P, ctypes.c_int64, ctypes.c_int, P, P, P]
    f.restype = ctypes.c_int
    return f


def _noalloc(ref, qry, k):
    nq = qry.shape[0]
    idx = torch.full((nq, k), -7, dtype=torch.int32, device="cuda")
    d2 = torch.full((nq, k), -1.0, dtype=torch.float32, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = _entry()(ctypes.c_void_p(ref.data_ptr()), ref.shape[0], ctypes.c_void_p(qry.data_ptr()), nq,
                  k, ctypes.c_void_p(idx.data_ptr()), ctypes.c_void_p(d2.data_ptr()), stream)
    return st, idx, d2


def test_noalloc_matches_knn_on_two_calls():
    cases = [
        (synth.surface_pair(21, n=20_000).target, None, 10),  # self-query
        (synth.surface_pair(22, n=MAX_POINTS).target, synth.surface_pair(23, n=5_001).source, 16),
    ]
    for ref_np, qry_np, k in cases:
        ref = torch.from_numpy(ref_np).cuda()
        qry = ref if qry_np is None else torch.from_numpy(qry_np).cuda()
        st, idx, d2 = _noalloc(ref, qry, k)
        assert st == 0, cil.STATUS.get(st, st)
        ref_idx, ref_d2 = cil.knn(ref, qry, k)
        torch.cuda.synchronize()
        assert torch.equal(idx, ref_idx)
        np.testing.assert_allclose(d2.cpu().numpy(), ref_d2.cpu().numpy(), rtol=1e-6, atol=0)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    big = torch.zeros((MAX_POINTS + 1, 3), dtype=torch.float32, device="cuda")
    small = torch.zeros((10, 3), dtype=torch.float32, device="cuda")
    st, _, _ = _noalloc(big, small, 4)
    assert st == CAPACITY
    st, _, _ = _noalloc(small, big, 4)
    assert st == CAPACITY


def test_noalloc_largest_case_and_empty_reference():
    # the case that reserves the most scratch: both sets at the limit, k at
    # its maximum, queries distinct from the reference points
    ref = torch.from_numpy(synth.surface_pair(24, n=MAX_POINTS).target).cuda()
    qry = torch.from_numpy(synth.surface_pair(25, n=MAX_POINTS).source).cuda()
    for _ in range(2):
        st, idx, d2 = _noalloc(ref, qry, 32)
        assert st == 0, cil.STATUS.get(st, st)
        ref_idx, ref_d2 = cil.knn(ref, qry, 32)
        torch.cuda.synchronize()
        assert torch.equal(idx, ref_idx)
        np.testing.assert_allclose(d2.cpu().numpy(), ref_d2.cpu().numpy(), rtol=1e-6, atol=0)
    # no reference points: every row is padding (-1, +inf), as cil_knn gives
    empty = torch.zeros((0, 3), dtype=torch.float32, device="cuda")
    st, idx, d2 = _noalloc(empty, qry[:100], 5)
    assert st == 0
    ref_idx, ref_d2 = cil.knn(empty, qry[:100], 5)
    torch.cuda.synchronize()
    assert torch.equal(idx, ref_idx) and torch.equal(d2, ref_d2)
    assert bool((idx == -1).all()) and bool(torch.isinf(d2).all())


def test_noalloc_takes_no_workspace_allocation():
    """An armed allocation failure stays pending across the call: it takes
    no memory from the library's pool (the next allocating call fails)."""
    L = cil.lib()
    ref = torch.from_numpy(synth.surface_pair(26, n=4_000).target).cuda()
    try:
        L.cil_test_fail_next_allocations(1)
        st, idx, _ = _noalloc(ref, ref, 8)
        assert st == 0
        with pytest.raises(cil.CilError) as e:
            cil.knn(ref, ref, 8)
        assert e.value.status == 7  # CIL_ERR_NOMEM: the armed failure was still pending
    finally:
        L.cil_test_fail_next_allocations(0)
    ref_idx, _ = cil.knn(ref, ref, 8)
    torch.cuda.synchronize()
    assert torch.equal(idx, ref_idx)
