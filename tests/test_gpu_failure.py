"""Failure paths on the GPU, made without faulting it: a bounded device wait
that runs out reports CIL_ERR_TIMEOUT through the error word and leaves the
context usable; a failed workspace allocation reports CIL_ERR_NOMEM and the
next call succeeds; non-finite inputs report CIL_ERR_NONFINITE."""
import numpy as np
import pytest
import torch

import paper_1807_00399_gb300 as cil

pytestmark = pytest.mark.gpu
CODE = {name: code for code, name in cil.STATUS.items()}


def _cloud(n=2000, seed=0):
    return torch.from_numpy(np.random.default_rng(seed).uniform(-1, 1, (n, 3)).astype(np.float32)).cuda()


def test_bounded_wait_times_out_and_the_context_survives():
    L = cil.lib()
    assert L.cil_check_bounded_wait(4096, None) == CODE["CIL_ERR_TIMEOUT"]
    assert cil.sync_status() == 0  # the word was read and cleared
    x = _cloud()
    idx, d2 = cil.knn(x, x, 8)
    torch.cuda.synchronize()
    assert (idx[:, 0].cpu().numpy() == np.arange(2000)).all()


def test_allocation_failure_then_recovery():
    L = cil.lib()
    x = _cloud(seed=1)
    L.cil_test_fail_next_allocations(1)
    with pytest.raises(cil.CilError) as e:
        cil.knn(x, x, 8)
    assert e.value.status == CODE["CIL_ERR_NOMEM"]
    idx, _ = cil.knn(x, x, 8)
    torch.cuda.synchronize()
    assert (idx[:, 0].cpu().numpy() == np.arange(2000)).all()
    L.cil_test_fail_next_allocations(0)


def test_nonfinite_input_is_reported():
    x = _cloud(seed=2)
    x[17, 1] = float("nan")
    cil.estimate_normals(x, 8, (0.0, 0.0, 5.0))
    torch.cuda.synchronize()
    assert cil.sync_status() == CODE["CIL_ERR_NONFINITE"]
    assert cil.sync_status() == 0  # read and cleared
