"""Shared checks comparing library results with the oracle (not a test file).

Tolerances (derived from the arithmetic; restated in the tests that use them):
* squared distances: the library forms each coordinate difference exactly
  rounded and sums three squares in FP32, so its d2 carries a relative error
  below 4 * 2^-24 ~ 2.4e-7; we allow 1e-6 relative.
* neighbour indices: bit-exact, except inside a tie group -- oracle distances
  within 1e-6 relative of each other (including the group straddling rank
  k / k+1), where only the set of distances must agree and every returned
  index must be a genuine point at that distance.
"""
from __future__ import annotations

import numpy as np

REL = 1e-6


def rel_close(a, b, rel=REL, tiny=1e-30):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    both_inf = np.isinf(a) & np.isinf(b)
    return both_inf | (np.abs(a - b) <= rel * np.maximum(np.abs(b), tiny))


def check_knn_rows(ref, qry_pts, gpu_idx, gpu_d2, ora_idx_ext, ora_d2_ext, k):
    """ora_*_ext hold k+1 oracle neighbours per row (to see ties across the
    rank-k boundary).  Raises AssertionError with a description on mismatch.
    Returns the number of rows whose indices differed inside tie groups."""
    gpu_idx = np.asarray(gpu_idx)
    gpu_d2 = np.asarray(gpu_d2, np.float64)
    oi = ora_idx_ext[:, :k]
    od = ora_d2_ext[:, :k]
    # 1. distances agree rank by rank
    ok = rel_close(gpu_d2, od)
    if not ok.all():
        r, c = np.argwhere(~ok)[0]
        raise AssertionError(f"d2 mismatch row {r} rank {c}: gpu {gpu_d2[r, c]!r} oracle {od[r, c]!r}")
    # 2. padding agrees
    pad_o = oi < 0
    if not np.array_equal(pad_o, gpu_idx < 0):
        raise AssertionError("padding (-1) positions differ")
    # 3. every returned index is a genuine point at its reported distance
    valid = gpu_idx >= 0
    rr, cc = np.nonzero(valid)
    P = ref[gpu_idx[rr, cc]].astype(np.float64)
    Q = qry_pts[rr].astype(np.float64)
    true_d2 = ((P - Q) ** 2).sum(1)
    good = rel_close(gpu_d2[rr, cc], true_d2)
    if not good.all():
        j = np.argmin(good)
        raise AssertionError(f"index {gpu_idx[rr[j], cc[j]]} is not at distance {gpu_d2[rr[j], cc[j]]}")
    # 4. indices equal outside tie groups
    d_ext = np.asarray(ora_d2_ext, np.float64)
    tie = np.zeros_like(od, dtype=bool)
    for c in range(k):
        for nb in (c - 1, c + 1):
            if 0 <= nb < d_ext.shape[1]:
                tie[:, c] |= rel_close(d_ext[:, nb], d_ext[:, c]) & np.isfinite(d_ext[:, c])
    mism = (gpu_idx != oi) & ~tie & valid
    if mism.any():
        r, c = np.argwhere(mism)[0]
        raise AssertionError(f"index mismatch outside ties row {r} rank {c}: gpu {gpu_idx[r, c]} "
                             f"oracle {oi[r, c]} (d2 {od[r, c]!r})")
    # 5. no duplicates within a row
    for r in np.nonzero(((gpu_idx != oi) & valid).any(1))[0]:
        row = gpu_idx[r][gpu_idx[r] >= 0]
        if len(set(row.tolist())) != len(row):
            raise AssertionError(f"duplicate neighbours in row {r}")
    return int(((gpu_idx != oi) & valid).any(1).sum())


def angle_unsigned(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    cr = np.linalg.norm(np.cross(a, b), axis=-1)
    dt = np.abs((a * b).sum(-1))
    return np.arctan2(cr, dt)


def rot_angle(Ra, Rb):
    M = np.asarray(Ra) @ np.asarray(Rb).T
    w = np.array([M[2, 1] - M[1, 2], M[0, 2] - M[2, 0], M[1, 0] - M[0, 1]]) / 2
    return float(np.arctan2(np.linalg.norm(w), (np.trace(M) - 1) / 2))


def extent(pts):
    p = np.asarray(pts, np.float64)
    return float(np.linalg.norm(p.max(0) - p.min(0)))


def rmse_tol(pts, rot=0.0, trans=0.0):
    """Bar on |RMSE_library - RMSE_oracle| (absolute) for point-to-plane ICP.
    Each FP32 residual r = n.(p' - q) carries the rounding of p' = R p + t,
    of the difference and of the dot product: |dr| <= ~4 eps32 M, with M the
    largest coordinate magnitude; the RMSE (a 2-norm over sqrt(n)) moves by
    at most max |dr|.  Transforms that differ by `rot` rad and `trans` move
    each residual by at most rot M + trans more."""
    M = float(np.abs(np.asarray(pts, np.float64)).max())
    return 4 * 2.0 ** -24 * M + rot * M + trans
