"""Certified correspondences are the exact search's, round by round.

From the second round on, the ICP search keeps a query's neighbour (or its
lack of one) without searching when a distance bound proves it unchanged;
queries searched a warp at a time, and queued ones finished with a grown
ball, record those bounds.  A call that starts at a given transform has no
bounds yet, so its first round searches every query exactly.  So round k of
a K-round run must produce the same correspondences as a one-round call
started at the transform that run holds after k rounds: the same inlier count
and the same normal-equation sums up to their summation order (the fresh call
orders its sources by where that transform puts them, so its tiles add the
same terms in another order: the compensated sums then agree to ~1e-15).  One
correspondence a certificate got wrong would move a sum by one term, ~1e-6 of
it and more, and the bar is 1e-12 of each sum's Cauchy-Schwarz scale.

Cases: a wavy patch with sources lifted 0..2 cm and points far above it (every
search stage, outliers kept as outliers, far inliers bounded by the finish),
at two rejection distances; the depth-frame pair with the library's normals
(the bench's workload: warp-per-query first stages once converged)."""
import numpy as np
import pytest
import torch

import paper_1807_00399_gb300 as cil
from paper_1807_00399_gb300 import synth
from test_gpu_icp import _offset_surface_case

pytestmark = pytest.mark.gpu


def _case(name):
    if name == "depth":
        p = synth.depth_frame_pair(0)
        D = torch.from_numpy(p.target).cuda()
        N, _ = cil.estimate_normals(D, 10, p.viewpoint)
        return torch.from_numpy(p.source).cuda(), D, N, 0.05, 30
    src, tgt, nrm = _offset_surface_case(11)
    dmax = {"offset_5mm": 0.005, "offset_2cm": 0.02}[name]
    return (torch.from_numpy(src).cuda(), torch.from_numpy(tgt).cuda(),
            torch.from_numpy(nrm).cuda(), dmax, 15)


IU = [(u, v) for u in range(6) for v in range(u, 6)]  # upper triangle, row by row


def _scales(row):
    """Cauchy-Schwarz scale of each of a round's 28 sums: sqrt(H_uu H_vv) for
    H, sqrt(H_uu sum r^2) for g, sum r^2 for itself."""
    d = [abs(row[IU.index((u, u))]) for u in range(6)]
    rr = abs(row[27])
    sc = [np.sqrt(d[u] * d[v]) for u, v in IU] + [np.sqrt(d[u] * rr) for u in range(6)] + [rr]
    return np.maximum(np.array(sc), 1e-300)


@pytest.mark.parametrize("name", ["offset_5mm", "offset_2cm", "depth"])
def test_certified_rounds_equal_fresh_searches(name):
    S, D, N, dmax, K = _case(name)
    _, rep = cil.icp(S, D, N, iters=K, max_corr_dist=dmax, with_sums=True)
    multi = rep["sums"]
    T = np.eye(4)
    for k in range(K):
        _, r1 = cil.icp(S, D, N, T_init=T, iters=1, max_corr_dist=dmax, with_sums=True)
        fresh, cert = r1["sums"][0], multi[k]
        assert fresh[28] == cert[28], f"round {k}: {cert[28]} inliers certified, {fresh[28]} searched"
        assert np.max(np.abs(fresh - cert)[:28] / _scales(fresh)) <= 1e-12, f"round {k}"
        # the transform the K-round run holds after k + 1 rounds
        T, _ = cil.icp(S, D, N, iters=k + 1, max_corr_dist=dmax)
