"""Batched registration (cil_icp_batch_*): B uneven pairs in one graph launch
must give, pair by pair, exactly what the single-pair call gives (same grid
per cloud, same stable order, same tiles and reduction order), and agree with
the oracle at the ICP tolerances."""
import numpy as np
import pytest
import torch

import oracle
import paper_1807_00399_gb300 as cil
from paper_1807_00399_gb300 import synth
from parity import extent, rot_angle

pytestmark = pytest.mark.gpu


def _pairs(sizes, seed0=1000):
    return [synth.surface_pair(seed0 + i, n=int(n)) for i, n in enumerate(sizes)]


def _cat(pairs):
    src = np.concatenate([p.source for p in pairs])
    dst = np.concatenate([p.target for p in pairs])
    return torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda()


def test_batch_equals_single_pair_calls_bitwise():
    sizes = [2000, 5313, 700, 12000, 3001, 40000, 1500, 9999]
    pairs = _pairs(sizes)
    src, dst = _cat(pairs)
    h = cil.Batch(sizes, sizes, k=10, iters=20, max_corr_dist=0.1, viewpoint=(0, 0, 10))
    nrm = torch.empty_like(dst)
    T, rep = h.run(src, dst, normals_out=nrm)
    torch.cuda.synchronize()
    reps = cil.decode_reports(rep, len(sizes))
    T = T.cpu().numpy().reshape(-1, 4, 4)
    off = 0
    for b, p in enumerate(pairs):
        s = torch.from_numpy(p.source).cuda()
        d = torch.from_numpy(p.target).cuda()
        n1 = torch.empty_like(d)
        T1, r1, _ = cil.register_pair(s, d, 10, (0, 0, 10), 20, 0.1, out_normals=n1)
        torch.cuda.synchronize()
        assert np.array_equal(T[b], T1.cpu().numpy().reshape(4, 4)), f"pair {b} transform"
        assert reps[b] == cil.decode_report(r1), f"pair {b} report"
        assert torch.equal(nrm[off:off + sizes[b]], n1), f"pair {b} normals"
        off += sizes[b]
    h.close()


def test_batch_matches_oracle_and_replays():
    sizes = [3000, 800, 6000]
    pairs = _pairs(sizes, seed0=2000)
    src, dst = _cat(pairs)
    h = cil.Batch(sizes, sizes, k=10, iters=15, max_corr_dist=0.1, viewpoint=(0, 0, 10))
    nrm = torch.empty_like(dst)
    T_a, rep_a = h.run(src, dst, normals_out=nrm)
    T_b, rep_b = h.run(src, dst, normals_out=nrm, T_out=torch.empty_like(T_a))  # re-capture
    T_c, rep_c = h.run(src, dst, normals_out=nrm, T_out=T_a, rep=rep_a)  # replay
    torch.cuda.synchronize()
    assert torch.equal(T_a, T_b) and torch.equal(T_a, T_c)
    T = T_a.cpu().numpy().reshape(-1, 4, 4)
    nrm_h = nrm.cpu().numpy()
    off = 0
    for b, p in enumerate(pairs):
        o = oracle.icp(p.source, p.target, nrm_h[off:off + sizes[b]], iters=15, max_corr_dist=0.1)
        assert rot_angle(T[b][:3, :3], o["T"][:3, :3]) <= 1e-5
        assert np.abs(T[b][:3, 3] - o["T"][:3, 3]).max() <= 1e-6 * extent(p.target)
        off += sizes[b]
    h.close()


def test_batch_with_initial_transforms_and_empty_pair():
    sizes_s = [2500, 0, 1800]
    sizes_d = [2500, 1000, 1800]
    pairs = _pairs([2500, 1000, 1800], seed0=3000)
    src = torch.from_numpy(np.concatenate([pairs[0].source, pairs[2].source])).cuda()
    dst = torch.from_numpy(np.concatenate([p.target for p in pairs])).cuda()
    T0 = np.tile(np.eye(4), (3, 1, 1))
    T0[2, :3, 3] = [0.01, 0.0, -0.01]
    T0d = torch.from_numpy(T0.reshape(3, 16)).cuda()
    h = cil.Batch(sizes_s, sizes_d, k=10, iters=5, max_corr_dist=0.1)
    T, rep = h.run(src, dst, T_init=T0d)
    torch.cuda.synchronize()
    reps = cil.decode_reports(rep, 3)
    assert reps[1]["status"] == cil.DEGENERATE and reps[1]["n_inliers"] == 0
    assert reps[0]["status"] == 0 and reps[2]["status"] == 0
    s2 = torch.from_numpy(pairs[2].source).cuda()
    d2 = torch.from_numpy(pairs[2].target).cuda()
    T2, r2, _ = cil.register_pair(s2, d2, 10, (0, 0, 10), 5, 0.1, T_init=T0d[2].contiguous())
    torch.cuda.synchronize()
    assert np.array_equal(T.cpu().numpy()[2], T2.cpu().numpy())
    h.close()
