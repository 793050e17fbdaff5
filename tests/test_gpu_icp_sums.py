"""Compensated FP32 sums of the ICP normal equations (cil_icp_sums), pinned two
ways.

1. Exact terms: a source lattice (i, j, 1/2) over a target lattice (i, j, 0)
   with normals e_z.  Every row (J, r) = ((j, -i, 0, 0, 0, 1), 1/2) and every
   product of two of its entries is an integer or half-integer below 2^24, so
   each FP32 term is exact and the only error left is the summation's.  The
   exact sums are Python integers.  Compensated (TwoSum) sums stay within a
   few eps32^2 of them (relative 1e-11 allowed); a plain FP32 sum of 3e5 terms
   whose totals exceed 2^24 misses by ~1e-7 relative or more.
2. Against the FP64 oracle on wavy-surface pairs of 1e3 .. 3e5 points: the
   first round's H and g (both sides start at the same transform, so the
   correspondences agree) differ only through the FP32 rounding of each term,
   which averages out: the error normalised by the Cauchy-Schwarz bound of
   each entry (sqrt(H_uu H_vv) for H, sqrt(H_uu sum r^2) for g) must stay
   below 1e-7 at every N and must not grow with N.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1807_00399_gb300 as cil
from paper_1807_00399_gb300 import synth

pytestmark = pytest.mark.gpu

IU = [(u, v) for u in range(6) for v in range(u, 6)]  # upper triangle, row by row


def _lattice(n_side_i, n_side_j, i0, j0):
    i, j = np.meshgrid(np.arange(i0, i0 + n_side_i), np.arange(j0, j0 + n_side_j), indexing="ij")
    i, j = i.ravel(), j.ravel()
    dst = np.column_stack([i, j, np.zeros_like(i)]).astype(np.float32)
    src = np.column_stack([i, j, np.full_like(i, 0.5, dtype=np.float64)]).astype(np.float32)
    return src, dst, i.astype(object), j.astype(object)


@pytest.mark.parametrize("shape", [(32, 32, -9, 4), (100, 101, -60, -13), (316, 317, -100, -200),
                                   (548, 548, -150, -199)])
def test_exact_lattice_sums(shape, parity_report):
    src, dst, i, j = _lattice(*shape)
    n = len(src)
    nrm = np.tile(np.float32([0, 0, 1]), (n, 1))
    S = torch.from_numpy(src).cuda()
    D = torch.from_numpy(dst).cuda()
    N = torch.from_numpy(nrm).cuda()
    T, rep = cil.icp(S, D, N, iters=1, max_corr_dist=0.75, with_sums=True)
    s = rep["sums"]
    # exact sums of the rows J = (j, -i, 0, 0, 0, 1), r = 1/2, as Python integers
    J = [j, -i, 0 * i, 0 * i, 0 * i, 0 * i + 1]
    H = {(u, v): int(sum(J[u] * J[v])) for u, v in IU}
    g2 = [int(sum(J[u])) for u in range(6)]  # g = g2 / 2
    for rnd in (0, 1):  # the round (degenerate: T stays) and the final pass
        row = s[rnd]
        assert row[28] == n
        worst = 0.0
        for q, (u, v) in enumerate(IU):
            scale = max(abs(H[(u, u)]) * abs(H[(v, v)]), 1) ** 0.5
            err = abs(row[q] - H[(u, v)]) / scale
            worst = max(worst, err)
            assert err <= 1e-11, f"H[{u}{v}]: {row[q]!r} vs {H[(u, v)]} (rel {err:.3g})"
        for u in range(6):
            scale = max(abs(H[(u, u)]) * (0.25 * n), 1) ** 0.5
            err = abs(row[21 + u] - g2[u] / 2) / scale
            worst = max(worst, err)
            assert err <= 1e-11, f"g[{u}]: {row[21 + u]!r} vs {g2[u] / 2}"
        assert abs(row[27] - 0.25 * n) <= 1e-11 * 0.25 * n
    parity_report(f"ICP sums, exact lattice N={n}", max_rel_err=worst,
                  H00=float(s[0][0]), exact=float(H[(0, 0)]))


@pytest.fixture(scope="module")
def surface_errors():
    out = {}
    for n in (1_000, 10_000, 100_000, 300_000):
        p = synth.surface_pair(40 + n % 97, n=n)
        on, _, _ = oracle.normals(p.target, 10, p.viewpoint, method="kdtree")
        nrm = on.astype(np.float32)
        _, rep = cil.icp(torch.from_numpy(p.source).cuda(), torch.from_numpy(p.target).cuda(),
                         torch.from_numpy(nrm).cuda(), iters=3, max_corr_dist=0.1, with_sums=True)
        o = oracle.icp(p.source, p.target, nrm, iters=3, max_corr_dist=0.1, method="kdtree",
                       want_trace=True)
        s = rep["sums"][0]
        Ho, go = o["H"][0], o["g"][0]
        rr = s[27]
        eh = max(abs(s[q] - Ho[u, v]) / np.sqrt(Ho[u, u] * Ho[v, v]) for q, (u, v) in enumerate(IU))
        eg = max(abs(s[21 + u] - go[u]) / np.sqrt(Ho[u, u] * rr) for u in range(6))
        out[n] = (eh, eg, int(s[28]))
    return out


def test_first_round_sums_match_oracle(surface_errors, parity_report):
    for n, (eh, eg, cnt) in surface_errors.items():
        parity_report(f"ICP sums vs FP64 oracle, wavy surface N={n}, round 1", H_rel=eh, g_rel=eg,
                      inliers=cnt)
        assert eh <= 1e-7 and eg <= 1e-7, f"N={n}: H {eh:.3g}, g {eg:.3g}"
    # the error must not grow with N (compensated sums: only the terms'
    # rounding remains, and it averages out)
    e = [max(v[0], v[1]) for _, v in sorted(surface_errors.items())]
    assert e[-1] <= 3 * e[0] + 1e-9
