"""The correspondence certificate's rule, checked on the CPU against brute
force: if a query's nearest target point q at position p0 has every other
point at least lb away, and the query moves to p1 by delta, then
|p1 - q| (1 + 1e-5) + delta (1 + 1e-5) < lb guarantees that q is still the
nearest point at p1 -- with a margin that survives FP32 rounding of the
squared distances the search compares."""
import numpy as np


def _nearest_two(P, x):
    d2 = ((P.astype(np.float64) - x) ** 2).sum(1)
    o = np.lexsort((np.arange(len(P)), d2))
    return o[0], d2[o[0]], d2[o[1]]


def _fp32_nearest(P, x):
    x = x.astype(np.float32)
    d = P - x
    d2 = (d[:, 2] * d[:, 2] + (d[:, 1] * d[:, 1] + d[:, 0] * d[:, 0])).astype(np.float32)
    return int(np.lexsort((np.arange(len(P)), d2))[0])


def test_certified_neighbours_are_unchanged():
    rng = np.random.default_rng(0)
    P = rng.uniform(-1, 1, (3000, 3)).astype(np.float32)
    certified = 0
    for t in range(3000):
        p0 = rng.uniform(-1, 1, 3)
        q, d1, d2 = _nearest_two(P, p0)
        lb = np.sqrt(d2) * (1 - 1e-5)
        move = rng.normal(size=3)
        move *= rng.uniform(0, 0.05) / np.linalg.norm(move)
        p1 = p0 + move
        delta = np.linalg.norm(p1 - p0) * (1 + 1e-5)
        dn = np.linalg.norm(P[q].astype(np.float64) - p1)
        if dn * (1 + 1e-5) + delta < lb:
            certified += 1
            assert _fp32_nearest(P, p1) == q
            # the carried bound stays a valid lower bound at p1
            others = np.delete(np.arange(len(P)), q)
            assert np.sqrt(((P[others].astype(np.float64) - p1) ** 2).sum(1)).min() >= lb - delta
    assert certified > 100  # the rule fires on a good share of small moves


def test_no_certificate_without_margin():
    # two points equidistant from p0: no positive margin, so no certificate
    P = np.array([[1.0, 0, 0], [-1.0, 0, 0], [0, 5.0, 0]], np.float32)
    p0 = np.zeros(3)
    q, d1, d2 = _nearest_two(P, p0)
    lb = np.sqrt(d2) * (1 - 1e-5)
    dn = np.sqrt(d1)
    assert not (dn * (1 + 1e-5) + 0.0 < lb)
