"""Writes the golden fixtures of this folder from the FP64 oracle (and only
from it).  The paper prints no worked example with numbers (its result
figures are not in the available text), so the fixtures are small cases
whose values also follow from a hand derivation, which tests/test_golden.py
re-does independently of the oracle:

  lattice_queries.txt  5x5x5 integer lattice, queries from its centre
                       (2, 2, 2) = point 62: the radius-1 ball (Sec. 3
                       radius query; inclusive boundary, (d^2, index) order)
                       and the 10 nearest (Sec. 3 k-NN; the point itself
                       first, ties by index);
  plane_normal.txt     the 10-NN PCA normal and curvature of a point on the
                       plane z = x/2 + y/4 (Sec. 3 normals, oriented towards
                       the viewpoint (0, 0, 10));
  icp_exact_motion.txt point-to-plane ICP (Sec. 3, Low 2004 linearisation)
                       of a noiseless rigidly moved copy: the exact motion.

    python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_1807_00399_gb300 import synth  # noqa: E402


def plane_cloud():
    g = np.stack(np.meshgrid(np.arange(-3, 4), np.arange(-3, 4), indexing="ij"), -1).reshape(-1, 2)
    x, y = g[:, 0].astype(np.float64) * 0.5, g[:, 1].astype(np.float64) * 0.5
    return np.column_stack([x, y, 0.5 * x + 0.25 * y]).astype(np.float32)


def motion_case():
    rng = np.random.default_rng(5)
    tgt = synth.surface_points(rng, 3000, noise=0.0).astype(np.float32)
    ang = np.radians(2.0)
    R = np.array([[np.cos(ang), -np.sin(ang), 0.0], [np.sin(ang), np.cos(ang), 0.0], [0, 0, 1.0]])
    t = np.array([0.01, -0.02, 0.005])
    src = ((tgt.astype(np.float64) - t) @ R).astype(np.float32)  # so that T = [R t] maps src -> tgt
    return src, tgt, R, t


def main():
    P = synth.lattice_points((5, 5, 5))
    off, idx, d2 = oracle.radius(P, P[62:63], 1.0)
    kidx, kd2 = oracle.knn(P, P[62:63], 10)
    with open(os.path.join(HERE, "lattice_queries.txt"), "w") as f:
        f.write("# 5x5x5 integer lattice (index = 25 x + 5 y + z), query = point 62 = (2, 2, 2)\n")
        f.write("# Sec. 3 radius query (r = 1, inclusive) and k-NN (k = 10), (d^2, index) order\n")
        f.write("radius_idx " + " ".join(map(str, idx.tolist())) + "\n")
        f.write("radius_d2 " + " ".join(f"{v:.1f}" for v in d2.tolist()) + "\n")
        f.write("knn_idx " + " ".join(map(str, kidx[0].tolist())) + "\n")
        f.write("knn_d2 " + " ".join(f"{v:.1f}" for v in kd2[0].tolist()) + "\n")
    Q = plane_cloud()
    n, c, _ = oracle.normals(Q, 10, (0.0, 0.0, 10.0))
    with open(os.path.join(HERE, "plane_normal.txt"), "w") as f:
        f.write("# 7x7 grid of spacing 0.5 on the plane z = x/2 + y/4; point 24 = the origin\n")
        f.write("# Sec. 3 normals (10 nearest, PCA), oriented towards (0, 0, 10)\n")
        f.write("normal " + " ".join(f"{v:.12f}" for v in n[24].tolist()) + "\n")
        f.write(f"curvature {abs(c[24]):.12f}\n")
    src, tgt, R, t = motion_case()
    nrm, _, _ = oracle.normals(tgt, 10, (0.0, 0.0, 10.0))
    out = oracle.icp(src, tgt, nrm.astype(np.float32), iters=30, max_corr_dist=0.2)
    with open(os.path.join(HERE, "icp_exact_motion.txt"), "w") as f:
        f.write("# noiseless wavy surface (3000 points) moved by 2 deg about z and (0.01, -0.02, 0.005)\n")
        f.write("# Sec. 3 point-to-plane ICP, 30 rounds, d_max 0.2: the transform source -> target\n")
        for r in out["T"]:
            f.write("T " + " ".join(f"{v:.12f}" for v in r.tolist()) + "\n")


if __name__ == "__main__":
    main()
