"""Golden fixtures (tests/golden/, written by make_golden.py from the oracle):
each value is re-derived here by hand, independently of the oracle, and the
oracle must still reproduce the stored file."""
import os
import subprocess
import sys

import numpy as np

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _read(name):
    out = {}
    with open(os.path.join(HERE, name)) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            key, *vals = line.split()
            out.setdefault(key, []).append([float(v) for v in vals])
    return out


def test_lattice_queries_by_hand():
    g = _read("lattice_queries.txt")
    # centre (2,2,2) of a 5x5x5 lattice indexed 25 x + 5 y + z; unit-distance
    # neighbours are the six face neighbours, ascending index
    face = sorted(25 * (2 + dx) + 5 * (2 + dy) + (2 + dz)
                  for dx, dy, dz in [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)])
    assert g["radius_idx"][0] == [62] + face
    assert g["radius_d2"][0] == [0.0] + [1.0] * 6
    # the next shell (d^2 = 2): the twelve edge neighbours, the three smallest indices
    edge = sorted(25 * (2 + a) + 5 * (2 + b) + (2 + c)
                  for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)
                  if abs(a) + abs(b) + abs(c) == 2)
    assert g["knn_idx"][0] == [62] + face + edge[:3]
    assert g["knn_d2"][0] == [0.0] + [1.0] * 6 + [2.0] * 3


def test_plane_normal_by_hand():
    g = _read("plane_normal.txt")
    n = np.array([-0.5, -0.25, 1.0])
    n /= np.linalg.norm(n)  # gradient of z - x/2 - y/4, oriented up towards (0, 0, 10)
    np.testing.assert_allclose(g["normal"][0], n, atol=1e-12)
    assert abs(g["curvature"][0][0]) < 1e-12


def test_icp_exact_motion_by_hand():
    T = np.array(_read("icp_exact_motion.txt")["T"])
    a = np.radians(2.0)
    R = np.array([[np.cos(a), -np.sin(a), 0.0], [np.sin(a), np.cos(a), 0.0], [0.0, 0.0, 1.0]])
    np.testing.assert_allclose(T[:3, :3], R, atol=1e-8)
    np.testing.assert_allclose(T[:3, 3], [0.01, -0.02, 0.005], atol=1e-8)
    np.testing.assert_array_equal(T[3], [0, 0, 0, 1])


def test_oracle_reproduces_the_fixtures(tmp_path):
    src = os.path.join(HERE, "make_golden.py")
    # run the generator on copies, then compare with the stored files
    import shutil
    work = tmp_path / "golden"
    work.mkdir()
    shutil.copy(src, work / "make_golden.py")
    env = dict(os.environ)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env["PYTHONPATH"] = root + os.pathsep + env.get("PYTHONPATH", "")
    # the generator writes next to itself; point it at the repo's packages
    code = open(src).read().replace(
        "sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))", f"sys.path.insert(0, {root!r})")
    (work / "make_golden.py").write_text(code)
    subprocess.run([sys.executable, str(work / "make_golden.py")], check=True, env=env)
    for name, tol in (("lattice_queries.txt", 0.0), ("plane_normal.txt", 1e-11),
                      ("icp_exact_motion.txt", 1e-10)):
        new = {}
        for line in (work / name).read_text().splitlines():
            if line.startswith("#") or not line.strip():
                continue
            key, *vals = line.split()
            new.setdefault(key, []).append([float(v) for v in vals])
        old = _read(name)
        assert new.keys() == old.keys(), name
        for k in old:
            np.testing.assert_allclose(np.array(new[k]), np.array(old[k]), atol=tol, rtol=0)
