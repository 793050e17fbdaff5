"""FP64 CPU oracle for kNN, radius search, PCA normals and point-to-plane ICP.

TEST INFRASTRUCTURE.  Only the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` import this package.  The product library
(``paper_1807_00399_gb300``) never imports, links or executes anything here,
and this package imports nothing from the product library: the two share only
the seeded input generators.

The arithmetic lives in ``cil_oracle.c`` (plain C, FP64, exhaustive search as
the definition, a kd-tree as a validated faster route for large inputs, cyclic
Jacobi for the 3x3 eigenproblem, Cholesky for the 6x6 Gauss-Newton system).
This module only marshals numpy arrays through ctypes.

Parity pins (each checked by a ``-m "not gpu"`` test against something other
than the oracle itself):

* kNN / radius: scipy's cKDTree (a library routine), exact integer-lattice
  neighbour sets and tie orders, permutation and rigid-motion equivariance;
* eigen: numpy.linalg.eigh;
* normals: exact normals of planes, analytic sphere normals, viewpoint
  orientation, rotation equivariance, degenerate neighbourhoods;
* ICP: the exact transform of a noiseless moved copy, one Gauss-Newton step
  equal to numpy.linalg.lstsq on independently built Jacobian rows,
  rigid-motion equivariance, invariance to normal signs and to permutations,
  and a planar (singular) target flagged degenerate.

The ICP variants of Sec. 3 (point-to-point, weighted combination, projective
association) are in ``icp_variants.py`` (numpy FP64, pinned by
``tests/test_oracle_icp_variants.py``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cil_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

ICP_DEGENERATE = 5


def build(force: bool = False) -> str:
    """Compile the oracle with the host C compiler (no target-specific flags,
    no contraction of multiply-adds, so x86 and Arm hosts agree bit for bit)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-fPIC", "-shared",
             "-pthread", _SRC, "-o", tmp, "-lm"]
        )
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    P = ctypes.c_void_p
    I64 = ctypes.c_int64
    I = ctypes.c_int
    D = ctypes.c_double
    lib.oracle_default_threads.restype = I
    lib.oracle_knn.argtypes = [P, I64, P, I64, I, P, P, I]
    lib.oracle_knn_kdtree.argtypes = [P, I64, P, I64, I, P, P, I]
    lib.oracle_radius.argtypes = [P, I64, P, I64, D, P, P, P, I]
    lib.oracle_sym3_eigen.argtypes = [P, P, P]
    lib.oracle_normals.argtypes = [P, I64, I, P, P, P, P, I, I]
    lib.oracle_normals_subset.argtypes = [P, I64, P, I64, I, P, P, P, P, I, I]
    lib.oracle_icp.argtypes = [P, I64, P, P, I64, P, I, D, P, P, P, P, P, P, I, I]
    lib.oracle_knn_hybrid.argtypes = [P, I64, P, I64, I, D, P, P, I]
    lib.oracle_normals_radius.argtypes = [P, I64, D, P, P, P, P, P, P, I64, I]
    lib.oracle_voxel_downsample.argtypes = [P, I64, ctypes.c_float, P, P, P]
    for f in ("oracle_knn", "oracle_knn_kdtree", "oracle_radius", "oracle_sym3_eigen",
              "oracle_normals", "oracle_normals_subset", "oracle_icp", "oracle_knn_hybrid",
              "oracle_normals_radius", "oracle_voxel_downsample"):
        getattr(lib, f).restype = I
    _lib = lib
    return lib


def _pts(a) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float32)
    if a.ndim != 2 or a.shape[1] != 3:
        raise ValueError("points must have shape (N, 3)")
    return a


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def default_threads() -> int:
    return int(_load().oracle_default_threads())


def knn(ref, qry, k: int, method: str = "brute", threads: int = 0):
    """k nearest neighbours of each query: (idx int32 (Nq,k), d2 float64 (Nq,k)),
    ordered by (d2, idx); padded with -1 / inf when k > len(ref)."""
    lib = _load()
    ref = _pts(ref)
    qry = _pts(qry)
    idx = np.empty((qry.shape[0], k), np.int32)
    d2 = np.empty((qry.shape[0], k), np.float64)
    f = lib.oracle_knn if method == "brute" else lib.oracle_knn_kdtree
    rc = f(_p(ref), ref.shape[0], _p(qry), qry.shape[0], int(k), _p(idx), _p(d2), int(threads))
    if rc:
        raise RuntimeError(f"oracle knn failed ({rc})")
    return idx, d2


def radius(ref, qry, r: float, threads: int = 0):
    """All neighbours within r (inclusive): CSR (offsets int64, idx int32, d2 f64),
    each row sorted by (d2, idx).  r is taken as the float32 value it would have
    at the C-ABI, promoted to double."""
    lib = _load()
    ref = _pts(ref)
    qry = _pts(qry)
    rr = float(np.float32(r))
    off = np.zeros(qry.shape[0] + 1, np.int64)
    rc = lib.oracle_radius(_p(ref), ref.shape[0], _p(qry), qry.shape[0], rr, _p(off), None, None,
                           int(threads))
    if rc:
        raise RuntimeError("oracle radius failed")
    nnz = int(off[-1])
    idx = np.empty(max(nnz, 1), np.int32)
    d2 = np.empty(max(nnz, 1), np.float64)
    rc = lib.oracle_radius(_p(ref), ref.shape[0], _p(qry), qry.shape[0], rr, _p(off), _p(idx),
                           _p(d2), int(threads))
    if rc:
        raise RuntimeError("oracle radius failed")
    return off, idx[:nnz], d2[:nnz]


def knn_hybrid(ref, qry, k: int, r: float, threads: int = 0):
    """The k nearest neighbours among those within r (inclusive): (idx, d2),
    padded with -1 / inf.  r is taken as its float32 value, promoted."""
    lib = _load()
    ref = _pts(ref)
    qry = _pts(qry)
    idx = np.empty((qry.shape[0], k), np.int32)
    d2 = np.empty((qry.shape[0], k), np.float64)
    rc = lib.oracle_knn_hybrid(_p(ref), ref.shape[0], _p(qry), qry.shape[0], int(k),
                               float(np.float32(r)), _p(idx), _p(d2), int(threads))
    if rc:
        raise RuntimeError("oracle knn_hybrid failed")
    return idx, d2


def normals_radius(xyz, r: float, viewpoint, sel=None, threads: int = 0):
    """PCA normals over radius neighbourhoods (every point within r, itself
    included): (normals, curvature, evals, neighbour counts), for every point
    or only for the points `sel` (neighbourhoods still searched in all of xyz)."""
    lib = _load()
    xyz = _pts(xyz)
    n = xyz.shape[0]
    vp = np.ascontiguousarray(viewpoint, np.float64).reshape(3)
    sel_a = None if sel is None else np.ascontiguousarray(sel, np.int64)
    m = n if sel_a is None else sel_a.shape[0]
    nrm = np.empty((m, 3), np.float64)
    cur = np.empty(m, np.float64)
    ev = np.empty((m, 3), np.float64)
    cnt = np.empty(m, np.int64)
    rc = lib.oracle_normals_radius(_p(xyz), n, float(np.float32(r)), _p(vp), _p(nrm), _p(cur),
                                   _p(ev), _p(cnt), None if sel_a is None else _p(sel_a), m,
                                   int(threads))
    if rc:
        raise RuntimeError("oracle normals_radius failed")
    return nrm, cur, ev, cnt


def voxel_downsample(xyz, voxel: float):
    """Mean of the points of every occupied voxel floor(p / voxel) (float32
    division), ascending (ix, iy, iz): (points f64 (M,3), counts int64 (M,))."""
    lib = _load()
    xyz = _pts(xyz)
    n = xyz.shape[0]
    out = np.empty((max(n, 1), 3), np.float64)
    cnt = np.empty(max(n, 1), np.int64)
    m = ctypes.c_int64()
    rc = lib.oracle_voxel_downsample(_p(xyz), n, float(np.float32(voxel)), _p(out), _p(cnt),
                                     ctypes.byref(m))
    if rc:
        raise RuntimeError("oracle voxel_downsample failed")
    return out[:m.value], cnt[:m.value]


def sym3_eigen(C):
    """Jacobi eigen-decomposition of a symmetric 3x3: (evals ascending, evecs
    as columns)."""
    C = np.asarray(C, np.float64)
    cu = np.ascontiguousarray([C[0, 0], C[0, 1], C[0, 2], C[1, 1], C[1, 2], C[2, 2]], np.float64)
    ev = np.empty(3, np.float64)
    vec = np.empty(9, np.float64)
    _load().oracle_sym3_eigen(_p(cu), _p(ev), _p(vec))
    return ev, vec.reshape(3, 3)


def normals(xyz, k: int, viewpoint, method: str = "auto", threads: int = 0):
    """PCA normals, curvature and covariance eigenvalues for every point:
    (normals f64 (N,3), curvature f64 (N,), evals f64 (N,3) ascending)."""
    lib = _load()
    xyz = _pts(xyz)
    n = xyz.shape[0]
    vp = np.ascontiguousarray(viewpoint, np.float64).reshape(3)
    nrm = np.empty((n, 3), np.float64)
    cur = np.empty(n, np.float64)
    ev = np.empty((n, 3), np.float64)
    use_kd = (n > 20000) if method == "auto" else (method == "kdtree")
    rc = lib.oracle_normals(_p(xyz), n, int(k), _p(vp), _p(nrm), _p(cur), _p(ev), int(use_kd),
                            int(threads))
    if rc:
        raise RuntimeError("oracle normals failed")
    return nrm, cur, ev


def normals_subset(xyz, sel, k: int, viewpoint, method: str = "brute", threads: int = 0):
    """Normals of the points xyz[sel] with neighbourhoods searched in all of xyz."""
    lib = _load()
    xyz = _pts(xyz)
    sel = np.ascontiguousarray(sel, np.int64)
    m = sel.shape[0]
    vp = np.ascontiguousarray(viewpoint, np.float64).reshape(3)
    nrm = np.empty((m, 3), np.float64)
    cur = np.empty(m, np.float64)
    ev = np.empty((m, 3), np.float64)
    rc = lib.oracle_normals_subset(_p(xyz), xyz.shape[0], _p(sel), m, int(k), _p(vp), _p(nrm),
                                   _p(cur), _p(ev), int(method == "kdtree"), int(threads))
    if rc:
        raise RuntimeError("oracle normals_subset failed")
    return nrm, cur, ev


def icp(src, dst, dst_normals, T_init=None, iters: int = 20, max_corr_dist: float = 0.1,
        method: str = "auto", threads: int = 0, want_trace: bool = False):
    """Rigid point-to-plane ICP.  Returns a dict with T (4x4 f64, source ->
    target), rmse, n_inliers, status (0 or ICP_DEGENERATE) and, on request,
    the per-round transforms and normal-equation sums."""
    lib = _load()
    src = _pts(src)
    dst = _pts(dst)
    nrm = _pts(dst_normals)
    if nrm.shape != dst.shape:
        raise ValueError("dst_normals must match dst")
    T0 = np.ascontiguousarray(np.eye(4) if T_init is None else T_init, np.float64).reshape(16)
    T = np.empty(16, np.float64)
    rmse = ctypes.c_double()
    ninl = ctypes.c_int64()
    status = ctypes.c_int()
    trace = np.empty((max(iters, 1), 16), np.float64) if want_trace else None
    sums = np.empty((max(iters, 1), 42), np.float64) if want_trace else None
    use_kd = (dst.shape[0] * src.shape[0] > 4e8) if method == "auto" else (method == "kdtree")
    # max_corr_dist reaches the library as a float32; use that value here too
    dmax = float(np.float32(max_corr_dist))
    rc = lib.oracle_icp(_p(src), src.shape[0], _p(dst), _p(nrm), dst.shape[0], _p(T0), int(iters),
                        dmax, _p(T), ctypes.byref(rmse), ctypes.byref(ninl), ctypes.byref(status),
                        _p(trace) if want_trace else None, _p(sums) if want_trace else None,
                        int(use_kd), int(threads))
    if rc:
        raise RuntimeError("oracle icp failed")
    out = {"T": T.reshape(4, 4), "rmse": rmse.value, "n_inliers": ninl.value,
           "status": status.value}
    if want_trace:
        out["trace"] = trace[:iters].reshape(-1, 4, 4)
        out["H"] = sums[:iters, :36].reshape(-1, 6, 6)
        out["g"] = sums[:iters, 36:]
    return out
