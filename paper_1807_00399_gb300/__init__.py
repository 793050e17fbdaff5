"""GB300 point-cloud hot path: grid kNN / radius search, PCA normals and
point-to-plane ICP as sm_103a CUDA kernels behind the C ABI in include/cil.h.

This module is a thin ctypes binding: it checks tensor shapes/devices, passes
raw device pointers and the current CUDA stream to libcil.so, and turns status
codes into exceptions.  Every step of the computation runs in the library's
kernels; there is no CPU path.  If libcil.so is missing it is built with nvcc
(``paper_1807_00399_gb300.build``); if that is impossible, loading fails.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

__all__ = [
    "CilError", "lib", "knn", "radius_search", "estimate_normals", "icp_point_to_plane",
    "register_pair", "sync_status", "Params", "STATUS", "MAX_K", "IcpReport", "Batch", "icp",
    "IcpOptions", "segment", "smooth_segment",
    "decode_report", "decode_reports",
]

MAX_K = 32
STATUS = {
    0: "CIL_OK", 1: "CIL_ERR_INVALID_ARG", 2: "CIL_ERR_CUDA", 3: "CIL_ERR_NONFINITE",
    4: "CIL_ERR_CAPACITY", 5: "CIL_ERR_DEGENERATE", 6: "CIL_ERR_TIMEOUT", 7: "CIL_ERR_NOMEM",
}
DEGENERATE = 5

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libcil.so")
_lib = None
_lock = threading.Lock()


class CilError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = int(status)
        super().__init__(f"{where}: {STATUS.get(self.status, self.status)}")


class Params(ctypes.Structure):
    """cil_params: cell_size (0 = from data), cell_scale (0 = 1.5), block,
    topk (0 = default, 1 = register list, 2 = shared-memory heap, 3 =
    warp-staged)."""
    _fields_ = [("cell_size", ctypes.c_float), ("cell_scale", ctypes.c_float),
                ("block", ctypes.c_int), ("topk", ctypes.c_int)]


class BatchParams(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int), ("iters", ctypes.c_int), ("max_corr_dist", ctypes.c_float),
                ("viewpoint", ctypes.c_float * 3), ("tune", Params)]


class IcpReport(ctypes.Structure):
    _fields_ = [("rmse", ctypes.c_double), ("n_inliers", ctypes.c_int64),
                ("iters_done", ctypes.c_int), ("status", ctypes.c_int)]


def lib():
    """Load libcil.so (building it first if it is absent or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        from . import build as _build
        path = _build.build()
        L = ctypes.CDLL(path)
        P, I64, I, F = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_float
        L.cil_status_string.argtypes = [I]
        L.cil_status_string.restype = ctypes.c_char_p
        L.cil_sync_status.argtypes = [P]
        L.cil_knn.argtypes = [P, I64, P, I64, I, P, P, P]
        L.cil_knn_ex.argtypes = [P, I64, P, I64, I, P, P, P, P]
        L.cil_radius_search.argtypes = [P, I64, P, I64, F, P, P, P, I64, P, P]
        L.cil_radius_search_ex.argtypes = [P, I64, P, I64, F, P, P, P, I64, P, P, P]
        L.cil_estimate_normals.argtypes = [P, I64, I, P, P, P, P]
        L.cil_estimate_normals_ex.argtypes = [P, I64, I, P, P, P, P, P]
        L.cil_icp_point_to_plane.argtypes = [P, I64, P, P, I64, P, I, F, P, P, P]
        L.cil_icp.argtypes = [P, I64, P, P, I64, P, I, F, P, P, P, P]
        L.cil_icp_sums.argtypes = [P, I64, P, P, I64, P, I, F, P, P, P, P, P]
        L.cil_segment.argtypes = [P, P, I64, I, F, F, P, P, P]
        L.cil_test_fail_next_allocations.argtypes = [I]
        L.cil_test_fail_next_allocations.restype = None
        L.cil_check_bounded_wait.argtypes = [ctypes.c_uint, P]
        L.cil_smooth_segment.argtypes = [P, I64, I, P, F, F, P, P, P, P]
        L.cil_register_pair.argtypes = [P, I64, P, I64, I, P, P, I, F, P, P, P, P, P]
        L.cil_icp_batch_create.argtypes = [P, P, I, P, P]
        L.cil_icp_batch_run.argtypes = [P, P, P, P, P, P, P, P]
        L.cil_icp_batch_destroy.argtypes = [P]
        L.cil_icp_batch_fallback.argtypes = [P, P, P, ctypes.c_double, P, P, P, P]
        L.cil_icp_batch_destroy.restype = None
        L.cil_launch_count.restype = I64
        L.cil_knn_hybrid.argtypes = [P, I64, P, I64, I, F, P, P, P]
        L.cil_knn_hybrid.restype = I
        L.cil_estimate_normals_radius.argtypes = [P, I64, F, P, P, P, P, P]
        L.cil_estimate_normals_radius.restype = I
        L.cil_voxel_downsample.argtypes = [P, I64, F, P, P, P, P]
        L.cil_voxel_downsample.restype = I
        L.cil_pointnet_num_params.restype = I
        L.cil_pointnet_create.argtypes = [I, I, P]
        L.cil_pointnet_destroy.argtypes = [P]
        L.cil_pointnet_destroy.restype = None
        L.cil_pointnet_set_params.argtypes = [P, P, P]
        L.cil_pointnet_get_params.argtypes = [P, P, P]
        L.cil_pointnet_forward.argtypes = [P, P, I, P, P, P]
        L.cil_pointnet_backward.argtypes = [P, P, P, I, P, P, P]
        L.cil_pointnet_adam_step.argtypes = [P, F, P]
        L.cil_timing_enable.argtypes = [I]
        L.cil_timing_enable.restype = None
        L.cil_timing_read.argtypes = [ctypes.c_char_p, P, P]
        L.cil_timing_reset.restype = None
        for name in ("cil_sync_status", "cil_knn", "cil_knn_ex", "cil_radius_search",
                     "cil_estimate_normals", "cil_estimate_normals_ex", "cil_icp_point_to_plane",
                     "cil_register_pair", "cil_icp_batch_create", "cil_icp_batch_run",
                     "cil_timing_read", "cil_pointnet_create", "cil_pointnet_set_params",
                     "cil_pointnet_get_params", "cil_pointnet_forward", "cil_pointnet_backward",
                     "cil_pointnet_adam_step"):
            getattr(L, name).restype = I
        _lib = L
        return L


# ---------------------------------------------------------------------------
# marshalling helpers
# ---------------------------------------------------------------------------
def _torch():
    import torch
    return torch


def _stream(stream=None):
    torch = _torch()
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _points(t, name):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float32 or t.dim() != 2 or t.shape[1] != 3:
        raise ValueError(f"{name} must be float32 of shape (N, 3)")
    return t.contiguous()


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr() if t is not None and t.numel() > 0 else 0)


def _check(st, where):
    if st != 0:
        raise CilError(st, where)


def _params(cell_size=0.0, cell_scale=0.0, block=0, topk=0):
    if not (cell_size or cell_scale or block or topk):
        return None
    return Params(float(cell_size), float(cell_scale), int(block), int(topk))


# ---------------------------------------------------------------------------
# public calls
# ---------------------------------------------------------------------------
def sync_status(stream=None) -> int:
    """Synchronise the stream and return (and clear) the device error word."""
    return int(lib().cil_sync_status(_stream(stream)))


def knn(ref, qry, k: int, *, cell_size=0.0, cell_scale=0.0, block=0, topk=0, with_d2=True,
        stream=None, out_idx=None, out_d2=None):
    """k nearest neighbours (cil_knn): (idx int32 (Nq,k), d2 float32 (Nq,k))."""
    torch = _torch()
    ref = _points(ref, "ref")
    same = qry is ref
    qry = ref if same else _points(qry, "qry")
    nq = qry.shape[0]
    if out_idx is None:
        out_idx = torch.empty((nq, k), dtype=torch.int32, device=qry.device)
    if with_d2 and out_d2 is None:
        out_d2 = torch.empty((nq, k), dtype=torch.float32, device=qry.device)
    prm = _params(cell_size, cell_scale, block, topk)
    st = lib().cil_knn_ex(_ptr(ref), ref.shape[0], _ptr(qry), nq, int(k), _ptr(out_idx),
                          _ptr(out_d2) if with_d2 else None,
                          ctypes.byref(prm) if prm is not None else None, _stream(stream))
    _check(st, "cil_knn")
    return out_idx, out_d2


def knn_hybrid(ref, qry, k: int, r: float, stream=None):
    """k nearest neighbours within radius r (cil_knn_hybrid): (idx, d2), rows
    padded with -1 / inf where the ball holds fewer than k points."""
    torch = _torch()
    ref = _points(ref, "ref")
    qry = ref if qry is ref else _points(qry, "qry")
    nq = qry.shape[0]
    idx = torch.empty((nq, k), dtype=torch.int32, device=qry.device)
    d2 = torch.empty((nq, k), dtype=torch.float32, device=qry.device)
    st = lib().cil_knn_hybrid(_ptr(ref), ref.shape[0], _ptr(qry), nq, int(k), float(r), _ptr(idx),
                              _ptr(d2), _stream(stream))
    _check(st, "cil_knn_hybrid")
    return idx, d2


def estimate_normals_radius(xyz, r: float, viewpoint, stream=None):
    """PCA normals over radius-r neighbourhoods (cil_estimate_normals_radius):
    (normals, curvature, neighbour counts)."""
    torch = _torch()
    xyz = _points(xyz, "xyz")
    n = xyz.shape[0]
    nrm = torch.empty((n, 3), dtype=torch.float32, device=xyz.device)
    cur = torch.empty(n, dtype=torch.float32, device=xyz.device)
    cnt = torch.empty(n, dtype=torch.int32, device=xyz.device)
    vp = (ctypes.c_float * 3)(*[float(v) for v in np.asarray(viewpoint, np.float64).reshape(3)])
    st = lib().cil_estimate_normals_radius(_ptr(xyz), n, float(r), vp, _ptr(nrm), _ptr(cur),
                                           _ptr(cnt), _stream(stream))
    _check(st, "cil_estimate_normals_radius")
    return nrm, cur, cnt


def voxel_downsample(xyz, voxel: float, stream=None):
    """Voxel-grid downsampling (cil_voxel_downsample): (means (M,3), counts (M,))."""
    torch = _torch()
    xyz = _points(xyz, "xyz")
    n = xyz.shape[0]
    out = torch.empty((max(n, 1), 3), dtype=torch.float32, device=xyz.device)
    cnt = torch.empty(max(n, 1), dtype=torch.int32, device=xyz.device)
    m = ctypes.c_int64(0)
    st = lib().cil_voxel_downsample(_ptr(xyz), n, float(voxel), _ptr(out), _ptr(cnt),
                                    ctypes.byref(m), _stream(stream))
    _check(st, "cil_voxel_downsample")
    return out[:m.value], cnt[:m.value]


def radius_search(ref, qry, r: float, capacity: int | None = None, *, cell_size=0.0,
                  cell_scale=0.0, stream=None):
    """All neighbours within r (cil_radius_search_ex): CSR (offsets int64, idx
    int32, d2 float32).  With capacity=None the call is made twice if needed:
    first to learn the size, then to fill.  cell_size / cell_scale: the
    search cells' edge (default r; results do not depend on it)."""
    torch = _torch()
    ref = _points(ref, "ref")
    qry = ref if qry is ref else _points(qry, "qry")
    nq = qry.shape[0]
    off = torch.empty(nq + 1, dtype=torch.int64, device=qry.device)
    cap = int(capacity) if capacity is not None else 0
    idx = torch.empty(max(cap, 1), dtype=torch.int32, device=qry.device)
    d2 = torch.empty(max(cap, 1), dtype=torch.float32, device=qry.device)
    nnz = ctypes.c_int64(0)
    L = lib()
    prm = _params(cell_size, cell_scale)
    pp = ctypes.byref(prm) if prm is not None else None
    st = L.cil_radius_search_ex(_ptr(ref), ref.shape[0], _ptr(qry), nq, float(r), _ptr(off),
                                _ptr(idx), _ptr(d2), cap, ctypes.byref(nnz), pp, _stream(stream))
    if st == 4 and capacity is None:
        cap = int(nnz.value)
        idx = torch.empty(max(cap, 1), dtype=torch.int32, device=qry.device)
        d2 = torch.empty(max(cap, 1), dtype=torch.float32, device=qry.device)
        st = L.cil_radius_search_ex(_ptr(ref), ref.shape[0], _ptr(qry), nq, float(r), _ptr(off),
                                    _ptr(idx), _ptr(d2), cap, ctypes.byref(nnz), pp,
                                    _stream(stream))
    _check(st, "cil_radius_search")
    n = int(nnz.value)
    return off, idx[:n], d2[:n]


def estimate_normals(xyz, k: int, viewpoint, *, cell_size=0.0, cell_scale=0.0, block=0, topk=0,
                     stream=None, out_normals=None, out_curvature=None, with_curvature=True):
    """PCA normals + curvature (cil_estimate_normals)."""
    torch = _torch()
    xyz = _points(xyz, "xyz")
    n = xyz.shape[0]
    if out_normals is None:
        out_normals = torch.empty((n, 3), dtype=torch.float32, device=xyz.device)
    if with_curvature and out_curvature is None:
        out_curvature = torch.empty(n, dtype=torch.float32, device=xyz.device)
    vp = (ctypes.c_float * 3)(*[float(v) for v in np.asarray(viewpoint, np.float64).reshape(3)])
    prm = _params(cell_size, cell_scale, block, topk)
    st = lib().cil_estimate_normals_ex(_ptr(xyz), n, int(k), vp, _ptr(out_normals),
                                       _ptr(out_curvature) if with_curvature else None,
                                       ctypes.byref(prm) if prm is not None else None,
                                       _stream(stream))
    _check(st, "cil_estimate_normals")
    return out_normals, out_curvature


def icp_point_to_plane(src, dst, dst_normals, T_init=None, iters: int = 20,
                       max_corr_dist: float = 0.1, stream=None):
    """Rigid point-to-plane ICP (cil_icp_point_to_plane).  Returns (T 4x4
    float64 numpy, report dict).  A degenerate round is reported in
    report['status'], not raised."""
    src = _points(src, "src")
    dst = _points(dst, "dst")
    nrm = _points(dst_normals, "dst_normals")
    if nrm.shape != dst.shape:
        raise ValueError("dst_normals must match dst")
    T0 = None
    if T_init is not None:
        T0 = (ctypes.c_double * 16)(*np.asarray(T_init, np.float64).reshape(16).tolist())
    Tout = (ctypes.c_double * 16)()
    rep = IcpReport()
    st = lib().cil_icp_point_to_plane(_ptr(src), src.shape[0], _ptr(dst), _ptr(nrm), dst.shape[0],
                                      T0, int(iters), float(max_corr_dist), Tout,
                                      ctypes.byref(rep), _stream(stream))
    _check(st, "cil_icp_point_to_plane")
    return np.array(Tout[:], np.float64).reshape(4, 4), {
        "rmse": rep.rmse, "n_inliers": int(rep.n_inliers), "iters_done": rep.iters_done,
        "status": rep.status}


class IcpOptions(ctypes.Structure):
    _fields_ = [("metric", ctypes.c_int), ("w_point", ctypes.c_float), ("w_plane", ctypes.c_float),
                ("association", ctypes.c_int), ("pixel_map", ctypes.c_void_p),
                ("width", ctypes.c_int), ("height", ctypes.c_int), ("fx", ctypes.c_float),
                ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float)]


METRICS = {"point_to_plane": 0, "point_to_point": 1, "combined": 2}
ASSOCIATIONS = {"nearest": 0, "projective": 1}


def icp(src, dst, dst_normals=None, T_init=None, iters: int = 20, max_corr_dist: float = 0.1, *,
        metric: str = "point_to_plane", w_point: float = 0.0, w_plane: float = 1.0,
        association: str = "nearest", pixel_map=None, intrinsics=None, with_sums: bool = False,
        stream=None):
    """Rigid ICP with a chosen metric and correspondence search (cil_icp).
    metric: point_to_plane | point_to_point | combined (weights w_point,
    w_plane); association: nearest | projective (pixel_map: int32 CUDA tensor
    (height, width) of target point indices or -1; intrinsics (fx, fy, cx,
    cy)).  Returns (T 4x4 float64 numpy, report dict); with_sums=True
    (cil_icp_sums) adds report['sums'], float64 (iters + 1, 29): each round's
    H upper triangle (21), g (6), sum r^2 and inlier count."""
    src = _points(src, "src")
    dst = _points(dst, "dst")
    nrm = None
    if dst_normals is not None:
        nrm = _points(dst_normals, "dst_normals")
        if nrm.shape != dst.shape:
            raise ValueError("dst_normals must match dst")
    o = IcpOptions()
    o.metric = METRICS[metric]
    o.w_point = float(w_point)
    o.w_plane = float(w_plane)
    o.association = ASSOCIATIONS[association]
    if association == "projective":
        torch = _torch()
        if pixel_map is None or intrinsics is None:
            raise ValueError("projective association needs pixel_map and intrinsics")
        if pixel_map.dtype != torch.int32 or pixel_map.dim() != 2 or not pixel_map.is_cuda:
            raise ValueError("pixel_map must be an int32 CUDA tensor (height, width)")
        pixel_map = pixel_map.contiguous()
        o.pixel_map = pixel_map.data_ptr()
        o.height, o.width = int(pixel_map.shape[0]), int(pixel_map.shape[1])
        o.fx, o.fy, o.cx, o.cy = [float(v) for v in intrinsics]
    T0 = None
    if T_init is not None:
        T0 = (ctypes.c_double * 16)(*np.asarray(T_init, np.float64).reshape(16).tolist())
    Tout = (ctypes.c_double * 16)()
    rep = IcpReport()
    args = (_ptr(src), src.shape[0], _ptr(dst), _ptr(nrm) if nrm is not None else None,
            dst.shape[0], T0, int(iters), float(max_corr_dist), ctypes.byref(o), Tout,
            ctypes.byref(rep))
    sums = None
    if with_sums:
        sums = np.zeros((int(iters) + 1, 29), np.float64)
        st = lib().cil_icp_sums(*args, sums.ctypes.data_as(ctypes.c_void_p), _stream(stream))
        _check(st, "cil_icp_sums")
    else:
        st = lib().cil_icp(*args, _stream(stream))
        _check(st, "cil_icp")
    out = {"rmse": rep.rmse, "n_inliers": int(rep.n_inliers), "iters_done": rep.iters_done,
           "status": rep.status}
    if sums is not None:
        out["sums"] = sums
    return np.array(Tout[:], np.float64).reshape(4, 4), out


def segment(xyz, normals, k: int = 30, theta: float = 2.8, radius: float = 0.0, stream=None):
    """Connected components of the k-NN graph under the normal-angle (and
    optional distance) similarity (cil_segment).  Returns (labels int32 CUDA
    tensor: smallest index of each point's component, number of components)."""
    torch = _torch()
    xyz = _points(xyz, "xyz")
    nrm = _points(normals, "normals")
    if nrm.shape != xyz.shape:
        raise ValueError("normals must match xyz")
    labels = torch.empty(xyz.shape[0], dtype=torch.int32, device=xyz.device)
    count = ctypes.c_int64()
    st = lib().cil_segment(_ptr(xyz), _ptr(nrm), xyz.shape[0], int(k), float(theta), float(radius),
                           _ptr(labels), ctypes.byref(count), _stream(stream))
    _check(st, "cil_segment")
    return labels, int(count.value)


def smooth_segment(xyz, k: int = 30, viewpoint=(0.0, 0.0, 0.0), theta: float = 2.8,
                   radius: float = 0.0, stream=None):
    """PCA normals and smooth segments from one k-NN search
    (cil_smooth_segment): (normals (N,3), labels int32, number of segments)."""
    torch = _torch()
    xyz = _points(xyz, "xyz")
    n = xyz.shape[0]
    nrm = torch.empty((n, 3), dtype=torch.float32, device=xyz.device)
    labels = torch.empty(n, dtype=torch.int32, device=xyz.device)
    vp = (ctypes.c_float * 3)(*[float(v) for v in np.asarray(viewpoint, np.float64).reshape(3)])
    count = ctypes.c_int64()
    st = lib().cil_smooth_segment(_ptr(xyz), n, int(k), vp, float(theta), float(radius), _ptr(nrm),
                                  _ptr(labels), ctypes.byref(count), _stream(stream))
    _check(st, "cil_smooth_segment")
    return nrm, labels, int(count.value)


def register_pair(src, dst, k: int, viewpoint, iters: int, max_corr_dist: float, *,
                  T_init=None, out_normals=None, out_T=None, out_report=None, cell_size=0.0,
                  cell_scale=0.0, block=0, topk=0, stream=None):
    """Target grid + k-NN normals + ICP in one enqueue (cil_register_pair).
    Everything stays on the device: returns (T (16,) float64 CUDA tensor,
    report (cil_icp_report bytes in a uint8 CUDA tensor, decode with
    decode_report), normals)."""
    torch = _torch()
    src = _points(src, "src")
    dst = _points(dst, "dst")
    dev = dst.device
    if out_T is None:
        out_T = torch.empty(16, dtype=torch.float64, device=dev)
    if out_report is None:
        out_report = torch.empty(ctypes.sizeof(IcpReport), dtype=torch.uint8, device=dev)
    vp = (ctypes.c_float * 3)(*[float(v) for v in np.asarray(viewpoint, np.float64).reshape(3)])
    prm = _params(cell_size, cell_scale, block, topk)
    st = lib().cil_register_pair(_ptr(src), src.shape[0], _ptr(dst), dst.shape[0], int(k), vp,
                                 _ptr(T_init) if T_init is not None else None, int(iters),
                                 float(max_corr_dist), _ptr(out_normals), _ptr(out_T),
                                 _ptr(out_report), ctypes.byref(prm) if prm is not None else None,
                                 _stream(stream))
    _check(st, "cil_register_pair")
    return out_T, out_report, out_normals


def decode_report(buf) -> dict:
    """Decode a cil_icp_report held in a (host or device) uint8 tensor."""
    raw = bytes(buf.cpu().numpy().tobytes()) if hasattr(buf, "cpu") else bytes(buf)
    rep = IcpReport.from_buffer_copy(raw[: ctypes.sizeof(IcpReport)])
    return {"rmse": rep.rmse, "n_inliers": int(rep.n_inliers), "iters_done": rep.iters_done,
            "status": rep.status}


def decode_reports(buf, B: int) -> list:
    raw = bytes(buf.cpu().numpy().tobytes()) if hasattr(buf, "cpu") else bytes(buf)
    sz = ctypes.sizeof(IcpReport)
    out = []
    for b in range(B):
        rep = IcpReport.from_buffer_copy(raw[b * sz:(b + 1) * sz])
        out.append({"rmse": rep.rmse, "n_inliers": int(rep.n_inliers),
                    "iters_done": rep.iters_done, "status": rep.status})
    return out


class Batch:
    """Batched registration handle (cil_icp_batch_*): B pairs of uneven sizes,
    one graph launch per run.  Inputs are the pairs' clouds concatenated."""

    def __init__(self, n_src, n_dst, *, k: int = 10, iters: int = 30, max_corr_dist: float = 0.1,
                 viewpoint=(0.0, 0.0, 10.0), cell_size=0.0, cell_scale=0.0, block=0, topk=0):
        self.n_src = np.ascontiguousarray(n_src, np.int64)
        self.n_dst = np.ascontiguousarray(n_dst, np.int64)
        if self.n_src.shape != self.n_dst.shape or self.n_src.ndim != 1:
            raise ValueError("n_src and n_dst must be 1-D of equal length")
        self.B = int(self.n_src.shape[0])
        self.params = BatchParams(int(k), int(iters), float(max_corr_dist),
                                  (ctypes.c_float * 3)(*[float(v) for v in viewpoint]),
                                  Params(float(cell_size), float(cell_scale), int(block),
                                         int(topk)))
        h = ctypes.c_void_p()
        st = lib().cil_icp_batch_create(self.n_src.ctypes.data_as(ctypes.c_void_p),
                                        self.n_dst.ctypes.data_as(ctypes.c_void_p), self.B,
                                        ctypes.byref(self.params), ctypes.byref(h))
        _check(st, "cil_icp_batch_create")
        self._h = h

    def run(self, src_cat, dst_cat, T_init=None, T_out=None, rep=None, normals_out=None,
            stream=None):
        torch = _torch()
        src_cat = _points(src_cat, "src_cat")
        dst_cat = _points(dst_cat, "dst_cat")
        if src_cat.shape[0] != int(self.n_src.sum()) or dst_cat.shape[0] != int(self.n_dst.sum()):
            raise ValueError("concatenated sizes do not match the handle")
        dev = dst_cat.device
        if T_out is None:
            T_out = torch.empty((self.B, 16), dtype=torch.float64, device=dev)
        if rep is None:
            rep = torch.empty((self.B, ctypes.sizeof(IcpReport)), dtype=torch.uint8, device=dev)
        st = lib().cil_icp_batch_run(self._h, _ptr(src_cat), _ptr(dst_cat),
                                     _ptr(T_init) if T_init is not None else None, _ptr(T_out),
                                     _ptr(rep), _ptr(normals_out), _stream(stream))
        _check(st, "cil_icp_batch_run")
        return T_out, rep

    def fallback(self, src_cat, dst_cat, T_out, rep, rmse_threshold: float = 0.005,
                 used_out=None, stream=None):
        """After run(..., T_init=warm start): re-register from the identity
        the pairs whose final RMSE is >= rmse_threshold (or NaN) and keep the
        better result in T_out / rep (cil_icp_batch_fallback).  Returns the
        int32 CUDA tensor `used` (0 kept, 1 re-registered but kept, 2
        replaced)."""
        torch = _torch()
        src_cat = _points(src_cat, "src_cat")
        dst_cat = _points(dst_cat, "dst_cat")
        if used_out is None:
            used_out = torch.empty(self.B, dtype=torch.int32, device=dst_cat.device)
        st = lib().cil_icp_batch_fallback(self._h, _ptr(src_cat), _ptr(dst_cat),
                                          float(rmse_threshold), _ptr(T_out), _ptr(rep),
                                          _ptr(used_out), _stream(stream))
        _check(st, "cil_icp_batch_fallback")
        return used_out

    def close(self):
        if getattr(self, "_h", None):
            lib().cil_icp_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class PointNet:
    """Learned warm start (cil_pointnet_*): a PointNet-style regressor of the
    source -> target transform with hand-written BF16 tensor-core forward,
    sparse max-pool backward and Adam.  Clouds are (B, 2, P, 3) float32 CUDA
    tensors (source, target per pair)."""

    def __init__(self, max_pairs: int, n_points: int = 4096, params=None):
        torch = _torch()
        L = lib()
        self.n_params = int(L.cil_pointnet_num_params())
        self.max_pairs = int(max_pairs)
        self.P = int(n_points)
        h = ctypes.c_void_p()
        _check(L.cil_pointnet_create(self.max_pairs, self.P, ctypes.byref(h)), "cil_pointnet_create")
        self._h = h
        if params is not None:
            self.set_params(params)

    def set_params(self, params, stream=None):
        torch = _torch()
        t = torch.as_tensor(params, dtype=torch.float32).reshape(-1).cuda().contiguous()
        if t.numel() != self.n_params:
            raise ValueError(f"expected {self.n_params} parameters")
        self._params_keep = t
        _check(lib().cil_pointnet_set_params(self._h, _ptr(t), _stream(stream)),
               "cil_pointnet_set_params")

    def get_params(self, stream=None):
        torch = _torch()
        out = torch.empty(self.n_params, dtype=torch.float32, device="cuda")
        _check(lib().cil_pointnet_get_params(self._h, _ptr(out), _stream(stream)),
               "cil_pointnet_get_params")
        return out

    def forward(self, clouds, T_out=None, feat_out=None, stream=None):
        torch = _torch()
        B = int(clouds.shape[0])
        if clouds.dtype != torch.float32 or tuple(clouds.shape[1:]) != (2, self.P, 3):
            raise ValueError("clouds must be float32 (B, 2, P, 3)")
        clouds = clouds.contiguous()
        if T_out is None:
            T_out = torch.empty((B, 16), dtype=torch.float64, device=clouds.device)
        _check(lib().cil_pointnet_forward(self._h, _ptr(clouds), B, _ptr(T_out), _ptr(feat_out),
                                          _stream(stream)), "cil_pointnet_forward")
        return T_out

    def backward(self, clouds, T_gt, loss_out=None, grad_out=None, stream=None):
        torch = _torch()
        B = int(clouds.shape[0])
        clouds = clouds.contiguous()
        T_gt = T_gt.reshape(B, 16).to(torch.float64).contiguous()
        if loss_out is None:
            loss_out = torch.empty(B, dtype=torch.float32, device=clouds.device)
        _check(lib().cil_pointnet_backward(self._h, _ptr(clouds), _ptr(T_gt), B, _ptr(loss_out),
                                           _ptr(grad_out), _stream(stream)),
               "cil_pointnet_backward")
        return loss_out, grad_out

    def adam_step(self, lr: float, stream=None):
        _check(lib().cil_pointnet_adam_step(self._h, float(lr), _stream(stream)),
               "cil_pointnet_adam_step")

    def close(self):
        if getattr(self, "_h", None):
            lib().cil_pointnet_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
