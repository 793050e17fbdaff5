"""Autotuner for batched registration (cil_icp_batch_*).

Three knobs, none of which changes a result (the searches are exact whatever
the cell size, block shape or top-k layout; tests check the transforms are
bitwise equal across every configuration tried):
  cell_scale  multiplier on the data-driven cell edge (each cloud's cell is
              the nearest power-of-two multiple of its fine lattice to scale x
              the median k-th neighbour distance of sampled points);
  block       threads per block of the normals kernel (64, 128, 256);
  topk        how the k-NN search runs: 1 = per query, k best in a sorted
              register list; 2 = per query, binary max-heap in shared memory;
              3 = warp-staged (32 queries scan one shared set of points);
              0 = the library's default.
The search is coordinate descent on whole timed batch runs (CUDA events):
the cell scale over SCALES at the default block and layout, extended by
factors of 1.5 past either end while the best scale sits on that end (so the
winner is bracketed), then the block size, then the top-k layout, each at the
best values found so far.  The winner is cached as JSON keyed by GPU name and
a size bucket (pairs rounded up to a power of two, mean cloud size to the
nearest power of two, k, rounds), in $CIL_TUNE_CACHE or
~/.cache/cil_gb300/tuning.json.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np

SCALES = (0.5, 0.75, 1.0, 1.5, 2.0, 3.0, 4.0)
BLOCKS = (64, 128, 256)
TOPK = (1, 2, 3)
SCALE_LIMITS = (0.125, 16.0)  # the range extension stops here


def cache_path() -> str:
    return os.environ.get("CIL_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "cil_gb300", "tuning.json"))


def bucket(n_src, n_dst, k: int, iters: int) -> str:
    B = len(n_src)
    mean = (float(np.sum(n_src)) + float(np.sum(n_dst))) / max(2 * B, 1)
    b2 = 1 << max(0, math.ceil(math.log2(max(B, 1))))
    m2 = 1 << max(0, round(math.log2(max(mean, 1.0))))
    return f"B{b2}-n{m2}-k{k}-i{iters}"


def _load(path):
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _store(path, data):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as fh:
        json.dump(data, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def time_batch(h, src, dst, reps: int = 3, warmup: int = 1) -> float:
    """Median milliseconds of `reps` runs of a Batch handle."""
    import ctypes

    import torch

    from . import IcpReport
    T = torch.empty((h.B, 16), dtype=torch.float64, device=dst.device)
    rep = torch.empty((h.B, ctypes.sizeof(IcpReport)), dtype=torch.uint8, device=dst.device)
    for _ in range(warmup):
        h.run(src, dst, T_out=T, rep=rep)
    ts = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        h.run(src, dst, T_out=T, rep=rep)
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return float(np.median(ts))


def coordinate_descent(time_fn, scales=SCALES, blocks=BLOCKS, topks=TOPK,
                       limits=SCALE_LIMITS, default_block: int = 128, default_topk: int = 0):
    """The search itself, on any cost function time_fn(cell_scale, block,
    topk) -> ms.  Returns (best (scale, block, topk), table of every timed
    configuration in the order tried, whether the best scale is interior to
    the scales tried)."""
    table, seen = [], {}

    def timed(sc, bl, tk):
        cfg = (float(sc), int(bl), int(tk))
        if cfg not in seen:
            seen[cfg] = float(time_fn(*cfg))
            table.append({"cell_scale": cfg[0], "block": cfg[1], "topk": cfg[2], "ms": seen[cfg]})
        return seen[cfg]

    bl0, tk0 = default_block, default_topk
    sc_list = sorted(float(v) for v in scales)
    for sc in sc_list:
        timed(sc, bl0, tk0)
    while True:  # extend past an edge winner until the best scale is bracketed
        best_sc = min(sc_list, key=lambda v: seen[(v, bl0, tk0)])
        if best_sc == sc_list[-1] and sc_list[-1] * 1.5 <= limits[1]:
            sc_list.append(sc_list[-1] * 1.5)
            timed(sc_list[-1], bl0, tk0)
        elif best_sc == sc_list[0] and sc_list[0] / 1.5 >= limits[0]:
            sc_list.insert(0, sc_list[0] / 1.5)
            timed(sc_list[0], bl0, tk0)
        else:
            break
    best_bl = min(blocks, key=lambda b: timed(best_sc, b, tk0))
    if seen[(best_sc, bl0, tk0)] <= seen[(best_sc, best_bl, tk0)]:
        best_bl = bl0
    best_tk = min(topks, key=lambda t: timed(best_sc, best_bl, t))
    if seen[(best_sc, best_bl, tk0)] <= seen[(best_sc, best_bl, best_tk)]:
        best_tk = tk0
    return (best_sc, best_bl, best_tk), table, sc_list[0] < best_sc < sc_list[-1]


def tune_batch(src_cat, dst_cat, n_src, n_dst, *, k: int = 10, iters: int = 30,
               max_corr_dist: float = 0.1, viewpoint=(0.0, 0.0, 10.0), reps: int = 3,
               use_cache: bool = True, scales=SCALES, blocks=BLOCKS, topks=TOPK) -> dict:
    """Return {"cell_scale", "block", "topk", "ms", "scale_interior", "key",
    "table", "cached"} for the fastest configuration of this batch shape
    found by coordinate descent (module docstring); "table" lists every
    configuration timed, in the order tried."""
    import torch

    from . import Batch

    name = torch.cuda.get_device_name()
    key = f"{name}|{bucket(n_src, n_dst, k, iters)}"
    path = cache_path()
    data = _load(path) if use_cache else {}
    if use_cache and key in data:
        out = dict(data[key])
        out["cached"] = True
        out["key"] = key
        return out

    def time_fn(sc, bl, tk):
        h = Batch(n_src, n_dst, k=k, iters=iters, max_corr_dist=max_corr_dist,
                  viewpoint=viewpoint, cell_scale=sc, block=bl, topk=tk)
        ms = time_batch(h, src_cat, dst_cat, reps=reps)
        h.close()
        return ms

    (sc, bl, tk), table, interior = coordinate_descent(time_fn, scales, blocks, topks)
    best_ms = min(r["ms"] for r in table if (r["cell_scale"], r["block"], r["topk"]) == (sc, bl, tk))
    out = {"cell_scale": sc, "block": bl, "topk": tk, "ms": best_ms, "scale_interior": interior,
           "table": table}
    if use_cache:
        data[key] = out
        _store(path, data)
    out = dict(out)
    out["cached"] = False
    out["key"] = key
    return out
