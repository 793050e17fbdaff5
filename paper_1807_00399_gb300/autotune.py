"""Autotuner for batched registration (cil_icp_batch_*).

Searches the grid cell-size multiplier (the cell edge is the nearest
power-of-two multiple of each cloud's fine lattice to scale x the data-driven
neighbourhood radius, so scales 1 / 1.5 / 2 select the estimate's level or
the one above, depending on where the estimate falls between two levels; 1.5
is the library default) and the query-kernel block size, timing whole batch
runs with CUDA events.  The winner is cached as JSON keyed by GPU name
and a size bucket (pairs rounded up to a power of two, mean cloud size to the
nearest power of two, k, rounds), in $CIL_TUNE_CACHE or
~/.cache/cil_gb300/tuning.json.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np

SCALES = (1.0, 1.5, 2.0)
BLOCKS = (64, 128, 256)


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


def tune_batch(src_cat, dst_cat, n_src, n_dst, *, k: int = 10, iters: int = 30,
               max_corr_dist: float = 0.1, viewpoint=(0.0, 0.0, 10.0), reps: int = 3,
               use_cache: bool = True, scales=SCALES, blocks=BLOCKS) -> dict:
    """Return {"cell_scale", "block", "ms", "key", "table", "cached"} for the
    fastest configuration of this batch shape."""
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
    table = []
    for sc in scales:
        for bl in blocks:
            h = Batch(n_src, n_dst, k=k, iters=iters, max_corr_dist=max_corr_dist,
                      viewpoint=viewpoint, cell_scale=sc, block=bl)
            ms = time_batch(h, src_cat, dst_cat, reps=reps)
            h.close()
            table.append({"cell_scale": sc, "block": bl, "ms": ms})
    best = min(table, key=lambda r: r["ms"])
    out = {"cell_scale": best["cell_scale"], "block": best["block"], "ms": best["ms"],
           "table": table}
    if use_cache:
        data[key] = out
        _store(path, data)
    out = dict(out)
    out["cached"] = False
    out["key"] = key
    return out
