"""One invocation of the hot path on a named synthetic workload, for
profilers (ncu) and quick timing.

    python -m paper_1807_00399_gb300.profile_run --workload depth --op register --iters 30
    python -m paper_1807_00399_gb300.profile_run --workload lidar --op radius

Workloads: surface (10,000-point wavy surface pair), depth (640x480 depth
frames, ~3.07e5 points), lidar (64 x 2048 sweep, ~1.2e5 returns), batch (256
surface pairs with sizes log-uniform in [2e3, 2e5]), apartment (7.8M points on
a furnished flat; op segment only).  Ops: register (grid,
k-NN normals and point-to-plane ICP), knn (self k-NN), normals, radius
(radius search), icp (ICP alone on library normals, with --metric and
--association), batch (the batched graph run; workload batch only), voxel
(voxel grid of edge --radius), hybrid (k nearest within --radius),
normals_r (normals over --radius balls), segment
(5 mm voxel grid, then k = 30 normals and smooth segments with a 2.8 rad
angle from one search; workload apartment only).  Each op
runs --repeat times after one warm-up call; the CUDA-event time per call and
the per-kernel times recorded by the library (not inside graph replays) are
printed as one JSON line.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import sys


def main(argv=None):
    ap = argparse.ArgumentParser(prog="python -m paper_1807_00399_gb300.profile_run")
    ap.add_argument("--workload", choices=["surface", "depth", "lidar", "batch", "apartment"],
                    default="depth")
    ap.add_argument("--op", choices=["register", "knn", "normals", "radius", "batch", "icp",
                                     "segment", "voxel", "hybrid", "normals_r"],
                    default="register")
    ap.add_argument("--iters", type=int, default=30, help="ICP iterations")
    ap.add_argument("--k", type=int, default=0, help="neighbours (default: 16 lidar, else 10)")
    ap.add_argument("--radius", type=float, default=0.5)
    ap.add_argument("--cell-scale", type=float, default=0.0,
                    help="grid cell-size multiplier (0: the library default)")
    ap.add_argument("--topk", type=int, default=0,
                    help="k-NN search layout (0 default, 1 list, 2 heap, 3 warp-staged)")
    ap.add_argument("--repeat", type=int, default=1)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--metric", choices=["point_to_plane", "point_to_point", "combined"],
                    default=None, help="op icp: the ICP metric (default point_to_plane)")
    ap.add_argument("--association", choices=["nearest", "projective"], default="nearest",
                    help="op icp: correspondence search (projective: depth workload only)")
    ap.add_argument("--no-regions", action="store_true",
                    help="time the calls only (no per-kernel event records between launches)")
    a = ap.parse_args(argv)

    import torch

    import paper_1807_00399_gb300 as cil
    from paper_1807_00399_gb300 import synth

    k = a.k or {"lidar": 16, "apartment": 30}.get(a.workload, 10)
    if (a.op == "segment") != (a.workload == "apartment"):
        raise SystemExit("op segment runs on the apartment workload, and only it")
    if a.workload == "apartment":
        P = torch.from_numpy(synth.apartment_scene(a.seed)).cuda()

        def fn():
            v, _ = cil.voxel_downsample(P, 0.005)
            return cil.smooth_segment(v, k, synth.APARTMENT_VIEWPOINT, theta=2.8)
    elif a.workload == "batch":
        sizes = synth.batch_sizes(a.seed, 256)
        src, dst, _ = synth.surface_batch_torch(1000 + a.seed, sizes)
        h = cil.Batch(sizes, sizes, k=k, iters=a.iters, max_corr_dist=0.1, viewpoint=(0.0, 0.0, 10.0))
        fn = lambda: h.run(src, dst)  # noqa: E731
    else:
        if a.workload == "surface":
            p, dmax = synth.surface_pair(a.seed, n=10_000), 0.1
        elif a.workload == "depth":
            p, dmax = synth.depth_frame_pair(a.seed), 0.05
        else:
            p, dmax = synth.lidar_sweep_pair(a.seed), 1.0
        src = torch.from_numpy(p.source).cuda()
        dst = torch.from_numpy(p.target).cuda()
        nrm = torch.empty_like(dst)
        vp = p.viewpoint
        icp_kw = {}
        if a.op == "icp":
            # target normals from the library, then ICP alone with the chosen variant
            nrm, _ = cil.estimate_normals(dst, k, vp)
            icp_kw = {"metric": a.metric or "point_to_plane", "association": a.association,
                      "w_point": 0.1, "w_plane": 1.0}
            if a.association == "projective":
                if a.workload != "depth":
                    raise SystemExit("projective association needs the depth workload")
                w, h = p.meta["w"], p.meta["h"]
                pm = torch.full((w * h,), -1, dtype=torch.int32)
                pm[torch.from_numpy(p.meta["target_pixels"]).long()] = torch.arange(
                    len(p.target), dtype=torch.int32)
                icp_kw.update(pixel_map=pm.reshape(h, w).cuda(), intrinsics=p.meta["intrinsics"])
        fn = {
            "icp": lambda: cil.icp(src, dst, nrm, iters=a.iters, max_corr_dist=dmax, **icp_kw),
            "register": lambda: cil.register_pair(src, dst, k, vp, a.iters, dmax, out_normals=nrm,
                                                  cell_scale=a.cell_scale, topk=a.topk),
            "knn": lambda: cil.knn(dst, dst, k, cell_scale=a.cell_scale, topk=a.topk),
            "normals": lambda: cil.estimate_normals(dst, k, vp, cell_scale=a.cell_scale,
                                                    topk=a.topk),
            "radius": lambda: cil.radius_search(dst, dst, a.radius, cell_scale=a.cell_scale),
            "voxel": lambda: cil.voxel_downsample(dst, a.radius),
            "hybrid": lambda: cil.knn_hybrid(dst, dst, k, a.radius),
            "normals_r": lambda: cil.estimate_normals_radius(dst, a.radius, vp),
        }[a.op]
    L = cil.lib()
    fn()
    torch.cuda.synchronize()
    L.cil_timing_reset()
    L.cil_timing_enable(0 if a.no_regions else 1)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.repeat):
        fn()
    e1.record()
    torch.cuda.synchronize()
    L.cil_timing_enable(0)
    out = {"workload": a.workload, "op": a.op, "k": k, "iters": a.iters, "repeat": a.repeat,
           "ms_per_call": e0.elapsed_time(e1) / a.repeat}
    for name in ("grid_build", "order_queries", "k_knn", "k_normals", "k_icp", "k_radius",
                 "voxel_downsample", "segment", "k_knn_hybrid", "k_normals_radius"):
        t, c = ctypes.c_double(), ctypes.c_int64()
        L.cil_timing_read(name.encode(), ctypes.byref(t), ctypes.byref(c))
        if c.value:
            out[name + "_ms"] = t.value / c.value
    print(json.dumps(out))
    return 0


if __name__ == "__main__":
    sys.exit(main())
