"""Training, checkpointing and evaluation of the learned ICP warm start.

The network and its kernels live in libcil (cil_pointnet_*, bound as
``paper_1807_00399_gb300.PointNet``).  This module only drives them:

* ``make_batch``: seeded training pairs generated on the GPU with torch random
  ops -- points uniform in (x, y) on [-1, 1]^2 on z = 0.1 sin(4x) cos(4y) with
  N(0, 0.002) noise, drawn independently for source and target (P points each,
  the distribution of a P-point subsample of a 10,000-point cloud), the source
  moved by a rigid transform with a uniform random axis, angle uniform in
  [0, 90] deg and translation uniform in [-0.5, 0.5]^3; the label maps source
  to target (the inverse of that motion).
* ``train``: Adam with cosine learning-rate decay, one library call for the
  forward + loss + backward and one for the update per step.
* ``evaluate``: on held-out pairs, predict T_init, run batched point-to-plane
  ICP from it and from identity, fall back to the identity result when the
  warm-started RMSE misses the success threshold, and report success rates
  (final point-to-plane RMSE < 0.005) and throughput.
"""
from __future__ import annotations

import json
import math
import os
import time

import numpy as np

SUCCESS_RMSE = 0.005

# Parameter layout of the network (the order of cil_pointnet_set_params):
# shared MLP 3 -> 64 -> 128 -> 256 on each cloud, max-pool, head 512 -> 256 -> 9.
LAYOUT = (("W1", (64, 3)), ("b1", (64,)), ("W2", (128, 64)), ("b2", (128,)),
          ("W3", (256, 128)), ("b3", (256,)), ("W4", (256, 512)), ("b4", (256,)),
          ("W5", (9, 256)), ("b5", (9,)))
CHECKPOINT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "warmstart")


def init_params(seed: int = 0) -> np.ndarray:
    """He-uniform weights and zero biases; the last layer starts near zero with
    a bias that makes the initial prediction the identity (6-D rotation
    (e1, e2), zero translation).  Flat float32 in LAYOUT order."""
    rng = np.random.default_rng(seed)
    out = []
    for name, shape in LAYOUT:
        if name.startswith("W"):
            lim = math.sqrt(6.0 / shape[1])
            w = rng.uniform(-lim, lim, shape)
            out.append((w * 1e-2 if name == "W5" else w).ravel())
        elif name == "b5":
            out.append(np.array([1.0, 0, 0, 0, 1.0, 0, 0, 0, 0]))
        else:
            out.append(np.zeros(shape))
    return np.concatenate(out).astype(np.float32)


def _rotations(u, angle):
    """Rotation matrices from unit axes u (B,3) and angles (B,) (Rodrigues,
    scene generation only)."""
    import torch
    K = torch.zeros(u.shape[0], 3, 3, dtype=u.dtype, device=u.device)
    K[:, 0, 1], K[:, 0, 2] = -u[:, 2], u[:, 1]
    K[:, 1, 0], K[:, 1, 2] = u[:, 2], -u[:, 0]
    K[:, 2, 0], K[:, 2, 1] = -u[:, 1], u[:, 0]
    s = torch.sin(angle)[:, None, None]
    c = torch.cos(angle)[:, None, None]
    eye = torch.eye(3, dtype=u.dtype, device=u.device).expand_as(K)
    return eye + s * K + (1 - c) * (K @ K)


def make_batch(gen, B: int, P: int = 4096, max_angle_deg: float = 90.0, max_trans: float = 0.5,
               noise: float = 0.002, device="cuda"):
    """Returns clouds (B, 2, P, 3) float32 and labels T_gt (B, 16) float64."""
    import torch
    f64 = torch.float64

    def surface(n):
        xy = torch.rand(B, n, 2, generator=gen, device=device, dtype=f64) * 2 - 1
        z = 0.1 * torch.sin(4 * xy[..., 0]) * torch.cos(4 * xy[..., 1])
        p = torch.cat([xy, z[..., None]], -1)
        return p + noise * torch.randn(B, n, 3, generator=gen, device=device, dtype=f64)

    tgt = surface(P)
    src0 = surface(P)
    u = torch.randn(B, 3, generator=gen, device=device, dtype=f64)
    u = u / u.norm(dim=1, keepdim=True)
    ang = torch.rand(B, generator=gen, device=device, dtype=f64) * math.radians(max_angle_deg)
    R = _rotations(u, ang)
    t = (torch.rand(B, 3, generator=gen, device=device, dtype=f64) * 2 - 1) * max_trans
    src = src0 @ R.transpose(1, 2) + t[:, None, :]
    # label: source -> target = inverse of the motion
    Rt = R.transpose(1, 2)
    T = torch.zeros(B, 4, 4, dtype=f64, device=device)
    T[:, :3, :3] = Rt
    T[:, :3, 3] = -(Rt @ t[:, :, None])[:, :, 0]
    T[:, 3, 3] = 1
    clouds = torch.stack([src, tgt], 1).to(torch.float32).contiguous()
    return clouds, T.reshape(B, 16).contiguous()


def train(net, steps: int, B: int = 256, lr: float = 1e-3, seed: int = 0, log_every: int = 0,
          min_lr_frac: float = 0.05, max_angle_deg: float = 90.0, start_step: int = 0,
          total_steps: int | None = None, gen=None):
    """Train `net` (a PointNet handle) for `steps` Adam steps on fresh batches.
    Returns (history of (step, mean loss), generator)."""
    import torch
    total = total_steps or steps
    if gen is None:
        gen = torch.Generator(device="cuda")
        gen.manual_seed(seed)
    loss = torch.empty(B, dtype=torch.float32, device="cuda")
    hist = []
    for i in range(steps):
        s = start_step + i
        cur = lr * (min_lr_frac + (1 - min_lr_frac) * 0.5 * (1 + math.cos(math.pi * s / total)))
        clouds, T = make_batch(gen, B, net.P, max_angle_deg=max_angle_deg)
        net.backward(clouds, T, loss_out=loss)
        net.adam_step(cur)
        if log_every and (i % log_every == 0 or i == steps - 1):
            hist.append((s, float(loss.mean())))
    return hist, gen


def save_checkpoint(net, path: str, step: int, seed: int, extra=None):
    """Raw little-endian FP32 parameters plus a JSON header."""
    params = net.get_params().cpu().numpy().astype("<f4")
    tmp = path + ".tmp"
    params.tofile(tmp + ".bin")
    os.replace(tmp + ".bin", path + ".bin")
    with open(path + ".json", "w") as fh:
        json.dump({"step": step, "seed": seed, "n_params": int(params.size),
                   "extra": extra or {}}, fh)


def load_checkpoint(net, path: str) -> dict:
    with open(path + ".json") as fh:
        meta = json.load(fh)
    params = np.fromfile(path + ".bin", dtype="<f4")
    net.set_params(params)
    return meta


def rot_err_deg(Ta, Tb):
    """Geodesic rotation angle (deg) between batches of 4x4 transforms."""
    Ra = np.asarray(Ta).reshape(-1, 4, 4)[:, :3, :3]
    Rb = np.asarray(Tb).reshape(-1, 4, 4)[:, :3, :3]
    M = Ra @ np.transpose(Rb, (0, 2, 1))
    c = np.clip((np.trace(M, axis1=1, axis2=2) - 1) / 2, -1, 1)
    return np.degrees(np.arccos(c))


def evaluate(net, pairs, src_sub, dst_sub, iters: int = 30, max_corr_dist: float = 0.1,
             k: int = 10, runs: int = 10):
    """Learned warm start + batched ICP + fallback against batched ICP from
    the identity and against the plain path (one single-pair call per pair,
    in sequence, from the identity), on held-out pairs.  The learned arm is the network's
    forward (encoder + head -> T_init), the batch run from T_init, and the
    library's fallback (pairs with final RMSE >= SUCCESS_RMSE re-registered
    from the identity, the better result kept); the identity arm is the batch
    run from the identity.  Each arm has its own handle (its own captured
    graph); times are medians of `runs` timed repetitions (CUDA events on the
    stream, the fallback's one host read of its tile count included)."""
    import torch

    from . import Batch, decode_reports

    B = len(pairs)
    clouds = torch.from_numpy(np.stack([src_sub, dst_sub], 1)).cuda()
    n = [len(p.source) for p in pairs]
    src = torch.from_numpy(np.concatenate([p.source for p in pairs])).cuda()
    dst = torch.from_numpy(np.concatenate([p.target for p in pairs])).cuda()
    kw = dict(k=k, iters=iters, max_corr_dist=max_corr_dist, viewpoint=(0.0, 0.0, 10.0))
    h_l = Batch(n, [len(p.target) for p in pairs], **kw)
    h_i = Batch(n, [len(p.target) for p in pairs], **kw)
    T_init = torch.empty((B, 16), dtype=torch.float64, device="cuda")
    T_l = torch.empty((B, 16), dtype=torch.float64, device="cuda")
    T_i = torch.empty((B, 16), dtype=torch.float64, device="cuda")
    rep_l = torch.empty((B, 24), dtype=torch.uint8, device="cuda")  # cil_icp_report
    rep_i = torch.empty((B, 24), dtype=torch.uint8, device="cuda")
    used = torch.empty(B, dtype=torch.int32, device="cuda")
    T_warm = torch.empty_like(T_l)
    rep_warm = torch.empty_like(rep_l)

    def learned_arm():
        net.forward(clouds, T_out=T_init)
        h_l.run(src, dst, T_init=T_init, T_out=T_l, rep=rep_l)
        T_warm.copy_(T_l)
        rep_warm.copy_(rep_l)
        h_l.fallback(src, dst, T_l, rep_l, rmse_threshold=SUCCESS_RMSE, used_out=used)

    def identity_arm():
        h_i.run(src, dst, T_init=None, T_out=T_i, rep=rep_i)

    # warm-up (graph capture) outside the timing
    learned_arm()
    identity_arm()
    torch.cuda.synchronize()
    ms = {"learned": [], "identity": []}
    for _ in range(runs):
        for name, fn in (("learned", learned_arm), ("identity", identity_arm)):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            ms[name].append(a.elapsed_time(b))
    ms_learned = float(np.median(ms["learned"]))
    ms_identity = float(np.median(ms["identity"]))
    # the plain path: one single-pair call (grid, normals, 30 rounds) per pair
    # from the identity, in sequence
    from . import register_pair
    offs = np.concatenate([[0], np.cumsum(n)])
    T_p = torch.empty((B, 16), dtype=torch.float64, device="cuda")
    rep_p = torch.empty((B, 24), dtype=torch.uint8, device="cuda")
    nrm = torch.empty_like(dst)

    def plain_arm():
        for b in range(B):
            s0, s1 = int(offs[b]), int(offs[b + 1])
            register_pair(src[s0:s1], dst[s0:s1], k, (0.0, 0.0, 10.0), iters, max_corr_dist,
                          out_normals=nrm[s0:s1], out_T=T_p[b], out_report=rep_p[b])

    plain_arm()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    e = torch.cuda.Event(enable_timing=True)
    a.record()
    plain_arm()
    e.record()
    torch.cuda.synchronize()
    ms_plain = a.elapsed_time(e)
    rp = decode_reports(rep_p, B)
    rl = decode_reports(rep_l, B)
    rw = decode_reports(rep_warm, B)
    ri = decode_reports(rep_i, B)
    used_h = used.cpu().numpy()
    h_l.close()
    h_i.close()
    T_gt = np.stack([p.T_gt for p in pairs]).reshape(B, 16)
    rm_l = np.array([r["rmse"] for r in rl])
    rm_w = np.array([r["rmse"] for r in rw])
    rm_i = np.array([r["rmse"] for r in ri])
    ok_l = np.nan_to_num(rm_l, nan=np.inf) < SUCCESS_RMSE
    ok_w = np.nan_to_num(rm_w, nan=np.inf) < SUCCESS_RMSE
    ok_i = np.nan_to_num(rm_i, nan=np.inf) < SUCCESS_RMSE
    rm_p = np.array([r["rmse"] for r in rp])
    ok_p = np.nan_to_num(rm_p, nan=np.inf) < SUCCESS_RMSE
    return {
        "pairs": B,
        "runs": runs,
        "success_learned_fallback": float(ok_l.mean()),
        "success_learned_before_fallback": float(ok_w.mean()),
        "success_identity": float(ok_i.mean()),
        "pairs_reregistered": int((used_h > 0).sum()),
        "pairs_replaced_by_fallback": int((used_h == 2).sum()),
        "median_rmse_success_learned_fallback": float(np.median(rm_l[ok_l])) if ok_l.any() else None,
        "median_rmse_success_identity": float(np.median(rm_i[ok_i])) if ok_i.any() else None,
        "warm_start_rot_err_deg_median": float(np.median(rot_err_deg(T_init.cpu().numpy(), T_gt))),
        "identity_rot_err_deg_median": float(np.median(rot_err_deg(np.tile(np.eye(4), (B, 1, 1)),
                                                                   T_gt))),
        "final_rot_err_deg_median_learned": float(np.median(rot_err_deg(T_l.cpu().numpy(), T_gt))),
        "ms_learned_fallback": ms_learned,
        "ms_identity_icp": ms_identity,
        "ms_learned_fallback_all": [round(v, 4) for v in ms["learned"]],
        "ms_identity_all": [round(v, 4) for v in ms["identity"]],
        "pairs_per_s_learned_fallback": B / (ms_learned / 1e3),
        "pairs_per_s_identity": B / (ms_identity / 1e3),
        "successful_pairs_per_s_learned_fallback": float(ok_l.sum()) / (ms_learned / 1e3),
        "successful_pairs_per_s_identity": float(ok_i.sum()) / (ms_identity / 1e3),
        "ms_plain_sequential": ms_plain,
        "pairs_per_s_plain": B / (ms_plain / 1e3),
        "success_plain": float(ok_p.mean()),
        "median_rmse_success_plain": float(np.median(rm_p[ok_p])) if ok_p.any() else None,
        "plain_equals_batched_identity": bool(torch.equal(T_p, T_i)),
    }


def check_labels(n_pairs: int = 64, seed: int = 99, iters: int = 30) -> dict:
    """Cross-check of the generator labels by plain ICP: pairs drawn like the
    training pairs (full 10,000-point clouds), registered from their label;
    ICP should barely move a correct label."""
    import torch

    from . import Batch, synth
    pairs, _, _ = synth.warm_start_pairs(seed, n_pairs, n=10_000)
    B = len(pairs)
    src = torch.from_numpy(np.concatenate([p.source for p in pairs])).cuda()
    dst = torch.from_numpy(np.concatenate([p.target for p in pairs])).cuda()
    T_gt = np.stack([p.T_gt for p in pairs]).reshape(B, 16)
    h = Batch([len(p.source) for p in pairs], [len(p.target) for p in pairs], k=10, iters=iters,
              max_corr_dist=0.1, viewpoint=(0.0, 0.0, 10.0))
    T, _ = h.run(src, dst, T_init=torch.from_numpy(T_gt).cuda())
    torch.cuda.synchronize()
    h.close()
    Tn = T.cpu().numpy().reshape(B, 4, 4)
    d_rot = rot_err_deg(Tn, T_gt)
    d_t = np.linalg.norm(Tn[:, :3, 3] - T_gt.reshape(B, 4, 4)[:, :3, 3], axis=1)
    return {"pairs": B, "icp_from_label_rot_change_deg_median": float(np.median(d_rot)),
            "icp_from_label_rot_change_deg_max": float(d_rot.max()),
            "icp_from_label_trans_change_median": float(np.median(d_t))}


def main(argv=None):
    """python -m paper_1807_00399_gb300.learned train|eval ..."""
    import argparse

    import torch

    from . import PointNet, synth
    ap = argparse.ArgumentParser(prog="python -m paper_1807_00399_gb300.learned")
    sub = ap.add_subparsers(dest="cmd", required=True)
    tr = sub.add_parser("train", help="train from the seeded initialisation, write a checkpoint")
    tr.add_argument("--pairs", type=int, default=200_000, help="training pairs (steps = pairs / batch)")
    tr.add_argument("--batch", type=int, default=256)
    tr.add_argument("--lr", type=float, default=1e-3)
    tr.add_argument("--seed", type=int, default=0)
    tr.add_argument("--out", default=CHECKPOINT)
    ev = sub.add_parser("eval", help="held-out evaluation of a checkpoint")
    ev.add_argument("--ckpt", default=CHECKPOINT)
    ev.add_argument("--pairs", type=int, default=256)
    ev.add_argument("--seed", type=int, default=777)
    a = ap.parse_args(argv)
    if a.cmd == "train":
        steps = -(-a.pairs // a.batch)
        net = PointNet(a.batch, 4096, params=init_params(a.seed))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hist, _ = train(net, steps, B=a.batch, lr=a.lr, seed=a.seed, log_every=max(1, steps // 20))
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        extra = {"pairs_seen": steps * a.batch, "batch": a.batch, "lr": a.lr, "wall_s": wall,
                 "loss_history": hist, "label_check": check_labels()}
        os.makedirs(os.path.dirname(os.path.abspath(a.out)), exist_ok=True)
        save_checkpoint(net, a.out, steps, a.seed, extra)
        net.close()
        print(json.dumps({"steps": steps, "wall_s": wall, "first_loss": hist[0][1],
                          "last_loss": hist[-1][1], "label_check": extra["label_check"]}))
    else:
        net = PointNet(a.pairs, 4096)
        meta = load_checkpoint(net, a.ckpt)
        pairs, s_sub, d_sub = synth.warm_start_pairs(a.seed, a.pairs, n=10_000)
        res = evaluate(net, pairs, s_sub, d_sub)
        net.close()
        res["checkpoint_steps"] = meta["step"]
        print(json.dumps(res))


if __name__ == "__main__":
    main()
