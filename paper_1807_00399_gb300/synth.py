"""Seeded synthetic point-cloud generators.

This module produces the inputs that both the CUDA path and the CPU oracle
consume.  It holds none of the method's arithmetic (no neighbour search, no
covariance, no registration): only scene sampling, ray casting and rigid
motions used to *create* data with a known ground truth.

The paper benchmarks on recorded data (TUM RGB-D fr1/desk VGA frames for
normals and point-to-plane ICP, Sec. 4; a BundleFusion reconstruction for
segmentation).  Those recordings are not available here, so every workload is
a seeded stand-in with the same shape and scale:

* ``surface_pair``  -- a 10,000-point noisy wavy surface and an independently
  resampled, rigidly moved copy (the small single-pair workload);
* ``depth_frame_pair`` -- two 640x480 pinhole depth frames of a box/sphere
  scene, back-projected to about 3e5 points each (stand-in for the paper's VGA
  depth frames, Sec. 4);
* ``lidar_sweep_pair`` -- two 64x2048 spinning-LiDAR sweeps of a box scene;
* ``surface_batch`` -- 256 surface pairs with log-uniform point counts;
* ``warm_start_pairs`` -- surface pairs with large rotations, subsampled to a
  fixed point count (inputs of the learned warm start).

Conventions: points are ``float32`` arrays of shape ``(N, 3)`` (one point per
row, x/y/z interleaved, i.e. the contiguous "one point per column" matrix view
of Sec. 2).  ``T_gt`` is a row-major 4x4 ``float64`` rigid transform that maps
*source* coordinates to *target* coordinates (so ICP started from identity
should converge to it).  All randomness comes from ``numpy.random.default_rng``
seeded by the caller.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "rotation_from_axis_angle",
    "random_rigid",
    "apply_rigid",
    "surface_points",
    "surface_pair",
    "depth_frame_pair",
    "lidar_sweep_pair",
    "surface_batch",
    "warm_start_pairs",
    "lattice_points",
    "Pair",
]


@dataclass
class Pair:
    """A registration problem: ``source`` should be mapped onto ``target``."""

    source: np.ndarray
    target: np.ndarray
    T_gt: np.ndarray  # (4,4) float64, maps source -> target
    viewpoint: np.ndarray = field(default_factory=lambda: np.array([0.0, 0.0, 10.0]))
    meta: dict = field(default_factory=dict)


# ---------------------------------------------------------------------------
# rigid motions (scene construction only)
# ---------------------------------------------------------------------------
def rotation_from_axis_angle(axis, angle) -> np.ndarray:
    """Rotation matrix of ``angle`` radians about ``axis`` built through a unit
    quaternion (w, x, y, z) = (cos a/2, sin a/2 * axis)."""
    axis = np.asarray(axis, dtype=np.float64)
    axis = axis / np.linalg.norm(axis)
    w = math.cos(angle / 2.0)
    x, y, z = math.sin(angle / 2.0) * axis
    return np.array(
        [
            [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
            [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
            [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)],
        ]
    )


def random_rigid(rng, max_angle_deg: float, max_trans: float, trans_mode: str = "cube"):
    """Random rigid transform: axis uniform on the sphere, angle uniform in
    [0, max_angle_deg], translation uniform in the cube [-max_trans, max_trans]^3
    (``trans_mode="cube"``) or with a uniform direction and a length uniform in
    [0, max_trans] (``trans_mode="ball"``)."""
    axis = rng.normal(size=3)
    while np.linalg.norm(axis) < 1e-9:
        axis = rng.normal(size=3)
    angle = math.radians(rng.uniform(0.0, max_angle_deg))
    if trans_mode == "cube":
        t = rng.uniform(-max_trans, max_trans, size=3)
    else:
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        t = d * rng.uniform(0.0, max_trans)
    T = np.eye(4)
    T[:3, :3] = rotation_from_axis_angle(axis, angle)
    T[:3, 3] = t
    return T


def apply_rigid(T: np.ndarray, pts: np.ndarray) -> np.ndarray:
    pts = np.asarray(pts, dtype=np.float64)
    return pts @ T[:3, :3].T + T[:3, 3]


# ---------------------------------------------------------------------------
# workload: small single pair (wavy surface)
# ---------------------------------------------------------------------------
def surface_points(rng, n: int, noise: float = 0.002) -> np.ndarray:
    """n points with (x, y) ~ U[-1,1]^2 on z = 0.1 sin(4x) cos(4y), plus
    isotropic Gaussian noise of standard deviation ``noise`` (float64)."""
    xy = rng.uniform(-1.0, 1.0, size=(n, 2))
    z = 0.1 * np.sin(4.0 * xy[:, 0]) * np.cos(4.0 * xy[:, 1])
    p = np.column_stack([xy, z])
    if noise > 0:
        p = p + rng.normal(0.0, noise, size=p.shape)
    return p


def surface_pair(
    seed: int,
    n: int = 10_000,
    n_src: int | None = None,
    noise: float = 0.002,
    max_angle_deg: float = 10.0,
    max_trans: float = 0.05,
) -> Pair:
    """Target: ``n`` noisy samples of the wavy surface.  Source: an independent
    resample (``n_src`` points, default ``n``) with independent noise, moved by
    a seeded rigid transform T_gen.  ``T_gt = inv(T_gen)``."""
    rng = np.random.default_rng(seed)
    n_src = n if n_src is None else n_src
    target = surface_points(rng, n, noise)
    src0 = surface_points(rng, n_src, noise)
    T_gen = random_rigid(rng, max_angle_deg, max_trans, "cube")
    source = apply_rigid(T_gen, src0)
    return Pair(
        source=source.astype(np.float32),
        target=target.astype(np.float32),
        T_gt=np.linalg.inv(T_gen),
        viewpoint=np.array([0.0, 0.0, 10.0]),
        meta={"kind": "surface", "seed": seed, "n": n, "n_src": n_src},
    )


# ---------------------------------------------------------------------------
# workload: depth frame (pinhole camera, ground + boxes + spheres)
# ---------------------------------------------------------------------------
def _ray_boxes(o, d, lo, hi):
    """Nearest positive hit distance of rays (o + t d) against axis-aligned
    boxes [lo, hi]; returns (n_rays,) with +inf where nothing is hit."""
    n = d.shape[0]
    best = np.full(n, np.inf)
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = 1.0 / d  # (n,3)
    for b in range(lo.shape[0]):
        t1 = (lo[b] - o) * inv
        t2 = (hi[b] - o) * inv
        tmin = np.nanmax(np.minimum(t1, t2), axis=1)
        tmax = np.nanmin(np.maximum(t1, t2), axis=1)
        hit = (tmax >= 0) & (tmax >= tmin) & np.isfinite(tmin)
        t = np.where(tmin > 1e-6, tmin, tmax)
        ok = hit & (t > 1e-6) & (t < best)
        best = np.where(ok, t, best)
    return best


def _ray_spheres(o, d, centers, radii):
    n = d.shape[0]
    best = np.full(n, np.inf)
    dd = np.einsum("ij,ij->i", d, d)
    for c, r in zip(centers, radii):
        oc = o - c
        b = np.einsum("ij,ij->i", d, oc) if oc.ndim == 2 else d @ oc
        cc = (np.einsum("ij,ij->i", oc, oc) if oc.ndim == 2 else oc @ oc) - r * r
        disc = b * b - dd * cc
        ok = disc >= 0
        sq = np.sqrt(np.where(ok, disc, 0.0))
        t0 = (-b - sq) / dd
        t1 = (-b + sq) / dd
        t = np.where(t0 > 1e-6, t0, t1)
        ok = ok & (t > 1e-6) & (t < best)
        best = np.where(ok, t, best)
    return best


def _depth_scene(rng, n_boxes=20, n_spheres=10):
    # footprint seen by a camera 1.5 m above the ground pitched 45 deg down
    bc = np.column_stack(
        [rng.uniform(-1.5, 1.5, n_boxes), rng.uniform(0.8, 3.5, n_boxes)]
    )
    sides = rng.uniform(0.1, 0.6, size=(n_boxes, 3))
    lo = np.column_stack([bc - sides[:, :2] / 2, np.zeros(n_boxes)])
    hi = np.column_stack([bc + sides[:, :2] / 2, sides[:, 2]])
    radii = rng.uniform(0.05, 0.3, n_spheres)
    sc = np.column_stack(
        [rng.uniform(-1.5, 1.5, n_spheres), rng.uniform(0.8, 3.5, n_spheres), radii]
    )
    return lo, hi, sc, radii


def _render_depth(rng, pose_wc, scene, width, height, fx, fy, cx, cy, zmin, zmax,
                  return_pixels: bool = False):
    """Ray-cast a pinhole camera (x right, y down, z forward; pose_wc maps
    camera to world) and back-project the noisy depth to camera-frame points
    (raster order of the valid pixels; with return_pixels also their flat
    pixel indices v * width + u)."""
    lo, hi, sc, radii = scene
    u, v = np.meshgrid(np.arange(width, dtype=np.float64), np.arange(height, dtype=np.float64))
    u = u.ravel()
    v = v.ravel()
    dc = np.column_stack([(u - cx) / fx, (v - cy) / fy, np.ones_like(u)])  # z = 1
    R = pose_wc[:3, :3]
    o = pose_wc[:3, 3]
    dw = dc @ R.T
    t = np.full(dc.shape[0], np.inf)
    with np.errstate(divide="ignore", invalid="ignore"):
        tg = np.where(dw[:, 2] < -1e-12, -o[2] / dw[:, 2], np.inf)
    t = np.minimum(t, np.where(tg > 0, tg, np.inf))
    t = np.minimum(t, _ray_boxes(o[None, :], dw, lo, hi))
    t = np.minimum(t, _ray_spheres(o, dw, sc, radii))
    z = t  # dc has unit z, so the ray parameter is the camera-frame depth
    valid = np.isfinite(z) & (z >= zmin) & (z <= zmax)
    z = z[valid]
    z = z + rng.normal(0.0, 1.0, size=z.shape) * 0.001 * z * z
    pts = dc[valid] * z[:, None]
    if return_pixels:
        return pts, np.nonzero(valid)[0].astype(np.int32)
    return pts


def depth_frame_pair(
    seed: int,
    width: int = 640,
    height: int = 480,
    fx: float = 525.0,
    fy: float = 525.0,
    cx: float = 319.5,
    cy: float = 239.5,
    max_angle_deg: float = 3.0,
    max_trans: float = 0.03,
) -> Pair:
    """Two depth frames of a seeded scene (ground plane, 20 boxes, 10 spheres).
    Camera 1 sits 1.5 m above the ground pitched 45 deg down; camera 2 is camera
    1 moved by a random rotation <= 3 deg and translation <= 3 cm (expressed in
    camera-1 coordinates).  Target = frame 1 points (camera-1 frame), source =
    frame 2 points (camera-2 frame), ``T_gt`` = camera-2 -> camera-1.
    ``meta["target_pixels"]`` holds the flat pixel index (v * w + u) of each
    target point and ``meta["intrinsics"]`` (fx, fy, cx, cy): the target frame
    as an organised image, for projective association."""
    rng = np.random.default_rng(seed)
    scene = _depth_scene(rng)
    s = c = math.sqrt(0.5)
    x = np.array([1.0, 0.0, 0.0])
    zf = np.array([0.0, c, -s])
    y = np.cross(zf, x)
    P1 = np.eye(4)
    P1[:3, :3] = np.column_stack([x, y, zf])
    P1[:3, 3] = [0.0, 0.0, 1.5]
    dT = random_rigid(rng, max_angle_deg, max_trans, "ball")
    P2 = P1 @ dT
    tgt, tgt_pix = _render_depth(rng, P1, scene, width, height, fx, fy, cx, cy, 0.5, 5.0,
                                 return_pixels=True)
    src = _render_depth(rng, P2, scene, width, height, fx, fy, cx, cy, 0.5, 5.0)
    return Pair(
        source=src.astype(np.float32),
        target=tgt.astype(np.float32),
        T_gt=dT,
        viewpoint=np.zeros(3),
        meta={"kind": "depth", "seed": seed, "w": width, "h": height,
              "intrinsics": (fx, fy, cx, cy), "target_pixels": tgt_pix},
    )


# ---------------------------------------------------------------------------
# workload: spinning LiDAR sweep (ground + boxes)
# ---------------------------------------------------------------------------
def _lidar_scene(rng, n_boxes=200, clear=((0.0, 0.0),), clear_r=3.0):
    centers = []
    while len(centers) < n_boxes:
        r = 100.0 * math.sqrt(rng.uniform(0.0, 1.0))
        a = rng.uniform(0.0, 2 * math.pi)
        sz = rng.uniform(1.0, 10.0, size=3)
        cxy = np.array([r * math.cos(a), r * math.sin(a)])
        # keep the box (with its half-diagonal) clear of the sensor positions
        half = 0.5 * math.hypot(sz[0], sz[1])
        if any(np.linalg.norm(cxy - np.asarray(q)) < clear_r + half for q in clear):
            continue
        centers.append((cxy, sz))
    lo = np.array([[c[0] - s[0] / 2, c[1] - s[1] / 2, 0.0] for c, s in centers])
    hi = np.array([[c[0] + s[0] / 2, c[1] + s[1] / 2, s[2]] for c, s in centers])
    return lo, hi


def _render_lidar(rng, pose_ws, scene, n_beams, n_az, elev_lo, elev_hi, max_range, noise):
    lo, hi = scene
    el = np.radians(np.linspace(elev_lo, elev_hi, n_beams))
    az = np.arange(n_az) * (2 * math.pi / n_az)
    E, A = np.meshgrid(el, az, indexing="ij")
    E = E.ravel()
    A = A.ravel()
    ds = np.column_stack([np.cos(E) * np.cos(A), np.cos(E) * np.sin(A), np.sin(E)])
    R = pose_ws[:3, :3]
    o = pose_ws[:3, 3]
    dw = ds @ R.T
    with np.errstate(divide="ignore", invalid="ignore"):
        tg = np.where(dw[:, 2] < -1e-12, -o[2] / dw[:, 2], np.inf)
    t = np.where(tg > 0, tg, np.inf)
    chunk = 8192
    for i in range(0, dw.shape[0], chunk):
        tb = _ray_boxes(o[None, :], dw[i : i + chunk], lo, hi)
        t[i : i + chunk] = np.minimum(t[i : i + chunk], tb)
    valid = np.isfinite(t) & (t <= max_range)
    rr = t[valid] + rng.normal(0.0, noise, size=int(valid.sum()))
    return ds[valid] * rr[:, None]


def lidar_sweep_pair(
    seed: int,
    n_beams: int = 64,
    n_az: int = 2048,
    elev_lo: float = -25.0,
    elev_hi: float = 3.0,
    height: float = 1.8,
    max_range: float = 120.0,
    noise: float = 0.02,
    max_move: float = 1.0,
    max_yaw_deg: float = 2.0,
) -> Pair:
    """Two sweeps of a 64-beam spinning sensor (evenly spaced elevations in
    [-25, +3] deg, 2048 azimuth steps, 1.8 m high) over a ground plane with 200
    boxes of side 1-10 m within 100 m.  The second pose is moved by <= 1 m in
    the ground plane and <= 2 deg of yaw.  Points are in each sensor's frame;
    ``T_gt`` maps sweep-2 sensor coordinates to sweep-1 sensor coordinates."""
    rng = np.random.default_rng(seed)
    P1 = np.eye(4)
    P1[:3, 3] = [0.0, 0.0, height]
    ang = rng.uniform(0.0, 2 * math.pi)
    dist = rng.uniform(0.0, max_move)
    yaw = math.radians(rng.uniform(-max_yaw_deg, max_yaw_deg))
    dT = np.eye(4)
    dT[:3, :3] = rotation_from_axis_angle([0.0, 0.0, 1.0], yaw)
    dT[:3, 3] = [dist * math.cos(ang), dist * math.sin(ang), 0.0]
    P2 = P1 @ dT
    scene = _lidar_scene(rng, clear=((0.0, 0.0), tuple(P2[:2, 3])))
    tgt = _render_lidar(rng, P1, scene, n_beams, n_az, elev_lo, elev_hi, max_range, noise)
    src = _render_lidar(rng, P2, scene, n_beams, n_az, elev_lo, elev_hi, max_range, noise)
    return Pair(
        source=src.astype(np.float32),
        target=tgt.astype(np.float32),
        T_gt=dT,
        viewpoint=np.zeros(3),
        meta={"kind": "lidar", "seed": seed},
    )


# ---------------------------------------------------------------------------
# workload: batch of uneven surface pairs
# ---------------------------------------------------------------------------
def batch_sizes(seed: int, B: int = 256, n_lo: int = 2_000, n_hi: int = 200_000) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.round(np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), size=B))).astype(np.int64)


def surface_batch(seed: int = 0, B: int = 256, n_lo: int = 2_000, n_hi: int = 200_000,
                  sizes=None, **kw) -> list[Pair]:
    """B surface pairs; pair i has n_i = round(exp(U[ln n_lo, ln n_hi])) points
    on both sides and per-pair seed 1000 + i."""
    if sizes is None:
        sizes = batch_sizes(seed, B, n_lo, n_hi)
    return [surface_pair(1000 + i, n=int(n), **kw) for i, n in enumerate(sizes)]


def warm_start_pairs(seed: int, B: int, n: int = 10_000, n_sub: int = 4096,
                     max_angle_deg: float = 90.0, max_trans: float = 0.5):
    """B surface pairs with rotations up to 90 deg and translations up to 0.5,
    each side subsampled to ``n_sub`` points (without replacement when
    n >= n_sub, else with replacement).  Returns (pairs, src_sub, dst_sub) where
    the subsamples are float32 arrays of shape (B, n_sub, 3)."""
    rng = np.random.default_rng(seed)
    seeds = rng.integers(0, 2**62, size=B)
    pairs = []
    src_sub = np.empty((B, n_sub, 3), np.float32)
    dst_sub = np.empty((B, n_sub, 3), np.float32)
    for b in range(B):
        p = surface_pair(int(seeds[b]), n=n, max_angle_deg=max_angle_deg, max_trans=max_trans)
        r = np.random.default_rng(int(seeds[b]) ^ 0x5EED)
        rep = n < n_sub
        src_sub[b] = p.source[r.choice(p.source.shape[0], n_sub, replace=rep)]
        dst_sub[b] = p.target[r.choice(p.target.shape[0], n_sub, replace=rep)]
        pairs.append(p)
    return pairs, src_sub, dst_sub


# ---------------------------------------------------------------------------
# small structured inputs used by edge-case tests
# ---------------------------------------------------------------------------
def lattice_points(shape=(4, 4, 4), spacing: float = 1.0, origin=(0.0, 0.0, 0.0)) -> np.ndarray:
    """Integer lattice (exactly representable in float32): every pairwise squared
    distance is an integer multiple of spacing^2, so ties are exact."""
    g = np.stack(np.meshgrid(*[np.arange(s) for s in shape], indexing="ij"), -1).reshape(-1, 3)
    return (g * spacing + np.asarray(origin)).astype(np.float32)


# ---------------------------------------------------------------------------
# the batch workload generated on the GPU (same distributions as
# surface_pair / surface_batch, drawn with a seeded torch generator)
# ---------------------------------------------------------------------------
def surface_batch_torch(seed: int, sizes, noise: float = 0.002, max_angle_deg: float = 10.0,
                        max_trans: float = 0.05, device="cuda"):
    """Concatenated source and target clouds of len(sizes) wavy-surface pairs
    (pair i has sizes[i] points on both sides), plus the source -> target
    labels.  Returns (src float32 (sum,3), dst float32 (sum,3), T_gt float64
    (B,4,4)), all on `device`."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    f64 = torch.float64
    sizes = [int(n) for n in sizes]
    tot = sum(sizes)
    B = len(sizes)
    pair_of = torch.repeat_interleave(torch.arange(B, device=device),
                                      torch.tensor(sizes, device=device))

    def surface(n):
        xy = torch.rand(n, 2, generator=gen, device=device, dtype=f64) * 2 - 1
        z = 0.1 * torch.sin(4 * xy[:, 0]) * torch.cos(4 * xy[:, 1])
        p = torch.cat([xy, z[:, None]], 1)
        return p + noise * torch.randn(n, 3, generator=gen, device=device, dtype=f64)

    dst = surface(tot)
    src0 = surface(tot)
    axis = torch.randn(B, 3, generator=gen, device=device, dtype=f64)
    axis = axis / axis.norm(dim=1, keepdim=True)
    ang = torch.rand(B, generator=gen, device=device, dtype=f64) * math.radians(max_angle_deg)
    # quaternion -> rotation matrix, as in rotation_from_axis_angle
    w = torch.cos(ang / 2)
    xyz = torch.sin(ang / 2)[:, None] * axis
    x, y, z = xyz[:, 0], xyz[:, 1], xyz[:, 2]
    R = torch.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
                     2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
                     2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], 1).reshape(B, 3, 3)
    t = (torch.rand(B, 3, generator=gen, device=device, dtype=f64) * 2 - 1) * max_trans
    src = torch.einsum("nij,nj->ni", R[pair_of], src0) + t[pair_of]
    T = torch.zeros(B, 4, 4, dtype=f64, device=device)
    Rt = R.transpose(1, 2)
    T[:, :3, :3] = Rt
    T[:, :3, 3] = -(Rt @ t[:, :, None])[:, :, 0]
    T[:, 3, 3] = 1
    return src.to(torch.float32).contiguous(), dst.to(torch.float32).contiguous(), T


def _box_faces(lo, hi, bottom: bool = True):
    """The faces of an axis-aligned box as (origin, edge u, edge v) rectangles."""
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    d = hi - lo
    ex, ey, ez = np.diag(d)
    faces = [(lo, ex, ey), (lo + ez, ex, ey), (lo, ex, ez), (lo + ey, ex, ez),
             (lo, ey, ez), (lo + ex, ey, ez)]
    return faces if bottom else faces[1:]


APARTMENT_VIEWPOINT = (3.0, 2.0, 1.3)  # the flat's middle, at head height


def apartment_scene(seed: int = 0, n: int = 7_800_000, noise: float = 0.0005, n_boxes: int = 12):
    """An apartment-scale reconstruction stand-in: `n` points sampled uniformly
    by area on a 7 m x 5 m x 2.6 m flat (floor, outer walls, two partition
    walls, no ceiling) furnished with 40 boxes (tables, cabinets, beds: open at
    the floor) and 8 spheres, with isotropic Gaussian noise of `noise` metres.
    The flat's corner sits at (0.0123, 0.0071, 0.0026), off the lattice of a
    5 mm voxel grid, which then keeps a little under 60 % of the points (4.49M
    of 7.8M at seed 0)."""

    rng = np.random.default_rng(seed)
    W, D, H = 6.0, 4.0, 2.5
    rects = [(np.zeros(3), np.array([W, 0, 0.0]), np.array([0, D, 0.0]))]
    rects += [(np.zeros(3), np.array([W, 0, 0.0]), np.array([0, 0, H])),
              (np.array([0, D, 0.0]), np.array([W, 0, 0.0]), np.array([0, 0, H])),
              (np.zeros(3), np.array([0, D, 0.0]), np.array([0, 0, H])),
              (np.array([W, 0, 0.0]), np.array([0, D, 0.0]), np.array([0, 0, H]))]
    # partition walls, 10 cm thick, with a doorway gap
    rects += _box_faces([3.0, 0.0, 0.0], [3.1, 3.0, H], bottom=False)
    for _ in range(n_boxes):
        c = rng.uniform([0.3, 0.3], [W - 0.3, D - 0.3])
        sz = rng.uniform([0.3, 0.3, 0.3], [1.6, 1.0, 1.8])
        lo = np.array([c[0] - sz[0] / 2, c[1] - sz[1] / 2, 0.0])
        rects += _box_faces(lo, lo + sz, bottom=False)
    org = np.array([r[0] for r in rects])
    U = np.array([r[1] for r in rects])
    V = np.array([r[2] for r in rects])
    area = np.linalg.norm(np.cross(U, V), axis=1)
    sc = np.column_stack([rng.uniform(0.5, W - 0.5, 8), rng.uniform(0.5, D - 0.5, 8)])
    sr = rng.uniform(0.1, 0.3, 8)
    sph_c = np.column_stack([sc, rng.uniform(0.4, 1.8, 8)])
    s_area = 4 * np.pi * sr ** 2
    w = np.concatenate([area, s_area])
    pick = rng.choice(len(w), size=n, p=w / w.sum())
    out = np.empty((n, 3), np.float64)
    m = pick < len(rects)
    r = pick[m]
    st = rng.random((len(r), 2))
    out[m] = org[r] + st[:, :1] * U[r] + st[:, 1:] * V[r]
    s = pick[~m] - len(rects)
    d = rng.normal(size=(len(s), 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    out[~m] = sph_c[s] + sr[s, None] * d
    out += rng.normal(0.0, noise, size=out.shape)
    out += np.array([0.0123, 0.0071, 0.0026])
    return out.astype(np.float32)
