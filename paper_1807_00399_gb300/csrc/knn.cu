// knn.cu -- k-nearest-neighbour queries and fused PCA normals.
//
// One thread per query.  Queries are visited in the Morton order of the
// reference grid (self-queries: the sorted points themselves; external
// queries: a stable Morton sort of the queries), so the threads of a warp
// search neighbouring cells and share their loads through L1.  Each thread
// keeps its k best (squared distance, index) keys: sorted in registers for
// k <= 4, in a max-heap in shared memory above (heap-sorted at the end).
//
// Normals (Sec. 3 normal/curvature estimation, Sec. 4 10-NN neighbourhoods):
// the k neighbours' offsets from the query give their mean, then the centred
// covariance C = (1/m) sum (p - mu)(p - mu)^T in a second pass; its smallest
// eigenpair comes from the closed-form trigonometric solution of the
// characteristic cubic, a cross product of two rows of C - l0 I and one
// Rayleigh-quotient refinement of l0.
#include <math.h>

#include "cil_host.h"
#include "cil_kernels.h"

namespace cil {

template <int KMAX, bool HEAP>
__global__ void __launch_bounds__(256) k_knn(GridView g, const float* __restrict__ qry, int64_t nq,
                                             const int* __restrict__ order, int k,
                                             int* __restrict__ out_idx, float* __restrict__ out_d2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nq) return;
  int64_t qi;
  float q[3];
  if (order) {
    qi = order[i];
    q[0] = qry[3 * qi];
    q[1] = qry[3 * qi + 1];
    q[2] = qry[3 * qi + 2];
  } else {
    const float4 p = g.pts[i];
    qi = __float_as_int(p.w);
    q[0] = p.x;
    q[1] = p.y;
    q[2] = p.z;
  }
  extern __shared__ u64 s_topk[];
  TopKSel<KMAX, HEAP> top;
  top.bind(s_topk + threadIdx.x, blockDim.x);
  top.init(k);
  grid_knn<KMAX>(g, 0, q, top);
  top.finish();
  int* oi = out_idx + qi * k;
  float* od = out_d2 ? out_d2 + qi * k : nullptr;
#pragma unroll
  for (int j = 0; j < KMAX; ++j) {
    if (j < k) {
      const u64 key = top.key_at(j);
      const bool none = key == kEmptyKey;
      oi[j] = none ? -1 : key_idx(key);
      if (od) od[j] = none ? __int_as_float(0x7f800000) : key_d2(key);
    }
  }
}

// Unit null vector of the symmetric matrix A - l I: the largest cross product
// of two of its rows (selects only, so everything stays in registers).  When
// A - l I has rank <= 1, any unit vector orthogonal to its largest row.
__device__ __forceinline__ void null_vector3(float a00, float a01, float a02, float a11, float a12,
                                             float a22, float l, float nv[3]) {
  const float r0x = a00 - l, r0y = a01, r0z = a02;
  const float r1x = a01, r1y = a11 - l, r1z = a12;
  const float r2x = a02, r2y = a12, r2z = a22 - l;
  const float ax = r0y * r1z - r0z * r1y, ay = r0z * r1x - r0x * r1z, az = r0x * r1y - r0y * r1x;
  const float bx = r0y * r2z - r0z * r2y, by = r0z * r2x - r0x * r2z, bz = r0x * r2y - r0y * r2x;
  const float cx = r1y * r2z - r1z * r2y, cy = r1z * r2x - r1x * r2z, cz = r1x * r2y - r1y * r2x;
  const float ma = ax * ax + ay * ay + az * az;
  const float mb = bx * bx + by * by + bz * bz;
  const float mc = cx * cx + cy * cy + cz * cz;
  float vx = ax, vy = ay, vz = az, best = ma;
  if (mb > best) {
    vx = bx;
    vy = by;
    vz = bz;
    best = mb;
  }
  if (mc > best) {
    vx = cx;
    vy = cy;
    vz = cz;
    best = mc;
  }
  if (best > 0.0f) {
    const float in = rsqrtf(best);
    nv[0] = vx * in;
    nv[1] = vy * in;
    nv[2] = vz * in;
    return;
  }
  const float m0 = r0x * r0x + r0y * r0y + r0z * r0z;
  const float m1 = r1x * r1x + r1y * r1y + r1z * r1z;
  const float m2 = r2x * r2x + r2y * r2y + r2z * r2z;
  float ex = r0x, ey = r0y, ez = r0z, em = m0;
  if (m1 > em) {
    ex = r1x;
    ey = r1y;
    ez = r1z;
    em = m1;
  }
  if (m2 > em) {
    ex = r2x;
    ey = r2y;
    ez = r2z;
  }
  float ux, uy, uz;
  if (fabsf(ex) <= fabsf(ey) && fabsf(ex) <= fabsf(ez)) {
    ux = 0.0f;
    uy = ez;
    uz = -ey;
  } else if (fabsf(ey) <= fabsf(ez)) {
    ux = -ez;
    uy = 0.0f;
    uz = ex;
  } else {
    ux = ey;
    uy = -ex;
    uz = 0.0f;
  }
  const float mu = ux * ux + uy * uy + uz * uz;
  if (mu > 0.0f) {
    const float in = rsqrtf(mu);
    nv[0] = ux * in;
    nv[1] = uy * in;
    nv[2] = uz * in;
  } else {
    nv[0] = 0.0f;
    nv[1] = 0.0f;
    nv[2] = 1.0f;
  }
}

// Smallest eigenpair of a symmetric 3x3 (c00, c01, c02, c11, c12, c22).
// Eigenvalues from the closed-form trigonometric solution of the
// characteristic cubic (matrix scaled to max |entry| = 1); the eigenvector of
// the smallest as the null vector of A - l0 I.  The trigonometric l0 carries
// an absolute error of tens of ulps of the largest eigenvalue, which would
// tilt the vector by that error over the gap l1 - l0; one Rayleigh-quotient
// step l0 <- v^T A v (error quadratic in the tilt) and a second null-vector
// solve remove it.  Returns false (and NaN) for a zero matrix.
__device__ __forceinline__ bool sym3_smallest(const float C[6], float ev[3], float nv[3]) {
  float s = 0.0f;
#pragma unroll
  for (int j = 0; j < 6; ++j) s = fmaxf(s, fabsf(C[j]));
  if (!(s > 0.0f) || !isfinite(s)) {
    ev[0] = ev[1] = ev[2] = __int_as_float(0x7fc00000);
    nv[0] = nv[1] = nv[2] = __int_as_float(0x7fc00000);
    return false;
  }
  const float inv = 1.0f / s;
  const float a00 = C[0] * inv, a01 = C[1] * inv, a02 = C[2] * inv;
  const float a11 = C[3] * inv, a12 = C[4] * inv, a22 = C[5] * inv;
  const float q = (a00 + a11 + a22) * (1.0f / 3.0f);
  const float b00 = a00 - q, b11 = a11 - q, b22 = a22 - q;
  const float p1 = a01 * a01 + a02 * a02 + a12 * a12;
  const float p2 = b00 * b00 + b11 * b11 + b22 * b22 + 2.0f * p1;
  const float p = sqrtf(p2 * (1.0f / 6.0f));
  float l0, l1, l2;
  if (!(p > 1e-30f)) {  // isotropic: every direction is an eigenvector
    l0 = l1 = l2 = q;
    nv[0] = 0.0f;
    nv[1] = 0.0f;
    nv[2] = 1.0f;
  } else {
    const float ip = 1.0f / p;
    const float B00 = b00 * ip, B11 = b11 * ip, B22 = b22 * ip;
    const float B01 = a01 * ip, B02 = a02 * ip, B12 = a12 * ip;
    const float det = B00 * (B11 * B22 - B12 * B12) - B01 * (B01 * B22 - B12 * B02) +
                      B02 * (B01 * B12 - B11 * B02);
    const float r = fminf(fmaxf(0.5f * det, -1.0f), 1.0f);
    const float phi = acosf(r) * (1.0f / 3.0f);
    l2 = q + 2.0f * p * cosf(phi);
    l0 = q + 2.0f * p * cosf(phi + 2.0943951023931957f);
    null_vector3(a00, a01, a02, a11, a12, a22, l0, nv);
    // Rayleigh-quotient refinement of l0, then the vector again
    const float v0 = nv[0], v1 = nv[1], v2 = nv[2];
    const float w0 = a00 * v0 + a01 * v1 + a02 * v2;
    const float w1 = a01 * v0 + a11 * v1 + a12 * v2;
    const float w2 = a02 * v0 + a12 * v1 + a22 * v2;
    l0 = v0 * w0 + v1 * w1 + v2 * w2;
    null_vector3(a00, a01, a02, a11, a12, a22, l0, nv);
    l1 = 3.0f * q - l0 - l2;
  }
  ev[0] = l0 * s;
  ev[1] = l1 * s;
  ev[2] = l2 * s;
  return true;
}

// Normal, orientation and curvature from a covariance (shared by the k-NN and
// the radius neighbourhoods).
__device__ __forceinline__ void finish_normal(const float C[6], const float q[3], const float vp[3],
                                              float out_n[3], float& out_c) {
  const float nan = __int_as_float(0x7fc00000);
  float ev[3], nv[3];
  if (!sym3_smallest(C, ev, nv)) {
    out_n[0] = out_n[1] = out_n[2] = nan;
    out_c = nan;
    return;
  }
  const float tr = ev[0] + ev[1] + ev[2];
  const float s = nv[0] * (vp[0] - q[0]) + nv[1] * (vp[1] - q[1]) + nv[2] * (vp[2] - q[2]);
  const float sg = s < 0.0f ? -1.0f : 1.0f;
  out_n[0] = sg * nv[0];
  out_n[1] = sg * nv[1];
  out_n[2] = sg * nv[2];
  out_c = tr > 0.0f ? fmaxf(ev[0], 0.0f) / tr : nan;
}

// PCA normal + curvature of one point from its neighbour keys.  `xyz` and the
// key indices are relative to the same cloud.
template <int KMAX, class Top>
__device__ __forceinline__ void normal_from_topk(const Top& top, int k,
                                                 const float* __restrict__ xyz, const float q[3],
                                                 const float vp[3], float out_n[3], float& out_c) {
  // pass 1: mean offset of the neighbours from the query (offsets of nearby
  // points are exact in FP32); pass 2: covariance about that mean (centred,
  // so no cancellation between second moments and the squared mean)
  float sx = 0.f, sy = 0.f, sz = 0.f;
  int m = 0;
#pragma unroll
  for (int j = 0; j < KMAX; ++j) {
    const u64 key = top.key_at(j);
    if (j < k && key != kEmptyKey) {
      const int64_t id = key_idx(key);
      sx += xyz[3 * id] - q[0];
      sy += xyz[3 * id + 1] - q[1];
      sz += xyz[3 * id + 2] - q[2];
      ++m;
    }
  }
  const float nan = __int_as_float(0x7fc00000);
  if (m < 3) {
    out_n[0] = out_n[1] = out_n[2] = nan;
    out_c = nan;
    return;
  }
  const float im = 1.0f / (float)m;
  const float mx = sx * im, my = sy * im, mz = sz * im;
  float cxx = 0.f, cxy = 0.f, cxz = 0.f, cyy = 0.f, cyz = 0.f, czz = 0.f;
#pragma unroll
  for (int j = 0; j < KMAX; ++j) {
    const u64 key = top.key_at(j);
    if (j < k && key != kEmptyKey) {
      const int64_t id = key_idx(key);
      const float ex = (xyz[3 * id] - q[0]) - mx;
      const float ey = (xyz[3 * id + 1] - q[1]) - my;
      const float ez = (xyz[3 * id + 2] - q[2]) - mz;
      cxx = fmaf(ex, ex, cxx);
      cxy = fmaf(ex, ey, cxy);
      cxz = fmaf(ex, ez, cxz);
      cyy = fmaf(ey, ey, cyy);
      cyz = fmaf(ey, ez, cyz);
      czz = fmaf(ez, ez, czz);
    }
  }
  const float C[6] = {cxx * im, cxy * im, cxz * im, cyy * im, cyz * im, czz * im};
  finish_normal(C, q, vp, out_n, out_c);
}

template <int KMAX, bool HEAP>
__global__ void __launch_bounds__(256) k_normals(GridView g, int cloud_count, int64_t n, int k,
                                                 const float* __restrict__ vp_all, float vx,
                                                 float vy, float vz,
                                                 const float* __restrict__ xyz,
                                                 float* __restrict__ out_n, float* __restrict__ out_c,
                                                 int* __restrict__ out_idx) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 p = g.pts[i];
  // the sorted array is grouped by cloud; find this point's cloud
  int cloud = 0;
  if (cloud_count > 1) {
    int lo = 0, hi = cloud_count;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if ((int64_t)g.prm[mid].start <= i) lo = mid;
      else hi = mid;
    }
    cloud = lo;
  }
  const int start = g.prm[cloud].start;
  const int64_t local = __float_as_int(p.w);
  const float q[3] = {p.x, p.y, p.z};
  extern __shared__ u64 s_topk[];
  TopKSel<KMAX, HEAP> top;
  top.bind(s_topk + threadIdx.x, blockDim.x);
  top.init(k);
  grid_knn<KMAX>(g, cloud, q, top);
  // ascending keys, so the sums below run in one order whatever order the
  // search met the points in (results independent of cell size and block)
  top.finish();
  const float vp[3] = {vp_all ? vp_all[3 * cloud] : vx, vp_all ? vp_all[3 * cloud + 1] : vy,
                       vp_all ? vp_all[3 * cloud + 2] : vz};
  float nv[3], c;
  normal_from_topk<KMAX>(top, k, xyz + 3 * (int64_t)start, q, vp, nv, c);
  const int64_t gi = start + local;
  out_n[3 * gi] = nv[0];
  out_n[3 * gi + 1] = nv[1];
  out_n[3 * gi + 2] = nv[2];
  if (out_c) out_c[gi] = c;
  if (out_idx) {
    int* oi = out_idx + gi * k;
#pragma unroll
    for (int j = 0; j < KMAX; ++j) {
      const u64 key = top.key_at(j);
      if (j < k) oi[j] = key == kEmptyKey ? -1 : key_idx(key);
    }
  }
}

// ---------------------------------------------------------------------------
// warp-staged search: the 32 queries of a warp (consecutive in the grid's
// Morton order, so neighbours in space) share one staged set of points -- the
// cells of the box spanned by their own cells plus one ring, looked up once by
// the lanes and copied to shared memory -- and every lane scans every staged
// point (one broadcast read per point for the whole warp, no divergence in
// the distance work, no per-query hash lookups).  A lane's result is kept
// when its k-th distance is proven: every point outside the box is farther
// (the padded distance to the grid outside the box); otherwise, or when the
// box is too large to stage, the lane runs the per-query ring search.  The
// kept keys are the same (d2, index) set either way, so results are bitwise
// those of the per-query search.
// ---------------------------------------------------------------------------
constexpr int kStageWarps = 4;    // warps (32 queries each) per block
constexpr int kStagePts = 512;    // staged points per warp at most
constexpr int kStageCells = 128;  // cells of a warp's box at most

struct StageSmem {
  float4 pts[kStagePts];
  int start[32], pre[33];
};

template <int KMAX, class Top>
__device__ __forceinline__ bool staged_knn(const GridView& g, int cloud, bool warp_ok,
                                           const float q[3], bool active, Top& top, StageSmem& S,
                                           int lane) {
  const unsigned full = 0xffffffffu;
  if (!warp_ok) return false;
  const GridParams& P = g.prm[cloud];
  CellFrame f;
  f.load(P, cloud);
  int lo[3], hi[3], qlo[3], qhi[3];  // the box; the queries' own cells
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int c = f.cell_of(q[a], a, P.inv_fine);
    qlo[a] = (int)__reduce_min_sync(full, active ? c : 0x7fffffff);
    qhi[a] = (int)__reduce_max_sync(full, active ? c : -1);
    lo[a] = max(qlo[a] - 1, 0);
    hi[a] = min(qhi[a] + 1, f.hi[a]);
  }
  const int nx = hi[0] - lo[0] + 1, nxy = nx * (hi[1] - lo[1] + 1);
  const int ncell = nxy * (hi[2] - lo[2] + 1);
  if (ncell > kStageCells) return false;
  const float inv_nx = 1.0f / (float)nx, inv_nxy = 1.0f / (float)nxy;
  int total = 0;
  // the queries' own cells are staged first, the ring around them last, so
  // every lane meets its nearest points early and later pushes are rare
  for (int pass = 0, c0 = 0; pass < 2; c0 += 32) {
    if (c0 >= ncell) {
      ++pass;
      c0 = -32;
      continue;
    }
    const int c = c0 + lane;
    int s = 0, n = 0;
    if (c < ncell) {
      // c = (z * ny + y) * nx + x (float quotients: exact for c < 2^22)
      const int z = __float2int_rz(((float)c + 0.5f) * inv_nxy), rem = c - z * nxy;
      const int y = __float2int_rz(((float)rem + 0.5f) * inv_nx), x = rem - y * nx;
      const int X = lo[0] + x, Y = lo[1] + y, Z = lo[2] + z;
      const bool own = X >= qlo[0] && X <= qhi[0] && Y >= qlo[1] && Y <= qhi[1] && Z >= qlo[2] &&
                       Z <= qhi[2];
      if (own == (pass == 0) && !cell_lookup(g, cell_key(f.level, cloud, X, Y, Z), s, n)) n = 0;
    }
    int incl = n;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(full, incl, o);
      if (lane >= o) incl += v;
    }
    const int chunk = __shfl_sync(full, incl, 31);
    if (total + chunk > kStagePts) return false;
    __syncwarp();
    S.start[lane] = s;
    S.pre[lane] = incl - n;
    if (lane == 31) S.pre[32] = chunk;
    __syncwarp();
    int ci = 0, cs = S.start[0], cp = 0, cn = S.pre[1];
    for (int t = lane; t < chunk; t += 32) {
      while (t >= cn) {
        ++ci;
        cp = cn;
        cs = S.start[ci];
        cn = S.pre[ci + 1];
      }
      S.pts[total + t] = __ldg(g.pts + cs + (t - cp));
    }
    total += chunk;
  }
  __syncwarp();
  top.init(top.k);
  if (active) {
    for (int j = 0; j < total; ++j) {
      const float4 p = S.pts[j];
      top.push(pack_key(sqdist(p.x, p.y, p.z, q[0], q[1], q[2]), __float_as_int(p.w)));
    }
  }
  __syncwarp();  // S is reused by the next call
  const float bound = f.unexplored_d2(q, lo, hi);
  if (top.full()) return top.thr_d2() < bound * (1.0f - 1e-6f);
  return !(bound < __int_as_float(0x7f800000));  // the whole cloud was staged
}

template <int KMAX, bool HEAP>
__global__ void __launch_bounds__(kStageWarps * 32) k_knn_staged(GridView g,
                                                                 const float* __restrict__ qry,
                                                                 int64_t nq,
                                                                 const int* __restrict__ order,
                                                                 int k, int* __restrict__ out_idx,
                                                                 float* __restrict__ out_d2) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  StageSmem& S = reinterpret_cast<StageSmem*>(smem_raw)[w];
  u64* s_topk = reinterpret_cast<u64*>(smem_raw + sizeof(StageSmem) * kStageWarps);
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + 32 * w;
  if (i0 >= nq) return;  // whole warp
  const bool active = i < nq;
  const int64_t ii = active ? i : i0;
  int64_t qi;
  float q[3];
  if (order) {
    qi = order[ii];
    q[0] = qry[3 * qi];
    q[1] = qry[3 * qi + 1];
    q[2] = qry[3 * qi + 2];
  } else {
    const float4 p = g.pts[ii];
    qi = __float_as_int(p.w);
    q[0] = p.x;
    q[1] = p.y;
    q[2] = p.z;
  }
  TopKSel<KMAX, HEAP> top;
  top.bind(s_topk + threadIdx.x, blockDim.x);
  top.init(k);
  const bool ok = staged_knn<KMAX>(g, 0, true, q, active, top, S, lane);
  if (!active) return;
  if (!ok) grid_knn<KMAX>(g, 0, q, top);
  top.finish();
  int* oi = out_idx + qi * k;
  float* od = out_d2 ? out_d2 + qi * k : nullptr;
#pragma unroll
  for (int j = 0; j < KMAX; ++j) {
    if (j < k) {
      const u64 key = top.key_at(j);
      const bool none = key == kEmptyKey;
      oi[j] = none ? -1 : key_idx(key);
      if (od) od[j] = none ? __int_as_float(0x7f800000) : key_d2(key);
    }
  }
}

template <int KMAX, bool HEAP>
__global__ void __launch_bounds__(kStageWarps * 32) k_normals_staged(
    GridView g, int cloud_count, int64_t n, int k, const float* __restrict__ vp_all, float vx,
    float vy, float vz, const float* __restrict__ xyz, float* __restrict__ out_n,
    float* __restrict__ out_c, int* __restrict__ out_idx) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  StageSmem& S = reinterpret_cast<StageSmem*>(smem_raw)[w];
  u64* s_topk = reinterpret_cast<u64*>(smem_raw + sizeof(StageSmem) * kStageWarps);
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + 32 * w;
  if (i0 >= n) return;  // whole warp
  const bool active = i < n;
  const float4 p = g.pts[active ? i : i0];
  // the sorted array is grouped by cloud; find this point's cloud
  int cloud = 0;
  if (cloud_count > 1) {
    int lo = 0, hi = cloud_count;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if ((int64_t)g.prm[mid].start <= (active ? i : i0)) lo = mid;
      else hi = mid;
    }
    cloud = lo;
  }
  const bool same = __all_sync(0xffffffffu, cloud == __shfl_sync(0xffffffffu, cloud, 0));
  const int start = g.prm[cloud].start;
  const int64_t local = __float_as_int(p.w);
  const float q[3] = {p.x, p.y, p.z};
  TopKSel<KMAX, HEAP> top;
  top.bind(s_topk + threadIdx.x, blockDim.x);
  top.init(k);
  const bool ok = staged_knn<KMAX>(g, cloud, same, q, active, top, S, lane);
  if (!active) return;
  if (!ok) grid_knn<KMAX>(g, cloud, q, top);
  top.finish();
  const float vp[3] = {vp_all ? vp_all[3 * cloud] : vx, vp_all ? vp_all[3 * cloud + 1] : vy,
                       vp_all ? vp_all[3 * cloud + 2] : vz};
  float nv[3], c;
  normal_from_topk<KMAX>(top, k, xyz + 3 * (int64_t)start, q, vp, nv, c);
  const int64_t gi = start + local;
  out_n[3 * gi] = nv[0];
  out_n[3 * gi + 1] = nv[1];
  out_n[3 * gi + 2] = nv[2];
  if (out_c) out_c[gi] = c;
  if (out_idx) {
    int* oi = out_idx + gi * k;
#pragma unroll
    for (int j = 0; j < KMAX; ++j) {
      const u64 key = top.key_at(j);
      if (j < k) oi[j] = key == kEmptyKey ? -1 : key_idx(key);
    }
  }
}

// ---------------------------------------------------------------------------
// hybrid query (k nearest within r) and radius-neighbourhood normals
// (Sec. 3 hybrid queries and radius normals; Sec. 4 uses 1 cm balls)
// ---------------------------------------------------------------------------
template <int KMAX>
__global__ void __launch_bounds__(256) k_knn_hybrid(GridView g, const float* __restrict__ qry,
                                                    int64_t nq, const int* __restrict__ order, int k,
                                                    float r2, int* __restrict__ out_idx,
                                                    float* __restrict__ out_d2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nq) return;
  int64_t qi;
  float q[3];
  if (order) {
    qi = order[i];
    q[0] = qry[3 * qi];
    q[1] = qry[3 * qi + 1];
    q[2] = qry[3 * qi + 2];
  } else {
    const float4 p = g.pts[i];
    qi = __float_as_int(p.w);
    q[0] = p.x;
    q[1] = p.y;
    q[2] = p.z;
  }
  extern __shared__ u64 s_topk[];
  TopKFor<KMAX> top;
  top.bind(s_topk + threadIdx.x, blockDim.x);
  top.init(k);
  grid_knn_within<KMAX>(g, 0, q, r2, top);
  top.finish();
  int* oi = out_idx + qi * k;
  float* od = out_d2 ? out_d2 + qi * k : nullptr;
#pragma unroll
  for (int j = 0; j < KMAX; ++j) {
    if (j < k) {
      const u64 key = top.key_at(j);
      const bool none = key == kEmptyKey;
      oi[j] = none ? -1 : key_idx(key);
      if (od) od[j] = none ? __int_as_float(0x7f800000) : key_d2(key);
    }
  }
}

// every point within r of each point (itself included): mean offset in a first
// pass over the ball's cells, centred covariance in a second
__global__ void __launch_bounds__(128) k_normals_radius(GridView g, int64_t n, float r, float vx,
                                                        float vy, float vz,
                                                        float* __restrict__ out_n,
                                                        float* __restrict__ out_c,
                                                        int* __restrict__ out_cnt) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 pq = g.pts[i];
  const int64_t qi = __float_as_int(pq.w);
  const float q[3] = {pq.x, pq.y, pq.z};
  const GridParams& P = g.prm[0];
  CellFrame f;
  f.load(P, 0);
  const float r2 = r * r;
  int lo[3], hi[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    lo[a] = f.cell_of(q[a] - r - f.eps, a, P.inv_fine);
    hi[a] = f.cell_of(q[a] + r + f.eps, a, P.inv_fine);
  }
  float sx = 0.f, sy = 0.f, sz = 0.f;
  int m = 0;
  for (int z = lo[2]; z <= hi[2]; ++z)
    for (int y = lo[1]; y <= hi[1]; ++y)
      for (int x = lo[0]; x <= hi[0]; ++x) {
        const int c3[3] = {x, y, z};
        if (f.range_d2(q, c3, c3) * (1.0f - 1e-6f) > r2) continue;
        int s, cnt;
        if (!cell_lookup(g, cell_key(P.level, 0, x, y, z), s, cnt)) continue;
        for_points(g.pts, s, cnt, [&](const float4& p, int) {
          if (sqdist(p.x, p.y, p.z, q[0], q[1], q[2]) <= r2) {
            sx += p.x - q[0];
            sy += p.y - q[1];
            sz += p.z - q[2];
            ++m;
          }
        });
      }
  if (out_cnt) out_cnt[qi] = m;
  const float nan = __int_as_float(0x7fc00000);
  if (m < 3) {
    out_n[3 * qi] = out_n[3 * qi + 1] = out_n[3 * qi + 2] = nan;
    if (out_c) out_c[qi] = nan;
    return;
  }
  const float im = 1.0f / (float)m;
  const float mx = sx * im, my = sy * im, mz = sz * im;
  float cxx = 0.f, cxy = 0.f, cxz = 0.f, cyy = 0.f, cyz = 0.f, czz = 0.f;
  for (int z = lo[2]; z <= hi[2]; ++z)
    for (int y = lo[1]; y <= hi[1]; ++y)
      for (int x = lo[0]; x <= hi[0]; ++x) {
        const int c3[3] = {x, y, z};
        if (f.range_d2(q, c3, c3) * (1.0f - 1e-6f) > r2) continue;
        int s, cnt;
        if (!cell_lookup(g, cell_key(P.level, 0, x, y, z), s, cnt)) continue;
        for_points(g.pts, s, cnt, [&](const float4& p, int) {
          if (sqdist(p.x, p.y, p.z, q[0], q[1], q[2]) <= r2) {
            const float ex = (p.x - q[0]) - mx, ey = (p.y - q[1]) - my, ez = (p.z - q[2]) - mz;
            cxx = fmaf(ex, ex, cxx);
            cxy = fmaf(ex, ey, cxy);
            cxz = fmaf(ex, ez, cxz);
            cyy = fmaf(ey, ey, cyy);
            cyz = fmaf(ey, ez, cyz);
            czz = fmaf(ez, ez, czz);
          }
        });
      }
  const float C[6] = {cxx * im, cxy * im, cxz * im, cyy * im, cyz * im, czz * im};
  const float vp[3] = {vx, vy, vz};
  float nv[3], c;
  finish_normal(C, q, vp, nv, c);
  out_n[3 * qi] = nv[0];
  out_n[3 * qi + 1] = nv[1];
  out_n[3 * qi + 2] = nv[2];
  if (out_c) out_c[qi] = c;
}

// ---------------------------------------------------------------------------
// host launchers: dispatch on the smallest compiled register capacity >= k
// (CIL_FOR_K, cil_dev.cuh)
// ---------------------------------------------------------------------------
// Threads per block for a top-k kind: the heap variants keep KMAX keys per
// thread in shared memory and run at most 128 threads per block (32 KB at
// KMAX = 32), so no launch needs the opt-in above 48 KB.
template <int KM, bool HEAP>
static int topk_block(int block) {
  if (block != 64 && block != 128 && block != 256) block = 128;
  return HEAP ? (block < 128 ? block : 128) : block;
}

template <int KM, bool HEAP>
static void knn_launch_as(const GridView& g, const float* qry, int64_t nq, const int* order, int k,
                          int* out_idx, float* out_d2, int block, cudaStream_t s) {
  const int b = topk_block<KM, HEAP>(block);
  const int smem = HEAP ? KM * (int)sizeof(u64) * b : 0;
  k_knn<KM, HEAP><<<ceil_div(nq, b), b, smem, s>>>(g, qry, nq, order, k, out_idx, out_d2);
}

// layout: 0 = by k, 1 = register list, 2 = shared-memory heap (k = 1 always
// takes the register list)
template <int KM, bool HEAP>
static int staged_smem() {
  return (int)sizeof(StageSmem) * kStageWarps + (HEAP ? KM * (int)sizeof(u64) * kStageWarps * 32 : 0);
}

template <int KM, bool HEAP>
static void knn_staged_as(const GridView& g, const float* qry, int64_t nq, const int* order, int k,
                          int* out_idx, float* out_d2, cudaStream_t s) {
  const int smem = staged_smem<KM, HEAP>();
  cudaFuncSetAttribute(k_knn_staged<KM, HEAP>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  k_knn_staged<KM, HEAP><<<ceil_div(nq, kStageWarps * 32), kStageWarps * 32, smem, s>>>(
      g, qry, nq, order, k, out_idx, out_d2);
}

template <int KM>
static void knn_launch(const GridView& g, const float* qry, int64_t nq, const int* order, int k,
                       int* out_idx, float* out_d2, int block, int layout, cudaStream_t s) {
  if (layout == 3) {
    if (KM > 1 && topk_heap(KM, 0))
      knn_staged_as<KM, (KM > 1)>(g, qry, nq, order, k, out_idx, out_d2, s);
    else
      knn_staged_as<KM, false>(g, qry, nq, order, k, out_idx, out_d2, s);
    return;
  }
  if (KM > 1 && topk_heap(KM, layout))
    knn_launch_as<KM, (KM > 1)>(g, qry, nq, order, k, out_idx, out_d2, block, s);
  else
    knn_launch_as<KM, false>(g, qry, nq, order, k, out_idx, out_d2, block, s);
}

template <int KM, bool HEAP>
static void normals_launch_as(const GridView& g, int clouds, int64_t n, int k, const float* vp_dev,
                              float vx, float vy, float vz, const float* xyz, float* out_n,
                              float* out_c, int* out_idx, int block, cudaStream_t s) {
  const int b = topk_block<KM, HEAP>(block);
  const int smem = HEAP ? KM * (int)sizeof(u64) * b : 0;
  k_normals<KM, HEAP><<<ceil_div(n, b), b, smem, s>>>(g, clouds, n, k, vp_dev, vx, vy, vz, xyz,
                                                      out_n, out_c, out_idx);
}

template <int KM, bool HEAP>
static void normals_staged_as(const GridView& g, int clouds, int64_t n, int k, const float* vp_dev,
                              float vx, float vy, float vz, const float* xyz, float* out_n,
                              float* out_c, int* out_idx, cudaStream_t s) {
  const int smem = staged_smem<KM, HEAP>();
  cudaFuncSetAttribute(k_normals_staged<KM, HEAP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       smem);
  k_normals_staged<KM, HEAP><<<ceil_div(n, kStageWarps * 32), kStageWarps * 32, smem, s>>>(
      g, clouds, n, k, vp_dev, vx, vy, vz, xyz, out_n, out_c, out_idx);
}

template <int KM>
static void normals_launch(const GridView& g, int clouds, int64_t n, int k, const float* vp_dev,
                           float vx, float vy, float vz, const float* xyz, float* out_n,
                           float* out_c, int* out_idx, int block, int layout, cudaStream_t s) {
  if (layout == 3) {
    if (KM > 1 && topk_heap(KM, 0))
      normals_staged_as<KM, (KM > 1)>(g, clouds, n, k, vp_dev, vx, vy, vz, xyz, out_n, out_c,
                                      out_idx, s);
    else
      normals_staged_as<KM, false>(g, clouds, n, k, vp_dev, vx, vy, vz, xyz, out_n, out_c, out_idx,
                                   s);
    return;
  }
  if (KM > 1 && topk_heap(KM, layout))
    normals_launch_as<KM, (KM > 1)>(g, clouds, n, k, vp_dev, vx, vy, vz, xyz, out_n, out_c,
                                    out_idx, block, s);
  else
    normals_launch_as<KM, false>(g, clouds, n, k, vp_dev, vx, vy, vz, xyz, out_n, out_c, out_idx,
                                 block, s);
}

cil_status launch_knn(const GridView& g, const float* qry, int64_t nq, const int* order, int k,
                      int* out_idx, float* out_d2, int block, cudaStream_t s, int topk_layout) {
  if (nq <= 0) return CIL_OK;
  TimedRegion timer("k_knn", s);
  note_launches(1);
  CIL_FOR_K(k, (knn_launch<KM>(g, qry, nq, order, k, out_idx, out_d2, block, topk_layout, s)));
  return cudaGetLastError() == cudaSuccess ? CIL_OK : CIL_ERR_CUDA;
}

cil_status launch_normals(const GridView& g, int clouds, int64_t n, int k, const float* vp_dev,
                          const float* vp_host, const float* xyz, float* out_n, float* out_c,
                          int block, cudaStream_t s, int* out_idx, int topk_layout) {
  if (n <= 0) return CIL_OK;
  TimedRegion timer("k_normals", s);
  note_launches(1);
  const float vx = vp_host ? vp_host[0] : 0.0f, vy = vp_host ? vp_host[1] : 0.0f,
              vz = vp_host ? vp_host[2] : 0.0f;
  CIL_FOR_K(k, (normals_launch<KM>(g, clouds, n, k, vp_dev, vx, vy, vz, xyz, out_n, out_c, out_idx,
                                   block, topk_layout, s)));
  return cudaGetLastError() == cudaSuccess ? CIL_OK : CIL_ERR_CUDA;
}

}  // namespace cil

namespace cil {

cil_status launch_knn_hybrid(const GridView& g, const float* qry, int64_t nq, const int* order,
                             int k, float r, int* out_idx, float* out_d2, cudaStream_t s) {
  if (nq <= 0) return CIL_OK;
  const int grid = ceil_div(nq, 128);
  TimedRegion timer("k_knn_hybrid", s);
  note_launches(1);
  const float r2 = r * r;
  CIL_FOR_K(k, (k_knn_hybrid<KM><<<grid, 128, topk_smem_per_thread<KM>() * 128, s>>>(
                   g, qry, nq, order, k, r2, out_idx, out_d2)));
  return cudaGetLastError() == cudaSuccess ? CIL_OK : CIL_ERR_CUDA;
}

cil_status launch_normals_radius(const GridView& g, int64_t n, float r, const float* vp_host,
                                 float* out_n, float* out_c, int* out_cnt, cudaStream_t s) {
  if (n <= 0) return CIL_OK;
  TimedRegion timer("k_normals_radius", s);
  note_launches(1);
  k_normals_radius<<<ceil_div(n, 128), 128, 0, s>>>(g, n, r, vp_host[0], vp_host[1], vp_host[2],
                                                    out_n, out_c, out_cnt);
  return cudaGetLastError() == cudaSuccess ? CIL_OK : CIL_ERR_CUDA;
}

}  // namespace cil
