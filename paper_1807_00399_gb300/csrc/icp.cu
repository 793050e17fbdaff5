// icp.cu -- rigid point-to-plane ICP (Sec. 2 ICP loop; Sec. 3 point-to-plane
// estimator after Low 2004; Sec. 4 fixed rounds and a rejection distance).
//
// One persistent launch runs every round of every pair.  Work items are tiles
// of kIcpThreads * kIcpPPT source points, numbered round-major; blocks grab
// them from an atomic counter.  A tile of round r of pair b first waits until
// pair b has published round r - 1 (a bounded spin), then:
//   p' = R p + t  (FP32),  q = exact nearest target point of p' within the
//   rejection distance, n = normal of q, r = n.(p' - q), J = [p' x n, n],
// and accumulates H = sum J J^T (21 terms), g = sum J r (6), sum r^2 with
// compensated FP32 sums; the block writes the tile's partial sums.  The block
// that completes the last tile of a pair's round reduces that pair's tile
// partials in tile order (deterministic), solves H xi = -g in FP64 by
// Cholesky, left-composes T <- [exp(w^), tau; 0 1] T in FP64 and publishes the
// round.  The extra last round only evaluates the final RMSE.
// A round only depends on earlier tiles, which running blocks hold, so the
// schedule cannot deadlock; every wait still has an iteration limit and
// reports CIL_ERR_TIMEOUT instead of hanging.
#include <math.h>

#include "cil_host.h"
#include "cil_kernels.h"

namespace cil {

constexpr int kTileSrc = kIcpThreads * kIcpPPT;
constexpr int kIcpWarps = kIcpThreads / 32;
constexpr long long kSpinLimit = 1ll << 22;

__device__ __forceinline__ int ld_acquire_i32(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_i32(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

struct IcpArgs {
  GridView g;
  const float* src;
  const int* order;     // sorted position -> global source index
  const float* dst_n;   // concatenated target normals
  const int* tile_off;  // [pairs + 1] tile prefix
  const int* src_start; // [pairs + 1] (null: one pair of n_src1 points)
  int n_src1;
  int pairs;
  int n_tiles;
  int rounds;           // iterations + 1
  IcpPairState* st;
  float* part_s;
  float* part_c;
  int* part_n;
  unsigned* work;
  int* abort;
  int* err;
};

// Nearest target point within dmax2, also returning the point itself.  The
// search starts at the cloud's k-NN level with at most one ring around the
// query's cell (a converged source point finds its neighbour there); a query
// that is not resolved by then -- an outlier or a point still far from the
// surface -- restarts at the 8x coarser levels, where the rejection distance
// bounds the rings.  Exact either way: a level's result is taken only once
// the unexplored region lies beyond min(best, dmax).
__device__ __forceinline__ u64 nearest_within(const GridView& g, int cloud, const float q[3],
                                              float dmax2, float4& bp) {
  const GridParams& P = g.prm[cloud];
  const float inv_fine = P.inv_fine;
  u64 best = kEmptyKey;
  for (int lvl = P.level;; lvl = next_level(lvl)) {
    CellFrame f;
    f.load_level(P, cloud, lvl, ldexpf(P.fine, lvl));
    const int cx = f.cell_of(q[0], 0, inv_fine);
    const int cy = f.cell_of(q[1], 1, inv_fine);
    const int cz = f.cell_of(q[2], 2, inv_fine);
    const int rmax = max(max(max(cx, f.hi[0] - cx), max(cy, f.hi[1] - cy)), max(cz, f.hi[2] - cz));
    const int rcap = (lvl == P.level && lvl < kFineBits) ? min(rmax, 1) : rmax;
    best = kEmptyKey;
    float lim = dmax2;
    bool done = false;
    for (int r = 0; r <= rcap; ++r) {
      if (r > 0) {
        const int e0[3] = {cx - r + 1, cy - r + 1, cz - r + 1};
        const int e1[3] = {cx + r - 1, cy + r - 1, cz + r - 1};
        if (f.unexplored_d2(q, e0, e1) * (1.0f - 1e-6f) > lim) {
          done = true;
          break;
        }
      }
      CIL_SHELL_FOR(f, cx, cy, cz, r, x, y, z) {
        const int c3[3] = {x, y, z};
        if (f.range_d2(q, c3, c3) * (1.0f - 1e-6f) > lim) continue;
        int s, n;
        if (!cell_lookup(g, cell_key(lvl, cloud, x, y, z), s, n)) continue;
        for (int j = s; j < s + n; ++j) {
          const float4 p = __ldg(g.pts + j);
          const float d2 = sqdist(p.x, p.y, p.z, q[0], q[1], q[2]);
          if (d2 <= dmax2) {
            const u64 key = pack_key(d2, __float_as_int(p.w));
            if (key < best) {
              best = key;
              bp = p;
              lim = fminf(lim, d2);
            }
          }
        }
      }
      if (r == rmax) {
        done = true;
        break;
      }
    }
    if (!done) {
      const int e0[3] = {cx - rcap, cy - rcap, cz - rcap};
      const int e1[3] = {cx + rcap, cy + rcap, cz + rcap};
      done = f.unexplored_d2(q, e0, e1) * (1.0f - 1e-6f) > lim;
    }
    if (done || lvl >= kFineBits) break;
  }
  return best;
}

// SO(3) exponential (Rodrigues), FP64
__device__ void so3_exp_d(const double w[3], double R[9]) {
  const double t2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
  const double t = sqrt(t2);
  double a, b;  // sin(t)/t and (1 - cos(t))/t^2
  if (t < 1e-8) {
    a = 1.0 - t2 / 6.0;
    b = 0.5 - t2 / 24.0;
  } else {
    a = sin(t) / t;
    b = (1.0 - cos(t)) / t2;
  }
  // R = I + a [w]x + b [w]x^2, with [w]x^2 = w w^T - t2 I
  R[0] = 1.0 + b * (w[0] * w[0] - t2);
  R[1] = -a * w[2] + b * w[0] * w[1];
  R[2] = a * w[1] + b * w[0] * w[2];
  R[3] = a * w[2] + b * w[1] * w[0];
  R[4] = 1.0 + b * (w[1] * w[1] - t2);
  R[5] = -a * w[0] + b * w[1] * w[2];
  R[6] = -a * w[1] + b * w[2] * w[0];
  R[7] = a * w[0] + b * w[2] * w[1];
  R[8] = 1.0 + b * (w[2] * w[2] - t2);
}

// H x = -g by Cholesky in FP64; false if a pivot <= 1e-12 trace(H)
__device__ bool chol_solve6(const double H[36], const double g[6], double x[6]) {
  double L[36];
  double tr = 0.0;
  for (int a = 0; a < 6; ++a) tr += H[7 * a];
  if (!(tr > 0.0)) return false;
  for (int j = 0; j < 6; ++j) {
    double d = H[7 * j];
    for (int m = 0; m < j; ++m) d -= L[6 * j + m] * L[6 * j + m];
    if (!(d > 1e-12 * tr)) return false;
    const double l = sqrt(d);
    L[7 * j] = l;
    for (int i = j + 1; i < 6; ++i) {
      double v = H[6 * i + j];
      for (int m = 0; m < j; ++m) v -= L[6 * i + m] * L[6 * j + m];
      L[6 * i + j] = v / l;
    }
  }
  double y[6];
  for (int i = 0; i < 6; ++i) {
    double v = -g[i];
    for (int m = 0; m < i; ++m) v -= L[6 * i + m] * y[m];
    y[i] = v / L[7 * i];
  }
  for (int i = 5; i >= 0; --i) {
    double v = y[i];
    for (int m = i + 1; m < 6; ++m) v -= L[6 * m + i] * x[m];
    x[i] = v / L[7 * i];
  }
  return true;
}

__device__ __forceinline__ void rt_from_T(const double T[16], float Rt[12]) {
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 4; ++b) Rt[4 * a + b] = (float)T[4 * a + b];
}

__global__ void k_icp_setup(IcpPairState* st, int pairs, const int* src_start, int64_t n_src_single,
                            int* tile_off, const double* T_init, Mat4 T_host, int use_host_T,
                            const float* dmax_dev, float dmax, int iters, float* rt_out) {
  // single block: tile prefix over pairs
  __shared__ int carry;
  __shared__ int tmp[1024];
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < pairs; base += blockDim.x) {
    const int b = base + threadIdx.x;
    int nt = 0;
    if (b < pairs) {
      const int64_t n = src_start ? (int64_t)(src_start[b + 1] - src_start[b]) : n_src_single;
      nt = (int)((n + kTileSrc - 1) / kTileSrc);
    }
    // serial exclusive prefix of this chunk of pairs (pairs are few)
    tmp[threadIdx.x] = nt;
    __syncthreads();
    if (threadIdx.x == 0) {
      int run = carry;
      for (int j = 0; j < (int)blockDim.x && base + j < pairs; ++j) {
        const int v = tmp[j];
        tmp[j] = run;
        run += v;
      }
      carry = run;
    }
    __syncthreads();
    if (b < pairs) {
      IcpPairState& S = st[b];
      double T[16];
      for (int j = 0; j < 16; ++j)
        T[j] = use_host_T ? T_host.m[j]
                          : (T_init ? T_init[16 * b + j] : ((j % 5) == 0 ? 1.0 : 0.0));
      for (int j = 0; j < 16; ++j) S.T[j] = T[j];
      float Rt[12];
      rt_from_T(T, Rt);
      for (int j = 0; j < 12; ++j) {
        S.Rt[j] = Rt[j];
        rt_out[12 * b + j] = Rt[j];
      }
      const float d = dmax_dev ? dmax_dev[b] : dmax;
      S.dmax2 = d * d;
      S.tile_begin = tmp[threadIdx.x];
      S.tile_end = tmp[threadIdx.x] + nt;
      tile_off[b] = tmp[threadIdx.x];
      S.tiles_done = 0;
      S.iters = iters;
      S.rmse = __longlong_as_double(0x7ff8000000000000ll);
      S.n_inl = 0;
      if (nt == 0) {  // no source points: nothing to estimate
        S.status = iters > 0 ? (int)CIL_ERR_DEGENERATE : (int)CIL_OK;
        S.iter_done = iters + 1;
      } else {
        S.status = CIL_OK;
        S.iter_done = 0;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) tile_off[pairs] = carry;
}

__device__ __forceinline__ int pair_of_tile(const int* tile_off, int pairs, int tt) {
  int lo = 0, hi = pairs;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(tile_off + mid) <= tt) lo = mid;
    else hi = mid;
  }
  return lo;
}

__global__ void __launch_bounds__(kIcpThreads, 2) k_icp(IcpArgs a) {
  __shared__ unsigned s_t;
  __shared__ int s_go, s_last, s_pair;
  __shared__ float s_Rt[12];
  __shared__ float s_dmax2;
  __shared__ float sm_s[kIcpWarps][kIcpQ];
  __shared__ float sm_c[kIcpWarps][kIcpQ];
  __shared__ int sm_n[kIcpWarps];
  __shared__ double sm_tot[kIcpQ];
  __shared__ long long sm_cnt;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned total = (unsigned)a.n_tiles * (unsigned)a.rounds;

  for (;;) {
    if (tid == 0) {
      const unsigned t = atomicAdd(a.work, 1u);
      int go = (t < total) && (ld_acquire_i32(a.abort) == 0);
      int b = 0;
      if (go) {
        const int it = (int)(t / (unsigned)a.n_tiles);
        const int tt = (int)(t % (unsigned)a.n_tiles);
        b = pair_of_tile(a.tile_off, a.pairs, tt);
        if (it > 0) {
          long long spins = 0;
          unsigned ns = 32;
          while (ld_acquire_i32(&a.st[b].iter_done) < it) {
            if (ld_acquire_i32(a.abort)) {
              go = 0;
              break;
            }
            if (++spins > kSpinLimit) {
              atomicExch(a.abort, 1);
              atomicCAS(a.err, 0, (int)CIL_ERR_TIMEOUT);
              go = 0;
              break;
            }
            __nanosleep(ns);
            if (ns < 2048) ns <<= 1;
          }
        }
        if (go) {
          for (int j = 0; j < 12; ++j) s_Rt[j] = __ldcg(&a.st[b].Rt[j]);
          s_dmax2 = __ldcg(&a.st[b].dmax2);
        }
      }
      s_t = t;
      s_go = go;
      s_pair = b;
    }
    __syncthreads();
    if (!s_go) break;
    const int it = (int)(s_t / (unsigned)a.n_tiles);
    const int tt = (int)(s_t % (unsigned)a.n_tiles);
    const int b = s_pair;
    const int tb = __ldg(a.tile_off + b);
    const int sb = a.src_start ? __ldg(a.src_start + b) : 0;
    const int se = a.src_start ? __ldg(a.src_start + b + 1) : a.n_src1;
    const int lo = sb + (tt - tb) * kTileSrc;
    const int hi = min(se, lo + kTileSrc);
    const int dst_start = a.g.prm[b].start;

    float R[12];
#pragma unroll
    for (int j = 0; j < 12; ++j) R[j] = s_Rt[j];
    const float dmax2 = s_dmax2;
    // per-thread partials over its <= kIcpPPT points are plain FP32 (at most
    // 3 roundings each); every combination across threads below is
    // compensated (error-free TwoSum merges)
    float part[kIcpQ];
#pragma unroll
    for (int q = 0; q < kIcpQ; ++q) part[q] = 0.0f;
    int cnt = 0;
    for (int pos = lo + tid; pos < hi; pos += kIcpThreads) {
      const int64_t si = __ldg(a.order + pos);
      const float x = __ldg(a.src + 3 * si), y = __ldg(a.src + 3 * si + 1),
                  z = __ldg(a.src + 3 * si + 2);
      float p[3];
      p[0] = fmaf(R[0], x, fmaf(R[1], y, fmaf(R[2], z, R[3])));
      p[1] = fmaf(R[4], x, fmaf(R[5], y, fmaf(R[6], z, R[7])));
      p[2] = fmaf(R[8], x, fmaf(R[9], y, fmaf(R[10], z, R[11])));
      float4 qp;
      const u64 key = nearest_within(a.g, b, p, dmax2, qp);
      if (key == kEmptyKey) continue;
      const int64_t j = dst_start + (int64_t)key_idx(key);
      const float nx = __ldg(a.dst_n + 3 * j), ny = __ldg(a.dst_n + 3 * j + 1),
                  nz = __ldg(a.dst_n + 3 * j + 2);
      if (!(isfinite(nx) && isfinite(ny) && isfinite(nz))) continue;
      const float r = nx * (p[0] - qp.x) + ny * (p[1] - qp.y) + nz * (p[2] - qp.z);
      const float J[6] = {p[1] * nz - p[2] * ny, p[2] * nx - p[0] * nz, p[0] * ny - p[1] * nx,
                          nx, ny, nz};
      int q = 0;
#pragma unroll
      for (int u = 0; u < 6; ++u)
#pragma unroll
        for (int v = u; v < 6; ++v) {
          part[q] = fmaf(J[u], J[v], part[q]);
          ++q;
        }
#pragma unroll
      for (int u = 0; u < 6; ++u) part[21 + u] = fmaf(J[u], r, part[21 + u]);
      part[27] = fmaf(r, r, part[27]);
      ++cnt;
    }
    // block reduction of the tile (fixed shuffle tree, then warps in order),
    // compensated: each merge is an error-free TwoSum of the partial sums;
    // one quantity at a time keeps the live registers low
#pragma unroll
    for (int q = 0; q < kIcpQ; ++q) {
      KSum t;
      t.s = part[q];
      t.c = 0.0f;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const float s2 = __shfl_down_sync(0xffffffffu, t.s, off);
        const float c2 = __shfl_down_sync(0xffffffffu, t.c, off);
        t.merge(s2, c2);
      }
      if (lane == 0) {
        sm_s[warp][q] = t.s;
        sm_c[warp][q] = t.c;
      }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, off);
    if (lane == 0) sm_n[warp] = cnt;
    __syncthreads();
    if (tid < kIcpQ) {
      KSum t;
      t.zero();
      for (int w = 0; w < kIcpWarps; ++w) t.merge(sm_s[w][tid], sm_c[w][tid]);
      a.part_s[(int64_t)tt * kIcpQ + tid] = t.s;
      a.part_c[(int64_t)tt * kIcpQ + tid] = t.c;
    } else if (tid == 32) {
      int n = 0;
      for (int w = 0; w < kIcpWarps; ++w) n += sm_n[w];
      a.part_n[tt] = n;
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) {
      const int ntiles_b = __ldg(a.tile_off + b + 1) - tb;
      const int old = atomicAdd(&a.st[b].tiles_done, 1);
      s_last = (old == ntiles_b - 1);
    }
    __syncthreads();
    if (!s_last) continue;

    // ---- this block closes round `it` of pair b ----
    __threadfence();
    const int te = __ldg(a.tile_off + b + 1);
    for (int q = warp; q < kIcpQ; q += kIcpWarps) {
      KSum t;
      t.zero();
      for (int u = tb + lane; u < te; u += 32)
        t.merge(__ldcg(a.part_s + (int64_t)u * kIcpQ + q), __ldcg(a.part_c + (int64_t)u * kIcpQ + q));
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const float s2 = __shfl_down_sync(0xffffffffu, t.s, off);
        const float c2 = __shfl_down_sync(0xffffffffu, t.c, off);
        t.merge(s2, c2);
      }
      if (lane == 0) sm_tot[q] = (double)t.s + (double)t.c;
    }
    if (warp == kIcpWarps - 1) {
      long long n = 0;
      for (int u = tb + lane; u < te; u += 32) n += __ldcg(a.part_n + u);
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) n += __shfl_down_sync(0xffffffffu, n, off);
      if (lane == 0) sm_cnt = n;
    }
    __syncthreads();
    if (tid == 0) {
      IcpPairState& S = a.st[b];
      const long long n = sm_cnt;
      if (it == a.rounds - 1) {
        S.n_inl = n;
        S.rmse = n > 0 ? sqrt(sm_tot[27] / (double)n) : __longlong_as_double(0x7ff8000000000000ll);
      } else {
        double H[36], g[6], xi[6];
        int q = 0;
        for (int u = 0; u < 6; ++u)
          for (int v = u; v < 6; ++v) {
            H[6 * u + v] = sm_tot[q];
            H[6 * v + u] = sm_tot[q];
            ++q;
          }
        for (int u = 0; u < 6; ++u) g[u] = sm_tot[21 + u];
        if (n < 6 || !chol_solve6(H, g, xi)) {
          S.status = CIL_ERR_DEGENERATE;
        } else {
          double T[16], dR[9], Tn[16];
          for (int j = 0; j < 16; ++j) T[j] = __ldcg(&S.T[j]);
          so3_exp_d(xi, dR);
          for (int u = 0; u < 3; ++u) {
            for (int v = 0; v < 4; ++v)
              Tn[4 * u + v] = dR[3 * u] * T[v] + dR[3 * u + 1] * T[4 + v] + dR[3 * u + 2] * T[8 + v];
            Tn[4 * u + 3] += xi[3 + u];
          }
          Tn[12] = 0.0;
          Tn[13] = 0.0;
          Tn[14] = 0.0;
          Tn[15] = 1.0;
          for (int j = 0; j < 16; ++j) S.T[j] = Tn[j];
          float Rt[12];
          rt_from_T(Tn, Rt);
          for (int j = 0; j < 12; ++j) S.Rt[j] = Rt[j];
        }
      }
      S.tiles_done = 0;
      __threadfence();
      st_release_i32(&S.iter_done, it + 1);
    }
    __syncthreads();
  }
}

__global__ void k_icp_export(const IcpPairState* st, int pairs, double* T_out,
                             cil_icp_report* rep) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= pairs) return;
  const IcpPairState& S = st[b];
  if (T_out)
    for (int j = 0; j < 16; ++j) T_out[16 * b + j] = S.T[j];
  if (rep) {
    cil_icp_report r;
    r.rmse = S.rmse;
    r.n_inliers = S.n_inl;
    r.iters_done = S.iters;
    r.status = S.status;
    rep[b] = r;
  }
}

// ---------------------------------------------------------------------------
void icp_plan(IcpPlan& p, Workspace& ws, const int64_t* src_counts, int pairs) {
  p.pairs = pairs;
  p.n_src = 0;
  p.n_tiles = 0;
  p.tile = kTileSrc;
  for (int b = 0; b < pairs; ++b) {
    p.n_src += src_counts[b];
    p.n_tiles += ceil_div(src_counts[b], kTileSrc);
  }
  const int nt = p.n_tiles > 0 ? p.n_tiles : 1;
  p.o_state = ws.reserve(sizeof(IcpPairState) * pairs);
  p.o_order = ws.reserve(sizeof(int) * (size_t)(p.n_src > 0 ? p.n_src : 1));
  p.o_tile_off = ws.reserve(sizeof(int) * (pairs + 1));
  p.o_rt = ws.reserve(sizeof(float) * 12 * pairs);
  p.o_part_s = ws.reserve(sizeof(float) * kIcpQ * nt);
  p.o_part_c = ws.reserve(sizeof(float) * kIcpQ * nt);
  p.o_part_n = ws.reserve(sizeof(int) * nt);
  p.o_work = ws.reserve(sizeof(unsigned) * 4);
  order_plan(p.order, ws, p.n_src);
}

IcpPairState* icp_state(const IcpPlan& p, const Workspace& ws) {
  return ws.at<IcpPairState>(p.o_state);
}

cil_status icp_run(const IcpPlan& p, const Workspace& ws, const GridView& tgt, const float* src,
                   const int* src_start_dev, const float* dst_normals, const double* T_init_dev,
                   const double* T_init_host, int iters, const float* dmax_dev, float dmax,
                   DeviceCtx* ctx, cudaStream_t s) {
  Mat4 Th;
  for (int j = 0; j < 16; ++j) Th.m[j] = T_init_host ? T_init_host[j] : 0.0;
  IcpPairState* st = ws.at<IcpPairState>(p.o_state);
  int* tile_off = ws.at<int>(p.o_tile_off);
  float* rt = ws.at<float>(p.o_rt);
  unsigned* work = ws.at<unsigned>(p.o_work);
  note_launches(1);
  k_icp_setup<<<1, 1024, 0, s>>>(st, p.pairs, src_start_dev, p.n_src, tile_off, T_init_dev, Th,
                                 T_init_host != nullptr, dmax_dev, dmax, iters, rt);
  if (cudaMemsetAsync(work, 0, sizeof(unsigned) * 4, s) != cudaSuccess) return CIL_ERR_CUDA;
  int* order = ws.at<int>(p.o_order);
  cil_status stt = order_queries(p.order, ws, src, src_start_dev, p.pairs, tgt.prm, rt, order, s);
  if (stt != CIL_OK) return stt;
  if (p.n_tiles == 0) return cudaGetLastError() == cudaSuccess ? CIL_OK : CIL_ERR_CUDA;
  IcpArgs a;
  a.g = tgt;
  a.src = src;
  a.order = order;
  a.dst_n = dst_normals;
  a.tile_off = tile_off;
  a.src_start = src_start_dev;
  a.n_src1 = (int)p.n_src;
  a.pairs = p.pairs;
  a.n_tiles = p.n_tiles;
  a.rounds = iters + 1;
  a.st = st;
  a.part_s = ws.at<float>(p.o_part_s);
  a.part_c = ws.at<float>(p.o_part_c);
  a.part_n = ws.at<int>(p.o_part_n);
  a.work = work;
  a.abort = reinterpret_cast<int*>(work + 1);
  a.err = ctx->err;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_icp, kIcpThreads, 0);
  if (per_sm < 1) per_sm = 1;
  const long long want = (long long)p.n_tiles * a.rounds;
  int grid = ctx->num_sms * per_sm;
  if (want < grid) grid = (int)want;
  {
    TimedRegion timer("k_icp", s);
    note_launches(1);
    k_icp<<<grid, kIcpThreads, 0, s>>>(a);
  }
  return cudaGetLastError() == cudaSuccess ? CIL_OK : CIL_ERR_CUDA;
}

cil_status icp_export(const IcpPlan& p, const Workspace& ws, double* T_out_dev,
                      cil_icp_report* rep_dev, cudaStream_t s) {
  note_launches(1);
  k_icp_export<<<ceil_div(p.pairs, 128), 128, 0, s>>>(ws.at<IcpPairState>(p.o_state), p.pairs,
                                                      T_out_dev, rep_dev);
  return cudaGetLastError() == cudaSuccess ? CIL_OK : CIL_ERR_CUDA;
}

}  // namespace cil
