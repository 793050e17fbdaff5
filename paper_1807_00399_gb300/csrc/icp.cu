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
// compensated FP32 sums; the block writes the tile's partial sums.  Tiles
// form groups of kIcpGroup: the block that completes a group's last tile
// reduces the group in a fixed order, and the block that completes a pair's
// last group reduces the group partials in order (deterministic), solves
// H xi = -g in FP64 by Cholesky, left-composes T <- [exp(w^), tau; 0 1] T in
// FP64 and publishes the round.  The extra last round only evaluates the
// final RMSE.
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
  float* grp_s;
  float* grp_c;
  int* grp_n;
  int* grp_done;
  unsigned* work;
  int* abort;
  int* err;
};

constexpr int kDirLevels = 2;     // directory level = base level + 2 (in the cell table)
constexpr int kDirCells = 125;    // directory cells meeting the ball at most
constexpr int kDirectScan = 128;  // coarse cells up to this many points are scanned whole
constexpr int kLookupCost = 4;

// Points of one cell that improve on (best, lim); lim = min(dmax2, best d^2).
__device__ __forceinline__ void scan_cell(const GridView& g, int s, int n, const float q[3],
                                          float dmax2, u64& best, int& bj, float& lim) {
  for_points(g.pts, s, n, [&](const float4& p, int j) {
    const float d2 = sqdist(p.x, p.y, p.z, q[0], q[1], q[2]);
    const u64 key = pack_key(d2, __float_as_int(p.w));
    if (d2 <= dmax2 && key < best) {
      best = key;
      bj = j;
      lim = fminf(lim, d2);
    }
  });
}

// The ball of radius sqrt(lim) around q leaves the 3x3x3 block around the
// base-level cell c (already searched).  The cells of the directory level
// (4x the base edge, hashed in the table for this) meeting the ball act as a
// directory: empty ones are skipped whole, small ones scanned,
// and in large ones that the ball meets in few base-level cells only those
// cells are looked up (dense surfaces seen from off the surface stay cheap).
// Returns false, having searched nothing, when the ball spans more than
// kDirCells coarse cells (large rejection distances), and true once every
// cell meeting the ball has been searched.
__device__ __forceinline__ bool escalate_directory(const GridView& g, int cloud, const float q[3],
                                                float dmax2, const int c[3], u64& best, int& bj,
                                                float& lim) {
  const GridParams& P = g.prm[cloud];
  const float inv_fine = P.inv_fine;
  CellFrame f;
  f.load(P, cloud);
  int s, n;
  const int Lc = min(f.level + kDirLevels, kFineBits);
  CellFrame fc;
  fc.load_level(P, cloud, Lc, ldexpf(P.fine, Lc));
  const float rad2 = fmaf(sqrtf(lim), 1.0f + 1e-6f, f.eps);
  int clo[3], chi[3], blo[3], bhi[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    clo[a] = fc.cell_of(q[a] - rad2, a, inv_fine);
    chi[a] = fc.cell_of(q[a] + rad2, a, inv_fine);
    blo[a] = f.cell_of(q[a] - rad2, a, inv_fine);
    bhi[a] = f.cell_of(q[a] + rad2, a, inv_fine);
  }
  if ((chi[0] - clo[0] + 1) * (chi[1] - clo[1] + 1) * (chi[2] - clo[2] + 1) <= kDirCells) {
    const int sh = Lc - f.level;
    for (int Z = clo[2]; Z <= chi[2]; ++Z)
      for (int Y = clo[1]; Y <= chi[1]; ++Y)
        for (int X = clo[0]; X <= chi[0]; ++X) {
          const int C3[3] = {X, Y, Z};
          if (fc.range_d2(q, C3, C3) * (1.0f - 1e-6f) > lim) continue;
          if (!cell_lookup(g, cell_key(Lc, cloud, X, Y, Z), s, n)) continue;
          const int zl = max(Z << sh, blo[2]), zh = min(((Z + 1) << sh) - 1, bhi[2]);
          const int yl = max(Y << sh, blo[1]), yh = min(((Y + 1) << sh) - 1, bhi[1]);
          const int xl = max(X << sh, blo[0]), xh = min(((X + 1) << sh) - 1, bhi[0]);
          // a base-level lookup costs about kLookupCost streamed point tests
          if (n <= kDirectScan || n < kLookupCost * (xh - xl + 1) * (yh - yl + 1) * (zh - zl + 1)) {
            scan_cell(g, s, n, q, dmax2, best, bj, lim);
            continue;
          }
          for (int z = zl; z <= zh; ++z)
            for (int y = yl; y <= yh; ++y)
              for (int x = xl; x <= xh; ++x) {
                if (abs(x - c[0]) <= 1 && abs(y - c[1]) <= 1 && abs(z - c[2]) <= 1)
                  continue;  // searched by the caller
                const int c3[3] = {x, y, z};
                if (f.range_d2(q, c3, c3) * (1.0f - 1e-6f) > lim) continue;
                int s2, n2;
                if (cell_lookup(g, cell_key(f.level, cloud, x, y, z), s2, n2))
                  scan_cell(g, s2, n2, q, dmax2, best, bj, lim);
              }
        }
    return true;  // every cell meeting the ball was searched
  }
  return false;
}

// Ring search from the first coarser level upward (kRingCap rings per level)
// for balls too large for the directory search.
__device__ __forceinline__ void escalate_rings(const GridView& g, int cloud, const float q[3],
                                            float dmax2, u64& best, int& bj, float& lim) {
  const GridParams& P = g.prm[cloud];
  const float inv_fine = P.inv_fine;
  for (int lvl = next_level(P.level);; lvl = next_level(lvl)) {
    CellFrame f;
    f.load_level(P, cloud, lvl, ldexpf(P.fine, lvl));
    const int cx = f.cell_of(q[0], 0, inv_fine);
    const int cy = f.cell_of(q[1], 1, inv_fine);
    const int cz = f.cell_of(q[2], 2, inv_fine);
    const int rmax = max(max(max(cx, f.hi[0] - cx), max(cy, f.hi[1] - cy)), max(cz, f.hi[2] - cz));
    const int rcap = lvl >= kFineBits ? rmax : min(rmax, kRingCap);
    for (int r = 0; r <= rcap; ++r) {
      if (r > 0) {
        const int e0[3] = {cx - r + 1, cy - r + 1, cz - r + 1};
        const int e1[3] = {cx + r - 1, cy + r - 1, cz + r - 1};
        if (f.unexplored_d2(q, e0, e1) * (1.0f - 1e-6f) > lim) return;
      }
      CIL_SHELL_FOR(f, cx, cy, cz, r, x, y, z) {
        const int c3[3] = {x, y, z};
        if (f.range_d2(q, c3, c3) * (1.0f - 1e-6f) > lim) continue;
        int s, n;
        if (cell_lookup(g, cell_key(lvl, cloud, x, y, z), s, n))
          scan_cell(g, s, n, q, dmax2, best, bj, lim);
      }
    }
    if (rcap == rmax) return;  // every ring of this level searched
    const int e0[3] = {cx - rcap, cy - rcap, cz - rcap};
    const int e1[3] = {cx + rcap, cy + rcap, cz + rcap};
    if (f.unexplored_d2(q, e0, e1) * (1.0f - 1e-6f) > lim) return;
  }
}

// Nearest target point within dmax2 (sorted position in bj, key returned, or
// kEmptyKey).  At the cloud's own level the query's cell is scanned first;
// then only the cells of its 3x3x3 block that meet the ball of the best
// distance so far (a converged source point finds its neighbour there).  A
// query whose ball leaves the block -- an outlier or a point still far from
// the surface -- continues with a ring search at the 8x coarser levels, where
// the rejection distance bounds the rings.  Exact: a level's search ends only
// once the unexplored region lies beyond min(best, dmax).
__device__ __forceinline__ u64 nearest_within(const GridView& g, int cloud, const float q[3],
                                              float dmax2, int& bj) {
  const GridParams& P = g.prm[cloud];
  const float inv_fine = P.inv_fine;
  u64 best = kEmptyKey;
  float lim = dmax2;
  bj = -1;
  {
    CellFrame f;
    f.load(P, cloud);
    const int c[3] = {f.cell_of(q[0], 0, inv_fine), f.cell_of(q[1], 1, inv_fine),
                      f.cell_of(q[2], 2, inv_fine)};
    int s, n;
    if (cell_lookup(g, cell_key(f.level, cloud, c[0], c[1], c[2]), s, n))
      scan_cell(g, s, n, q, dmax2, best, bj, lim);
    if (f.level >= kFineBits) return best;  // one cell holds the whole cloud
    // cells of the block meeting the ball of radius sqrt(lim) (padded)
    const float rad = fmaf(sqrtf(lim), 1.0f + 1e-6f, f.eps);
    int lo[3], hi[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      lo[a] = max(f.cell_of(q[a] - rad, a, inv_fine), c[a] - 1);
      hi[a] = min(f.cell_of(q[a] + rad, a, inv_fine), c[a] + 1);
    }
    for (int z = lo[2]; z <= hi[2]; ++z)
      for (int y = lo[1]; y <= hi[1]; ++y)
        for (int x = lo[0]; x <= hi[0]; ++x) {
          if (x == c[0] && y == c[1] && z == c[2]) continue;
          const int c3[3] = {x, y, z};
          if (f.range_d2(q, c3, c3) * (1.0f - 1e-6f) > lim) continue;
          if (cell_lookup(g, cell_key(f.level, cloud, x, y, z), s, n))
            scan_cell(g, s, n, q, dmax2, best, bj, lim);
        }
    const int e0[3] = {c[0] - 1, c[1] - 1, c[2] - 1};
    const int e1[3] = {c[0] + 1, c[1] + 1, c[2] + 1};
    if (f.unexplored_d2(q, e0, e1) * (1.0f - 1e-6f) > lim) return best;

    if (escalate_directory(g, cloud, q, dmax2, c, best, bj, lim)) return best;
  }
  // a ball spanning many coarse cells (large rejection distance)
  escalate_rings(g, cloud, q, dmax2, best, bj, lim);
  return best;
}

// FP64 runs at 1/64 of the FP32 rate on this part, so the two solvers below
// are written for few FP64 instructions: one reciprocal square root per
// Cholesky column instead of a square root and a division per entry, and one
// sincos of the half angle for the rotation.

// SO(3) exponential (Rodrigues), FP64.  With t = |w|, s = sin(t/2), c = cos(t/2):
// sin(t)/t = 2 s c / t and (1 - cos t)/t^2 = 2 s^2 / t^2 (no cancellation).
__device__ void so3_exp_d(const double w[3], double R[9]) {
  const double t2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
  double a, b;  // sin(t)/t and (1 - cos(t))/t^2
  if (t2 < 1e-16) {
    a = 1.0 - t2 / 6.0;
    b = 0.5 - t2 / 24.0;
  } else {
    const double it = rsqrt(t2);  // 1/t
    double s, c;
    sincos(0.5 * (t2 * it), &s, &c);
    const double si = s * it;
    a = 2.0 * si * c;
    b = 2.0 * si * si;
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

// H x = -g by Cholesky H = L L^T in FP64; false if a pivot <= 1e-12 trace(H).
// Only the reciprocals of L's diagonal are kept (r_j = 1 / L_jj).
__device__ bool chol_solve6(const double H[36], const double g[6], double x[6]) {
  double L[36], r[6];
  double tr = 0.0;
  for (int a = 0; a < 6; ++a) tr += H[7 * a];
  if (!(tr > 0.0)) return false;
  const double piv_min = 1e-12 * tr;
  for (int j = 0; j < 6; ++j) {
    double d = H[7 * j];
    for (int m = 0; m < j; ++m) d = fma(-L[6 * j + m], L[6 * j + m], d);
    if (!(d > piv_min)) return false;
    r[j] = rsqrt(d);
    for (int i = j + 1; i < 6; ++i) {
      double v = H[6 * i + j];
      for (int m = 0; m < j; ++m) v = fma(-L[6 * i + m], L[6 * j + m], v);
      L[6 * i + j] = v * r[j];
    }
  }
  double y[6];
  for (int i = 0; i < 6; ++i) {
    double v = -g[i];
    for (int m = 0; m < i; ++m) v = fma(-L[6 * i + m], y[m], v);
    y[i] = v * r[i];
  }
  for (int i = 5; i >= 0; --i) {
    double v = y[i];
    for (int m = i + 1; m < 6; ++m) v = fma(-L[6 * m + i], x[m], v);
    x[i] = v * r[i];
  }
  return true;
}

__device__ __forceinline__ void rt_from_T(const double T[16], float Rt[12]) {
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 4; ++b) Rt[4 * a + b] = (float)T[4 * a + b];
}

// Round close of one pair (one thread): the final round records the RMSE and
// inlier count; any other solves H xi = -g and left-composes the update.
// Out of line so that its FP64 temporaries do not count against the
// registers of the search.
__device__ __noinline__ void close_round(IcpPairState& S, const double* tot, long long n,
                                         bool final_round) {
  if (final_round) {
    S.n_inl = n;
    S.rmse = n > 0 ? sqrt(tot[27] / (double)n) : __longlong_as_double(0x7ff8000000000000ll);
    return;
  }
  double H[36], g[6], xi[6];
  int q = 0;
  for (int u = 0; u < 6; ++u)
    for (int v = u; v < 6; ++v) {
      H[6 * u + v] = tot[q];
      H[6 * v + u] = tot[q];
      ++q;
    }
  for (int u = 0; u < 6; ++u) g[u] = tot[21 + u];
  if (n < 6 || !chol_solve6(H, g, xi)) {
    S.status = CIL_ERR_DEGENERATE;
    return;
  }
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

__global__ void k_icp_setup(IcpPairState* st, int pairs, const int* src_start, int64_t n_src_single,
                            int* tile_off, const double* T_init, Mat4 T_host, int use_host_T,
                            const float* dmax_dev, float dmax, int iters, float* rt_out) {
  // single block: tile prefix over pairs
  __shared__ int carry, gcarry;
  __shared__ int tmp[1024], gtmp[1024];
  if (threadIdx.x == 0) {
    carry = 0;
    gcarry = 0;
  }
  __syncthreads();
  for (int base = 0; base < pairs; base += blockDim.x) {
    const int b = base + threadIdx.x;
    int nt = 0;
    if (b < pairs) {
      const int64_t n = src_start ? (int64_t)(src_start[b + 1] - src_start[b]) : n_src_single;
      nt = (int)((n + kTileSrc - 1) / kTileSrc);
    }
    // serial exclusive prefix of this chunk of pairs (pairs are few)
    const int ng = (nt + kIcpGroup - 1) / kIcpGroup;
    tmp[threadIdx.x] = nt;
    gtmp[threadIdx.x] = ng;
    __syncthreads();
    if (threadIdx.x == 0) {
      int run = carry, grun = gcarry;
      for (int j = 0; j < (int)blockDim.x && base + j < pairs; ++j) {
        const int v = tmp[j], w = gtmp[j];
        tmp[j] = run;
        gtmp[j] = grun;
        run += v;
        grun += w;
      }
      carry = run;
      gcarry = grun;
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
      S.grp_begin = gtmp[threadIdx.x];
      S.n_grp = ng;
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

// Operands of sum q of the normal equations in a row (J0..J5, r):
// q = 0..20 the upper triangle of J J^T row by row, 21..26 J r, 27 r r.
__device__ __forceinline__ void q_operands(int q, int& ia, int& ib) {
  if (q >= 21) {
    ia = q == 27 ? 6 : q - 21;
    ib = 6;
    return;
  }
  int u = 0, base = 0;
  while (q >= base + 6 - u) {
    base += 6 - u;
    ++u;
  }
  ia = u;
  ib = u + (q - base);
}

constexpr int kRowChunks = 8;  // chunks of a tile's rows summed in parallel

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
  __shared__ int s_go, s_last, s_pair, s_gid, s_g0, s_gsize;
  __shared__ float s_Rt[12];
  __shared__ float s_dmax2;
  __shared__ int s_corr[kTileSrc];
  __shared__ float s_row[7][kTileSrc + 8];  // J (6) and r per tile point; +8 spreads banks
  __shared__ float s_ps[kIcpQ][kRowChunks], s_pc[kIcpQ][kRowChunks];
  __shared__ int s_cnt;
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
            if (ns < 512) ns <<= 1;
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

    const float dmax2 = s_dmax2;
    // phase 1: correspondences (sorted target position or -1) of the tile's
    // points, kept in shared memory so that the search and the accumulation
    // below do not hold their registers at the same time
#pragma unroll 1
    for (int pass = 0; pass < kIcpPPT; ++pass) {
      const int pos = lo + pass * kIcpThreads + tid;
      int bj = -1;
      if (pos < hi) {
        const int64_t si = __ldg(a.order + pos);
        const float x = __ldg(a.src + 3 * si), y = __ldg(a.src + 3 * si + 1),
                    z = __ldg(a.src + 3 * si + 2);
        float p[3];
        p[0] = fmaf(s_Rt[0], x, fmaf(s_Rt[1], y, fmaf(s_Rt[2], z, s_Rt[3])));
        p[1] = fmaf(s_Rt[4], x, fmaf(s_Rt[5], y, fmaf(s_Rt[6], z, s_Rt[7])));
        p[2] = fmaf(s_Rt[8], x, fmaf(s_Rt[9], y, fmaf(s_Rt[10], z, s_Rt[11])));
        nearest_within(a.g, b, p, dmax2, bj);
      }
      s_corr[pass * kIcpThreads + tid] = bj;
    }
    // phase 2: the residual and Jacobian row of each point of the tile into
    // shared memory (zeros where there is no correspondence)
    if (tid == 0) s_cnt = 0;
    int cnt = 0;
#pragma unroll 1
    for (int pass = 0; pass < kIcpPPT; ++pass) {
      const int u = pass * kIcpThreads + tid;
      const int pos = lo + u;
      const int bj = s_corr[u];
      float row[7] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
      if (pos < hi && bj >= 0) {
        const int64_t si = __ldg(a.order + pos);
        const float x = __ldg(a.src + 3 * si), y = __ldg(a.src + 3 * si + 1),
                    z = __ldg(a.src + 3 * si + 2);
        float p[3];
        p[0] = fmaf(s_Rt[0], x, fmaf(s_Rt[1], y, fmaf(s_Rt[2], z, s_Rt[3])));
        p[1] = fmaf(s_Rt[4], x, fmaf(s_Rt[5], y, fmaf(s_Rt[6], z, s_Rt[7])));
        p[2] = fmaf(s_Rt[8], x, fmaf(s_Rt[9], y, fmaf(s_Rt[10], z, s_Rt[11])));
        const float4 qp = __ldg(a.g.pts + bj);
        const int64_t j = dst_start + (int64_t)__float_as_int(qp.w);
        const float nx = __ldg(a.dst_n + 3 * j), ny = __ldg(a.dst_n + 3 * j + 1),
                    nz = __ldg(a.dst_n + 3 * j + 2);
        if (isfinite(nx) && isfinite(ny) && isfinite(nz)) {
          row[0] = p[1] * nz - p[2] * ny;
          row[1] = p[2] * nx - p[0] * nz;
          row[2] = p[0] * ny - p[1] * nx;
          row[3] = nx;
          row[4] = ny;
          row[5] = nz;
          row[6] = nx * (p[0] - qp.x) + ny * (p[1] - qp.y) + nz * (p[2] - qp.z);
          ++cnt;
        }
      }
#pragma unroll
      for (int k = 0; k < 7; ++k) s_row[k][u] = row[k];
    }
    __syncthreads();
    if (cnt) atomicAdd(&s_cnt, cnt);
    // the tile's 21 + 6 + 1 sums: item (q, ch) adds the products of rows
    // ch, ch + kRowChunks, ... in that order (compensated), then the chunks
    // are merged in order -- a fixed order, so the result is deterministic
    for (int w = tid; w < kIcpQ * kRowChunks; w += kIcpThreads) {
      const int q = w / kRowChunks, ch = w - q * kRowChunks;
      int ia, ib;
      q_operands(q, ia, ib);
      KSum t;
      t.zero();
      for (int i = ch; i < kTileSrc; i += kRowChunks) t.add(__fmul_rn(s_row[ia][i], s_row[ib][i]));
      s_ps[q][ch] = t.s;
      s_pc[q][ch] = t.c;
    }
    __syncthreads();
    if (tid < kIcpQ) {
      KSum t;
      t.zero();
      for (int ch = 0; ch < kRowChunks; ++ch) t.merge(s_ps[tid][ch], s_pc[tid][ch]);
      a.part_s[(int64_t)tt * kIcpQ + tid] = t.s;
      a.part_c[(int64_t)tt * kIcpQ + tid] = t.c;
    } else if (tid == 32) {
      a.part_n[tt] = s_cnt;
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) {
      const int ntiles_b = __ldg(a.tile_off + b + 1) - tb;
      const int gl = (tt - tb) / kIcpGroup;
      const int gid = a.st[b].grp_begin + gl;
      const int gsize = min(kIcpGroup, ntiles_b - gl * kIcpGroup);
      const int old = atomicAdd(a.grp_done + gid, 1);
      s_last = (old == gsize - 1);
      s_gid = gid;
      s_g0 = tb + gl * kIcpGroup;
      s_gsize = gsize;
    }
    __syncthreads();
    if (!s_last) continue;

    // ---- this block reduces its tile group: tile u of the group in lane u,
    // a fixed compensated shuffle tree ----
    __threadfence();
    {
      const int gid = s_gid, g0 = s_g0, gs = s_gsize;
      for (int q = warp; q < kIcpQ; q += kIcpWarps) {
        KSum t;
        t.zero();
        if (lane < gs) {
          t.s = __ldcg(a.part_s + (int64_t)(g0 + lane) * kIcpQ + q);
          t.c = __ldcg(a.part_c + (int64_t)(g0 + lane) * kIcpQ + q);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
          const float s2 = __shfl_down_sync(0xffffffffu, t.s, off);
          const float c2 = __shfl_down_sync(0xffffffffu, t.c, off);
          t.merge(s2, c2);
        }
        if (lane == 0) {
          a.grp_s[(int64_t)gid * kIcpQ + q] = t.s;
          a.grp_c[(int64_t)gid * kIcpQ + q] = t.c;
        }
      }
      if (warp == kIcpWarps - 1) {
        int n = lane < gs ? __ldcg(a.part_n + g0 + lane) : 0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) n += __shfl_down_sync(0xffffffffu, n, off);
        if (lane == 0) a.grp_n[gid] = n;
      }
      // every tile of this group has been counted for this round; the next
      // round's tiles start only after the round is published
      if (tid == 0) a.grp_done[gid] = 0;
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) {
      const int old = atomicAdd(&a.st[b].tiles_done, 1);
      s_last = (old == a.st[b].n_grp - 1);
    }
    __syncthreads();
    if (!s_last) continue;

    // ---- this block closes round `it` of pair b: group partials in order ----
    __threadfence();
    {
      const int gb = a.st[b].grp_begin, ge = gb + a.st[b].n_grp;
      for (int q = warp; q < kIcpQ; q += kIcpWarps) {
        KSum t;
        t.zero();
        for (int u = gb + lane; u < ge; u += 32)
          t.merge(__ldcg(a.grp_s + (int64_t)u * kIcpQ + q), __ldcg(a.grp_c + (int64_t)u * kIcpQ + q));
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
        for (int u = gb + lane; u < ge; u += 32) n += __ldcg(a.grp_n + u);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) n += __shfl_down_sync(0xffffffffu, n, off);
        if (lane == 0) sm_cnt = n;
      }
    }
    __syncthreads();
    if (tid == 0) {
      IcpPairState& S = a.st[b];
      close_round(S, sm_tot, sm_cnt, it == a.rounds - 1);
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
  p.n_groups = 0;
  p.tile = kTileSrc;
  for (int b = 0; b < pairs; ++b) {
    p.n_src += src_counts[b];
    const int64_t t = ceil_div(src_counts[b], kTileSrc);
    p.n_tiles += t;
    p.n_groups += ceil_div(t, kIcpGroup);
  }
  const int nt = p.n_tiles > 0 ? p.n_tiles : 1;
  p.o_state = ws.reserve(sizeof(IcpPairState) * pairs);
  p.o_order = ws.reserve(sizeof(int) * (size_t)(p.n_src > 0 ? p.n_src : 1));
  p.o_tile_off = ws.reserve(sizeof(int) * (pairs + 1));
  p.o_rt = ws.reserve(sizeof(float) * 12 * pairs);
  p.o_part_s = ws.reserve(sizeof(float) * kIcpQ * nt);
  p.o_part_c = ws.reserve(sizeof(float) * kIcpQ * nt);
  p.o_part_n = ws.reserve(sizeof(int) * nt);
  const int ng = p.n_groups > 0 ? p.n_groups : 1;
  p.o_grp_s = ws.reserve(sizeof(float) * kIcpQ * ng);
  p.o_grp_c = ws.reserve(sizeof(float) * kIcpQ * ng);
  p.o_grp_n = ws.reserve(sizeof(int) * ng);
  p.o_grp_done = ws.reserve(sizeof(int) * ng);
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
  if (cudaMemsetAsync(ws.at<int>(p.o_grp_done), 0,
                      sizeof(int) * (size_t)(p.n_groups > 0 ? p.n_groups : 1), s) != cudaSuccess)
    return CIL_ERR_CUDA;
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
  a.grp_s = ws.at<float>(p.o_grp_s);
  a.grp_c = ws.at<float>(p.o_grp_c);
  a.grp_n = ws.at<int>(p.o_grp_n);
  a.grp_done = ws.at<int>(p.o_grp_done);
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
