// radius.cu -- fixed-radius neighbour search (Sec. 3, KDTree radius query).
//
// Grid cells are sized to the radius (nearest power-of-two multiple of the
// fine lattice), so each query's ball meets at most 4 x 4 x 4 cells.  One
// warp per query, queries in the grid's Morton order (neighbouring warps read
// the same cells through L1):
//   count  the lanes look up the ball's cells in parallel, the cells' points
//          are concatenated and split over the lanes, and accepted points
//          (d2 <= r*r, inclusive) are counted with a ballot;
//   scan   int64 CSR offsets (rows longer than kRowCapW are listed);
//   fill   the same walk; accepted (index, d2) appended to the query's CSR
//          row in visiting order (ballot positions: coalesced stores); no
//          shared memory, so it runs at the count pass's occupancy;
//   sort   rows up to kRowCapW keys: one warp per row, a bucket sort in
//          shared memory by (d2, index) -- buckets of d2 * NB / r^2 (a
//          monotone map, so bucket order agrees with key order), histogram
//          and scan, the keys scattered into bucket order, each bucket
//          insertion-sorted by its lane, the row written back coalesced;
//          longer rows (listed by the count pass): one block each, an
//          all-ascending bitonic network (in shared memory up to kRowCap
//          keys, else in place in global memory; virtual +inf padding past
//          the row end never moves).
#include <math.h>

#include "cil_host.h"
#include "cil_kernels.h"

namespace cil {

constexpr int kRowCap = 4096;      // block sort: rows up to this many keys in shared memory
constexpr int kSortThreads = 256;
constexpr int kRowCapW = 1024;     // warp sort: rows up to this many keys in shared memory
constexpr int kBucketsMax = 512;   // buckets of the warp sort (a power of two)
constexpr int kCountWarps = 8;     // warps (queries) per block of the count pass
constexpr int kSortWarps = 4;      // warps (rows) per block of the warp sort

// Cells of the query's ball: the range [lo, hi] of cells meeting the cube of
// half-edge r + eps around q, walked 32 at a time (lane c takes cell c of the
// chunk), each looked up if its box meets the ball.
struct BallCells {
  int lo[3], nx, nxy, ncell;
  float inv_nx, inv_nxy;
  __device__ __forceinline__ void init(const CellFrame& f, const GridParams& P, const float q[3],
                                       float r) {
    int hi[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      lo[a] = f.cell_of(q[a] - r - f.eps, a, P.inv_fine);
      hi[a] = f.cell_of(q[a] + r + f.eps, a, P.inv_fine);
    }
    nx = hi[0] - lo[0] + 1;
    nxy = nx * (hi[1] - lo[1] + 1);
    ncell = nxy * (hi[2] - lo[2] + 1);
    inv_nx = 1.0f / (float)nx;
    inv_nxy = 1.0f / (float)nxy;
  }
  // (start, count) of cell c (0 when outside the range, beyond the ball or empty)
  __device__ __forceinline__ void cell(const GridView& g, const CellFrame& f, const float q[3],
                                       float r2, int c, int& s, int& n) const {
    s = 0;
    n = 0;
    if (c >= ncell) return;
    // c = (z * ny + y) * nx + x without integer division: (c + 1/2) / m is at
    // least 1 / (2m) from an integer, above the float rounding of the product
    // for every c < 2^22 (a ball meets at most 4 x 4 x 4 cells of edge >= r / 2)
    const int z = __float2int_rz(((float)c + 0.5f) * inv_nxy), rem = c - z * nxy;
    const int y = __float2int_rz(((float)rem + 0.5f) * inv_nx), x = rem - y * nx;
    const int c3[3] = {lo[0] + x, lo[1] + y, lo[2] + z};
    if (f.range_d2(q, c3, c3) * (1.0f - 1e-6f) > r2) return;
    if (!cell_lookup(g, cell_key(f.level, 0, c3[0], c3[1], c3[2]), s, n)) n = 0;
  }
};

// Visit every point of the query's ball cells: fn(accept, d2, index) is called
// by every lane for every group of 32 candidates (accept false on lanes
// without a candidate), so warp-wide operations inside fn are safe.
template <class F>
__device__ __forceinline__ void walk_ball(const GridView& g, const float q[3], float r, int lane,
                                          int* s_start, int* s_pre, F&& fn) {
  const GridParams& P = g.prm[0];
  CellFrame f;
  f.load(P, 0);
  const float r2 = r * r;
  BallCells bc;
  bc.init(f, P, q, r);
  for (int c0 = 0; c0 < bc.ncell; c0 += 32) {
    int s, n;
    bc.cell(g, f, q, r2, c0 + lane, s, n);
    // exclusive prefix of the chunk's cell sizes
    int incl = n;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    __syncwarp();
    s_start[lane] = s;
    s_pre[lane] = incl - n;
    if (lane == 31) s_pre[32] = total;
    __syncwarp();
    // candidate t of the chunk lies in cell ci with s_pre[ci] <= t < s_pre[ci + 1];
    // each lane's t only grows, so its cell pointer (held in registers: the
    // cell's start, first and end candidate) only moves forward
    int ci = 0, cs = s_start[0], cp = 0, cn = s_pre[1];
    for (int base = 0; base < total; base += 32) {
      const int t = base + lane;
      bool acc = false;
      float d2 = 0.0f;
      int idx = -1;
      if (t < total) {
        while (t >= cn) {
          ++ci;
          cp = cn;
          cs = s_start[ci];
          cn = s_pre[ci + 1];
        }
        const float4 p = __ldg(g.pts + cs + (t - cp));
        d2 = sqdist(p.x, p.y, p.z, q[0], q[1], q[2]);
        idx = __float_as_int(p.w);
        acc = d2 <= r2;
      }
      fn(acc, d2, idx);
    }
  }
}

__global__ void __launch_bounds__(kCountWarps * 32) k_radius_count(GridView g,
                                                                   const float* __restrict__ qry,
                                                                   int64_t nq,
                                                                   const int* __restrict__ order,
                                                                   float r,
                                                                   long long* __restrict__ off,
                                                                   unsigned* __restrict__ n_long,
                                                                   int* __restrict__ long_rows) {
  __shared__ int s_start[kCountWarps][32], s_pre[kCountWarps][33];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t i = (int64_t)blockIdx.x * kCountWarps + w;
  if (i >= nq) return;  // whole warp
  const int64_t qi = order ? order[i] : i;
  const float q[3] = {qry[3 * qi], qry[3 * qi + 1], qry[3 * qi + 2]};
  long long cnt = 0;
  walk_ball(g, q, r, lane, s_start[w], s_pre[w], [&](bool acc, float, int) {
    cnt += __popc(__ballot_sync(0xffffffffu, acc));
  });
  if (lane == 0) {
    off[qi] = cnt;
    if (cnt > kRowCapW) long_rows[atomicAdd(n_long, 1u)] = (int)qi;  // at most nq rows
  }
}

// bucket of a squared distance in [0, r^2]: floor(d2 * NB / r^2) clamped to
// NB - 1 (NaN, from r = 0, also to NB - 1); monotone in d2
__device__ __forceinline__ int d2_bucket(float d2, float scale, int nb) {
  return (int)fminf(d2 * scale, (float)(nb - 1));
}

// fill: the same walk; accepted points appended to the row in visiting order
// (ballot positions: a warp's stores are consecutive words)
__global__ void __launch_bounds__(kCountWarps * 32) k_radius_fill(GridView g,
                                                                  const float* __restrict__ qry,
                                                                  int64_t nq,
                                                                  const int* __restrict__ order,
                                                                  float r,
                                                                  const long long* __restrict__ off,
                                                                  int* __restrict__ out_idx,
                                                                  float* __restrict__ out_d2) {
  __shared__ int s_start[kCountWarps][32], s_pre[kCountWarps][33];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t i = (int64_t)blockIdx.x * kCountWarps + w;
  if (i >= nq) return;  // whole warp
  const int64_t qi = order ? order[i] : i;
  const float q[3] = {qry[3 * qi], qry[3 * qi + 1], qry[3 * qi + 2]};
  const long long b = off[qi];
  const int n = (int)(off[qi + 1] - b);
  if (n == 0) return;
  int nacc = 0;
  walk_ball(g, q, r, lane, s_start[w], s_pre[w], [&](bool acc, float d2, int idx) {
    const unsigned m = __ballot_sync(0xffffffffu, acc);
    // p < n: both passes take the same decisions in the same arithmetic (the
    // test only keeps a disagreement from writing out of bounds)
    const int p = nacc + __popc(m & ((1u << lane) - 1u));
    if (acc && p < n) {
      out_idx[b + p] = idx;
      out_d2[b + p] = d2;
    }
    nacc += __popc(m);
  });
}

struct SortSmem {
  u64 key[kRowCapW];     // the row's keys in bucket order
  int cnt[kBucketsMax];  // bucket histogram, then bucket starts, then ends
};

// sort: one warp per row of 2 .. kRowCapW keys, by (d2, index), with a
// bucket sort: buckets of d2 * NB / r^2 (a monotone map, so bucket order
// agrees with key order; NB a power of two >= n / 2), a histogram of the row
// as filled, its scan, a scatter of the keys into bucket order in shared
// memory, an insertion sort of each bucket by the lane that owns it (buckets
// hold ~2 keys), and one coalesced write of the sorted row over the filled one
__global__ void __launch_bounds__(kSortWarps * 32) k_sort_rows_warp(const long long* __restrict__ off,
                                                                    int64_t nq, float r,
                                                                    int* __restrict__ idx,
                                                                    float* __restrict__ d2) {
  __shared__ SortSmem smem[kSortWarps];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  SortSmem& S = smem[w];
  const int64_t row = (int64_t)blockIdx.x * kSortWarps + w;
  if (row >= nq) return;  // whole warp
  const long long b = off[row];
  const int n = (int)(off[row + 1] - b);
  if (n <= 1 || n > kRowCapW) return;  // nothing to sort, or a listed long row
  int nb = 32;
  while (nb < kBucketsMax && 2 * nb < n) nb <<= 1;
  const float r2 = r * r;
  const float scale = (float)nb / r2;
  for (int j = lane; j < nb; j += 32) S.cnt[j] = 0;
  __syncwarp();
  for (int j = lane; j < n; j += 32) atomicAdd(&S.cnt[d2_bucket(d2[b + j], scale, nb)], 1);
  __syncwarp();
  // exclusive scan of the histogram, 32 buckets at a time (conflict free)
  int carry = 0;
  for (int c0 = 0; c0 < nb; c0 += 32) {
    const int v = S.cnt[c0 + lane];
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    S.cnt[c0 + lane] = carry + incl - v;
    carry += __shfl_sync(0xffffffffu, incl, 31);
  }
  __syncwarp();
  // keys into bucket order (S.cnt[k] ends as the end of bucket k)
  for (int j = lane; j < n; j += 32) {
    const float dd = d2[b + j];
    S.key[atomicAdd(&S.cnt[d2_bucket(dd, scale, nb)], 1)] = pack_key(dd, idx[b + j]);
  }
  __syncwarp();
  // each lane sorts its buckets in place (bucket k spans [end(k-1), end(k)))
  for (int k = lane; k < nb; k += 32) {
    const int beg = k ? S.cnt[k - 1] : 0, end = S.cnt[k];
    for (int i = beg + 1; i < end; ++i) {
      const u64 x = S.key[i];
      int j = i - 1;
      while (j >= beg && S.key[j] > x) {
        S.key[j + 1] = S.key[j];
        --j;
      }
      S.key[j + 1] = x;
    }
  }
  __syncwarp();
  for (int j = lane; j < n; j += 32) {
    const u64 key = S.key[j];
    idx[b + j] = key_idx(key);
    d2[b + j] = key_d2(key);
  }
}

__device__ __forceinline__ void cmp_swap_keys(u64& a, u64& b) {
  if (b < a) {
    const u64 t = a;
    a = b;
    b = t;
  }
}

// all-ascending bitonic sort of the listed rows, one block each: for each
// size, a "flip" compare (i, i^(size-1)) then half-cleaners (i, i+stride); the
// smaller key always goes to the lower index, so entries past n behave as
// +inf and are never touched
__global__ void __launch_bounds__(kSortThreads) k_sort_rows(const long long* __restrict__ off,
                                                            const int* __restrict__ rows,
                                                            int* __restrict__ idx,
                                                            float* __restrict__ d2) {
  __shared__ u64 sk[kRowCap];
  const int64_t row = rows[blockIdx.x];
  const long long b = off[row];
  const int n = (int)(off[row + 1] - b);
  if (n <= 1) return;
  int np = 1, lg = 0;
  while (np < n) {
    np <<= 1;
    ++lg;
  }
  if (n <= kRowCap) {
    for (int i = threadIdx.x; i < n; i += kSortThreads) sk[i] = pack_key(d2[b + i], idx[b + i]);
    __syncthreads();
    // sizes are powers of two: block and offset by shift and mask
    for (int ls = 1; ls <= lg; ++ls) {
      const int size = 1 << ls, half = size >> 1;
      for (int t = threadIdx.x; t < np / 2; t += kSortThreads) {
        const int blk = t >> (ls - 1), o = t & (half - 1);
        const int i = (blk << ls) + o, j = (blk << ls) + size - 1 - o;
        if (j < n) cmp_swap_keys(sk[i], sk[j]);
      }
      __syncthreads();
      for (int stride = size / 4; stride > 0; stride >>= 1) {
        for (int t = threadIdx.x; t < np / 2; t += kSortThreads) {
          const int i = 2 * t - (t & (stride - 1));
          const int j = i + stride;
          if (j < n) cmp_swap_keys(sk[i], sk[j]);
        }
        __syncthreads();
      }
    }
    for (int i = threadIdx.x; i < n; i += kSortThreads) {
      d2[b + i] = key_d2(sk[i]);
      idx[b + i] = key_idx(sk[i]);
    }
  } else {
    for (int ls = 1; ls <= lg; ++ls) {
      const int size = 1 << ls;
      for (int stride = size / 2; stride > 0; stride >>= 1) {
        for (int t = threadIdx.x; t < np / 2; t += kSortThreads) {
          int i, j;
          if (stride == size / 2) {
            const int blk = t >> (ls - 1), o = t & (stride - 1);
            i = (blk << ls) + o;
            j = (blk << ls) + size - 1 - o;
          } else {
            i = 2 * t - (t & (stride - 1));
            j = i + stride;
          }
          if (j < n) {
            u64 ka = pack_key(d2[b + i], idx[b + i]);
            u64 kb = pack_key(d2[b + j], idx[b + j]);
            if (kb < ka) {
              d2[b + i] = key_d2(kb);
              idx[b + i] = key_idx(kb);
              d2[b + j] = key_d2(ka);
              idx[b + j] = key_idx(ka);
            }
          }
        }
        __threadfence_block();
        __syncthreads();
      }
    }
  }
}

}  // namespace cil

using namespace cil;

static cil_status radius_impl(const float* ref, int64_t n_ref, const float* qry, int64_t n_qry,
                              float r, int64_t* out_offsets, int32_t* out_idx, float* out_d2,
                              int64_t capacity, int64_t* out_nnz, float cell_edge, void* stream) {
  if (n_ref < 0 || n_qry < 0 || n_ref > 0x7fffffff || n_qry > 0x7fffffff || !(r >= 0.0f) ||
      !isfinite(r) || capacity < 0 || !out_nnz || !(cell_edge >= 0.0f) || !isfinite(cell_edge))
    return CIL_ERR_INVALID_ARG;
  if (n_qry > 0 && (!qry || !out_offsets)) return CIL_ERR_INVALID_ARG;
  if (n_ref > 0 && !ref) return CIL_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  *out_nnz = 0;
  if (n_qry == 0) {
    if (out_offsets &&
        cudaMemsetAsync(out_offsets, 0, sizeof(int64_t), s) != cudaSuccess)
      return CIL_ERR_CUDA;
    return cudaStreamSynchronize(s) == cudaSuccess ? CIL_OK : CIL_ERR_CUDA;
  }
  cil_status st = CIL_OK;
  DeviceCtx* ctx = device_ctx(&st);
  if (!ctx) return st;
  Workspace ws;
  GridPlan gp;
  grid_plan(gp, ws, n_ref, 1);
  OrderPlan op;
  order_plan(op, ws, n_qry);
  const size_t o_order = ws.reserve(sizeof(int) * (size_t)n_qry);
  const size_t o_tmp = ws.reserve(sizeof(long long) * (scan_tmp_ints(n_qry + 1) * 2 + 2));
  const size_t o_long = ws.reserve(sizeof(unsigned) * 2);
  const size_t o_long_rows = ws.reserve(sizeof(int) * (size_t)n_qry);  // rows over kRowCapW
  if ((st = ws.allocate(ctx, s)) != CIL_OK) return st;
  GridOptions opt;
  opt.k_est = 10;
  opt.cell_size = cell_edge;
  if ((st = grid_build(gp, ws, ref, nullptr, opt, ctx, s)) != CIL_OK) return st;
  const GridView g = grid_view(gp, ws);
  int* order = ws.at<int>(o_order);
  if ((st = order_queries(op, ws, qry, nullptr, 1, g.prm, nullptr, order, s)) != CIL_OK) return st;
  long long* off = reinterpret_cast<long long*>(out_offsets);
  unsigned* n_long = ws.at<unsigned>(o_long);  // rows longer than kRowCapW
  int* long_rows = ws.at<int>(o_long_rows);     // and their indices
  if (cudaMemsetAsync(n_long, 0, sizeof(unsigned), s) != cudaSuccess) return CIL_ERR_CUDA;
  {
    TimedRegion timer("k_radius", s);
    note_launches(1);
    k_radius_count<<<ceil_div(n_qry, kCountWarps), kCountWarps * 32, 0, s>>>(g, qry, n_qry, order, r,
                                                                            off, n_long, long_rows);
  }
  if (cudaMemsetAsync(off + n_qry, 0, sizeof(long long), s) != cudaSuccess) return CIL_ERR_CUDA;
  scan_exclusive_i64(off, n_qry + 1, ws.at<long long>(o_tmp), s);
  struct {
    long long nnz;
    unsigned n_long;
  } h = {0, 0};
  if (cudaMemcpyAsync(&h.nnz, off + n_qry, sizeof(long long), cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaMemcpyAsync(&h.n_long, n_long, sizeof(unsigned), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return CIL_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return CIL_ERR_CUDA;
  *out_nnz = h.nnz;
  if (h.nnz > capacity) {
    ws.release(s);
    cudaStreamSynchronize(s);
    return CIL_ERR_CAPACITY;
  }
  if (h.nnz > 0) {
    if (!out_idx) return CIL_ERR_INVALID_ARG;
    float* d2 = out_d2;
    void* tmp = nullptr;
    if (!d2) {
      if (cudaMallocFromPoolAsync(&tmp, sizeof(float) * (size_t)h.nnz, ctx->pool, s) != cudaSuccess)
        return CIL_ERR_NOMEM;
      d2 = static_cast<float*>(tmp);
    }
    TimedRegion timer("k_radius", s);
    note_launches(h.n_long > 0 ? 3 : 2);
    k_radius_fill<<<ceil_div(n_qry, kCountWarps), kCountWarps * 32, 0, s>>>(g, qry, n_qry, order, r,
                                                                           off, out_idx, d2);
    k_sort_rows_warp<<<ceil_div(n_qry, kSortWarps), kSortWarps * 32, 0, s>>>(off, n_qry, r,
                                                                            out_idx, d2);
    if (h.n_long > 0) k_sort_rows<<<h.n_long, kSortThreads, 0, s>>>(off, long_rows, out_idx, d2);
    if (tmp) cudaFreeAsync(tmp, s);
  }
  ws.release(s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return CIL_ERR_CUDA;
  if (cudaGetLastError() != cudaSuccess) return CIL_ERR_CUDA;
  int v = 0;
  cudaMemcpy(&v, ctx->err, sizeof(int), cudaMemcpyDeviceToHost);
  if (v) {
    cudaMemset(ctx->err, 0, sizeof(int));
    return (cil_status)v;
  }
  return CIL_OK;
}

// The ball's cells: edge r by default (at most 4 x 4 x 4 cells per query);
// params->cell_size (> 0) sets the edge, else params->cell_scale (> 0)
// multiplies r.  The edge is rounded to a power-of-two multiple of the fine
// lattice; it changes the time, not the result.
extern "C" cil_status cil_radius_search_ex(const float* ref, int64_t n_ref, const float* qry,
                                           int64_t n_qry, float r, int64_t* out_offsets,
                                           int32_t* out_idx, float* out_d2, int64_t capacity,
                                           int64_t* out_nnz, const cil_params* params,
                                           void* stream) {
  float edge = r > 0.0f ? r : 0.0f;
  if (params && params->cell_size > 0.0f) edge = params->cell_size;
  else if (params && params->cell_scale > 0.0f && r > 0.0f) edge = r * params->cell_scale;
  return radius_impl(ref, n_ref, qry, n_qry, r, out_offsets, out_idx, out_d2, capacity, out_nnz,
                     edge, stream);
}

extern "C" cil_status cil_radius_search(const float* ref, int64_t n_ref, const float* qry,
                                        int64_t n_qry, float r, int64_t* out_offsets,
                                        int32_t* out_idx, float* out_d2, int64_t capacity,
                                        int64_t* out_nnz, void* stream) {
  return cil_radius_search_ex(ref, n_ref, qry, n_qry, r, out_offsets, out_idx, out_d2, capacity,
                              out_nnz, nullptr, stream);
}
