// radius.cu -- fixed-radius neighbour search (Sec. 3, KDTree radius query).
//
// Grid cells are sized to the radius (nearest power-of-two multiple of the
// fine lattice), so each query visits the few cells its ball touches.
//   pass 1: count neighbours with d2 <= r*r per query (one thread per query);
//   scan:   int64 CSR offsets;
//   pass 2: write (index, d2) of each row in visiting order;
//   sort:   each row by (d2, index) -- rows up to kRowCap keys in shared
//           memory, longer rows in place in global memory; both with the
//           same all-ascending bitonic network, where virtual +inf padding
//           past the row end never moves.
#include <math.h>

#include "cil_host.h"
#include "cil_kernels.h"

namespace cil {

constexpr int kRowCap = 4096;
constexpr int kSortThreads = 256;

template <bool kFill>
__global__ void __launch_bounds__(128) k_radius(GridView g, const float* __restrict__ qry, int64_t nq,
                                                const int* __restrict__ order, float r,
                                                long long* __restrict__ off, int* __restrict__ out_idx,
                                                float* __restrict__ out_d2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nq) return;
  const int64_t qi = order ? order[i] : i;
  const float q[3] = {qry[3 * qi], qry[3 * qi + 1], qry[3 * qi + 2]};
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
  long long cnt = 0;
  long long w = kFill ? off[qi] : 0;
  for (int z = lo[2]; z <= hi[2]; ++z)
    for (int y = lo[1]; y <= hi[1]; ++y)
      for (int x = lo[0]; x <= hi[0]; ++x) {
        const int c3[3] = {x, y, z};
        if (f.range_d2(q, c3, c3) * (1.0f - 1e-6f) > r2) continue;
        int s, n;
        if (!cell_lookup(g, cell_key(P.level, 0, x, y, z), s, n)) continue;
        for_points(g.pts, s, n, [&](const float4& p, int) {
          const float d2 = sqdist(p.x, p.y, p.z, q[0], q[1], q[2]);
          if (d2 <= r2) {
            if (kFill) {
              out_idx[w] = __float_as_int(p.w);
              out_d2[w] = d2;
              ++w;
            } else {
              ++cnt;
            }
          }
        });
      }
  if (!kFill) off[qi] = cnt;
}

__device__ __forceinline__ void cmp_swap_keys(u64& a, u64& b) {
  if (b < a) {
    const u64 t = a;
    a = b;
    b = t;
  }
}

// all-ascending bitonic sort: for each size, a "flip" compare (i, i^(size-1))
// then half-cleaners (i, i+stride); the smaller key always goes to the lower
// index, so entries past n behave as +inf and are never touched
__global__ void __launch_bounds__(kSortThreads) k_sort_rows(const long long* __restrict__ off,
                                                            int64_t nq, int* __restrict__ idx,
                                                            float* __restrict__ d2) {
  __shared__ u64 sk[kRowCap];
  const int64_t row = blockIdx.x;
  if (row >= nq) return;
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

extern "C" cil_status cil_radius_search(const float* ref, int64_t n_ref, const float* qry,
                                        int64_t n_qry, float r, int64_t* out_offsets,
                                        int32_t* out_idx, float* out_d2, int64_t capacity,
                                        int64_t* out_nnz, void* stream) {
  if (n_ref < 0 || n_qry < 0 || n_ref > 0x7fffffff || n_qry > 0x7fffffff || !(r >= 0.0f) ||
      !isfinite(r) || capacity < 0 || !out_nnz)
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
  if ((st = ws.allocate(ctx, s)) != CIL_OK) return st;
  GridOptions opt;
  opt.k_est = 10;
  opt.cell_size = r > 0.0f ? r : 0.0f;
  if ((st = grid_build(gp, ws, ref, nullptr, opt, ctx, s)) != CIL_OK) return st;
  const GridView g = grid_view(gp, ws);
  int* order = ws.at<int>(o_order);
  if ((st = order_queries(op, ws, qry, nullptr, 1, g.prm, nullptr, order, s)) != CIL_OK) return st;
  long long* off = reinterpret_cast<long long*>(out_offsets);
  const int grid = ceil_div(n_qry, 128);
  {
    TimedRegion timer("k_radius", s);
    note_launches(1);
    k_radius<false><<<grid, 128, 0, s>>>(g, qry, n_qry, order, r, off, nullptr, nullptr);
  }
  if (cudaMemsetAsync(off + n_qry, 0, sizeof(long long), s) != cudaSuccess) return CIL_ERR_CUDA;
  scan_exclusive_i64(off, n_qry + 1, ws.at<long long>(o_tmp), s);
  long long nnz = 0;
  if (cudaMemcpyAsync(&nnz, off + n_qry, sizeof(long long), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return CIL_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return CIL_ERR_CUDA;
  *out_nnz = nnz;
  if (nnz > capacity) {
    ws.release(s);
    cudaStreamSynchronize(s);
    return CIL_ERR_CAPACITY;
  }
  if (nnz > 0) {
    if (!out_idx) return CIL_ERR_INVALID_ARG;
    float* d2 = out_d2;
    void* d2_tmp = nullptr;
    if (!d2) {
      if (cudaMallocFromPoolAsync(&d2_tmp, sizeof(float) * (size_t)nnz, ctx->pool, s) != cudaSuccess)
        return CIL_ERR_NOMEM;
      d2 = static_cast<float*>(d2_tmp);
    }
    TimedRegion timer("k_radius", s);
    note_launches(2);
    k_radius<true><<<grid, 128, 0, s>>>(g, qry, n_qry, order, r, off, out_idx, d2);
    k_sort_rows<<<(unsigned)n_qry, kSortThreads, 0, s>>>(off, n_qry, out_idx, d2);
    if (d2_tmp) cudaFreeAsync(d2_tmp, s);
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
