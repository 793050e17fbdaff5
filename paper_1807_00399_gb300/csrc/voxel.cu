// voxel.cu -- voxel-grid downsampling (Sec. 3 GridAccumulator; Sec. 4
// downsamples to 1 cm voxels before ICP).
//
// Point i falls in voxel (floor(x/v), floor(y/v), floor(z/v)) with correctly
// rounded FP32 division (clamped to 21 bits per axis).  A first pass finds the
// occupied range of each voxel coordinate; the key packs the coordinates'
// offsets from the range's low corner in just the bits their spans need
// (x highest), so it orders voxels by (ix, iy, iz) and the stable radix sort
// with the point index takes only ceil(bits / 10) passes (3 for a 1 cm grid
// of a depth frame instead of 7 for the full 63 bits).  Voxel heads are
// marked and scanned into output slots, and each voxel's mean is accumulated
// over its run in index order with compensated FP32 sums (deterministic).
// Output voxels ascend by (ix, iy, iz).
#include <math.h>

#include <algorithm>

#include "cil_host.h"
#include "cil_kernels.h"

namespace cil {

constexpr int kVoxBias = 1 << 20;

// voxel coordinate of x, biased into [0, 2^21)
__device__ __forceinline__ int voxel_coord(float x, float v) {
  float f = floorf(__fdiv_rn(x, v));
  f = fminf(fmaxf(f, -(float)kVoxBias), (float)(kVoxBias - 1));  // NaN -> lower bound
  return (int)f + kVoxBias;
}

// Occupied range of the biased coordinates: ext[a] = max (2^21 - 1 - c_a)
// (the low corner, kept as a maximum) and ext[3 + a] = max c_a; ext starts
// zeroed, every value is in [0, 2^21).
__global__ void __launch_bounds__(256) k_voxel_range(const float* __restrict__ xyz, int64_t n,
                                                     float v, int* __restrict__ ext) {
  int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int c = voxel_coord(xyz[3 * i + a], v);
      lo[a] = max(lo[a], (2 * kVoxBias - 1) - c);
      hi[a] = max(hi[a], c);
    }
  }
  // warp, then block maxima; one atomic per value and block
  __shared__ int s_m[6][8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    lo[a] = (int)__reduce_max_sync(0xffffffffu, (unsigned)lo[a]);
    hi[a] = (int)__reduce_max_sync(0xffffffffu, (unsigned)hi[a]);
    if (lane == 0) {
      s_m[a][warp] = lo[a];
      s_m[3 + a][warp] = hi[a];
    }
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    int m = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = max(m, s_m[threadIdx.x][w]);
    atomicMax(ext + threadIdx.x, m);
  }
}

// key = (cx - lo_x) << (by + bz) | (cy - lo_y) << bz | (cz - lo_z)
__global__ void k_voxel_keys(const float* __restrict__ xyz, int64_t n, float v, int lx, int ly,
                             int lz, int by, int bz, u64* __restrict__ keys, int* __restrict__ vals) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const u64 cx = (u64)(voxel_coord(xyz[3 * i], v) - lx);
  const u64 cy = (u64)(voxel_coord(xyz[3 * i + 1], v) - ly);
  const u64 cz = (u64)(voxel_coord(xyz[3 * i + 2], v) - lz);
  keys[i] = (cx << (by + bz)) | (cy << bz) | cz;
  vals[i] = (int)i;
}

// bits that hold 0 .. span - 1
static int span_bits(int span) {
  int b = 0;
  while ((1 << b) < span) ++b;
  return b;
}

__global__ void k_voxel_heads(const u64* __restrict__ keys, int64_t n, int* __restrict__ head) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i > n) return;
  if (i == n) {
    head[n] = 0;
    return;
  }
  head[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1 : 0;
}

// one thread per voxel run: compensated mean in sorted (= index) order
__global__ void k_voxel_reduce(const u64* __restrict__ keys, const int* __restrict__ vals,
                               const int* __restrict__ slot, int64_t n, const float* __restrict__ xyz,
                               float* __restrict__ out_xyz, int* __restrict__ out_counts) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (i > 0 && keys[i] == keys[i - 1]) return;  // not a run head
  KSum s[3];
  s[0].zero();
  s[1].zero();
  s[2].zero();
  int64_t j = i;
  const u64 key = keys[i];
  for (; j < n && keys[j] == key; ++j) {
    const int64_t p = vals[j];
    s[0].add(xyz[3 * p]);
    s[1].add(xyz[3 * p + 1]);
    s[2].add(xyz[3 * p + 2]);
  }
  const int m = (int)(j - i);
  const int o = slot[i];
  const double inv = 1.0 / (double)m;
  for (int a = 0; a < 3; ++a) out_xyz[3 * (int64_t)o + a] = (float)(((double)s[a].s + (double)s[a].c) * inv);
  if (out_counts) out_counts[o] = m;
}

}  // namespace cil

using namespace cil;

extern "C" cil_status cil_voxel_downsample(const float* xyz, int64_t n, float voxel, float* out_xyz,
                                           int32_t* out_counts, int64_t* out_n, void* stream) {
  if (n < 0 || n > 0x7fffffff || !(voxel > 0.0f) || !isfinite(voxel) || !out_n)
    return CIL_ERR_INVALID_ARG;
  *out_n = 0;
  if (n == 0) return CIL_OK;
  if (!xyz || !out_xyz) return CIL_ERR_INVALID_ARG;
  cil_status st = CIL_OK;
  DeviceCtx* ctx = device_ctx(&st);
  if (!ctx) return st;
  cudaStream_t s = (cudaStream_t)stream;
  Workspace ws;
  RadixPlan rp;
  radix_sort_plan(rp, ws, n);
  const size_t o_head = ws.reserve(sizeof(int) * (size_t)(n + 1));
  const size_t o_tmp = ws.reserve(sizeof(int) * scan_tmp_ints(n + 1));
  const size_t o_ext = ws.reserve(sizeof(int) * 6);
  if ((st = ws.allocate(ctx, s)) != CIL_OK) return st;
  TimedRegion timer("voxel_downsample", s);
  note_launches(4);
  int* ext = ws.at<int>(o_ext);
  if (cudaMemsetAsync(ext, 0, sizeof(int) * 6, s) != cudaSuccess) return CIL_ERR_CUDA;
  const int rblocks = std::max(1, std::min(ceil_div(n, 256), 2 * ctx->num_sms));
  k_voxel_range<<<rblocks, 256, 0, s>>>(xyz, n, voxel, ext);
  int e[6];
  if (cudaMemcpyAsync(e, ext, sizeof(e), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return CIL_ERR_CUDA;
  int lo[3], bits[3];
  for (int a = 0; a < 3; ++a) {
    lo[a] = (2 * kVoxBias - 1) - e[a];
    bits[a] = span_bits(e[3 + a] - lo[a] + 1);
  }
  k_voxel_keys<<<ceil_div(n, 256), 256, 0, s>>>(xyz, n, voxel, lo[0], lo[1], lo[2], bits[1],
                                                 bits[2], ws.at<u64>(rp.o_keys0),
                                                 ws.at<int>(rp.o_vals0));
  const int which = radix_sort_pairs(rp, ws, bits[0] + bits[1] + bits[2], s);
  const u64* keys = ws.at<u64>(which ? rp.o_keys1 : rp.o_keys0);
  const int* vals = ws.at<int>(which ? rp.o_vals1 : rp.o_vals0);
  int* head = ws.at<int>(o_head);
  k_voxel_heads<<<ceil_div(n + 1, 256), 256, 0, s>>>(keys, n, head);
  scan_exclusive(head, n + 1, ws.at<int>(o_tmp), s);
  int m = 0;
  if (cudaMemcpyAsync(&m, head + n, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return CIL_ERR_CUDA;
  k_voxel_reduce<<<ceil_div(n, 256), 256, 0, s>>>(keys, vals, head, n, xyz, out_xyz, out_counts);
  ws.release(s);
  if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess)
    return CIL_ERR_CUDA;
  *out_n = m;
  return CIL_OK;
}
