// grid.cu -- uniform-grid spatial index over one or many clouds.
//
// Build steps (all on the caller's stream, no host synchronisation):
//   1. per-cloud bounding box (order-independent integer min/max atomics, so
//      the result is deterministic) and count of non-finite coordinates;
//   2. fine lattice: cubic cells of edge max_extent / 1023 over the box;
//   3. key = (cloud << 30) | Morton(fine cell), stable LSD radix sort of
//      (key, index) with 10-bit digits;
//   4. gather the sorted points as float4 (x, y, z, index within its cloud);
//   5. choose the search level per cloud (cell = fine * 2^level) from the
//      k-th neighbour distance among Morton neighbours of sampled points;
//   6. hash table (cloud, cell) -> (first sorted position, point count).
// The sort is stable and keyed only by the input, so the sorted order -- and
// every result built on it -- is identical from run to run.
#include <math.h>

#include "cil_host.h"

namespace cil {

constexpr int kRadixBits = 10;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kRsThreads = 256;
constexpr int kRsItems = 8;
constexpr int kRsTile = kRsThreads * kRsItems;
constexpr int kRsWarps = kRsThreads / 32;
constexpr int kScanThreads = 1024;

int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

unsigned next_pow2_u32(uint64_t v) {
  uint64_t p = 1;
  while (p < v) p <<= 1;
  return (unsigned)p;
}

__device__ __forceinline__ int cloud_of(const int* cs, int clouds, int64_t i) {
  if (clouds <= 1 || cs == nullptr) return 0;
  int lo = 0, hi = clouds;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if ((int64_t)cs[mid] <= i) lo = mid;
    else hi = mid;
  }
  return lo;
}

// ---------------------------------------------------------------------------
// 1-2. parameters and bounding box
// ---------------------------------------------------------------------------
__global__ void k_init_params(GridParams* prm, int clouds, const int* cs, int64_t n_total) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= clouds) return;
  GridParams P;
  P.start = cs ? cs[b] : 0;
  P.n = (cs ? cs[b + 1] : (int)n_total) - P.start;
  for (int a = 0; a < 3; ++a) {
    P.o[a] = 0.0f;
    P.bmax[a] = 0.0f;
    P.hi_fine[a] = 0;
    P.bbox_enc[a] = 0xffffffffu;  // running minimum
    P.bbox_enc[3 + a] = 0u;       // running maximum
  }
  P.fine = 1.0f;
  P.inv_fine = 1.0f;
  P.eps = 0.0f;
  P.level = 0;
  P.cell = 1.0f;
  P.nonfinite = 0;
  P.pad[0] = P.pad[1] = P.pad[2] = 0;
  prm[b] = P;
}

__global__ void k_bbox(const float* __restrict__ xyz, int64_t n, const int* cs, int clouds,
                       GridParams* prm) {
  constexpr int CH = 8;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t i0 = t * CH, i1 = min(i0 + CH, n);
  int cur = -1, nf = 0;
  float mn[3], mx[3];
  auto reset = [&]() {
    for (int a = 0; a < 3; ++a) {
      mn[a] = __int_as_float(0x7f800000);
      mx[a] = -__int_as_float(0x7f800000);
    }
  };
  auto flush = [&](int c) {
    if (c < 0) return;
    for (int a = 0; a < 3; ++a) {
      if (mn[a] <= mx[a]) {
        atomicMin(&prm[c].bbox_enc[a], float_to_ordered(mn[a]));
        atomicMax(&prm[c].bbox_enc[3 + a], float_to_ordered(mx[a]));
      }
    }
  };
  reset();
  for (int64_t i = i0; i < i1; ++i) {
    const int c = cloud_of(cs, clouds, i);
    if (c != cur) {
      flush(cur);
      if (cur >= 0 && nf) {
        atomicAdd(&prm[cur].nonfinite, nf);
        nf = 0;
      }
      cur = c;
      reset();
    }
    const float x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
    if (!(isfinite(x) && isfinite(y) && isfinite(z))) {
      ++nf;
      continue;
    }
    mn[0] = fminf(mn[0], x);
    mn[1] = fminf(mn[1], y);
    mn[2] = fminf(mn[2], z);
    mx[0] = fmaxf(mx[0], x);
    mx[1] = fmaxf(mx[1], y);
    mx[2] = fmaxf(mx[2], z);
  }
  if (cur >= 0 && nf) atomicAdd(&prm[cur].nonfinite, nf);
  // warp-combine when the whole warp ends in the same cloud
  const unsigned full = 0xffffffffu;
  const int c0 = __shfl_sync(full, cur, 0);
  const bool uniform = __all_sync(full, cur == c0 || cur < 0) && c0 >= 0;
  if (uniform) {
    for (int a = 0; a < 3; ++a) {
      for (int off = 16; off > 0; off >>= 1) {
        mn[a] = fminf(mn[a], __shfl_xor_sync(full, mn[a], off));
        mx[a] = fmaxf(mx[a], __shfl_xor_sync(full, mx[a], off));
      }
    }
    if ((threadIdx.x & 31) == 0) flush(c0);
  } else {
    flush(cur);
  }
}

__global__ void k_finalize(GridParams* prm, int clouds, int* err) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= clouds) return;
  GridParams& P = prm[b];
  if (P.nonfinite) atomicCAS(err, 0, (int)CIL_ERR_NONFINITE);
  float mn[3], mx[3];
  bool any = true;
  for (int a = 0; a < 3; ++a) {
    if (P.bbox_enc[a] == 0xffffffffu) any = false;
    mn[a] = ordered_to_float(P.bbox_enc[a]);
    mx[a] = ordered_to_float(P.bbox_enc[3 + a]);
  }
  if (!any) {  // empty cloud (or nothing finite)
    for (int a = 0; a < 3; ++a) {
      mn[a] = 0.0f;
      mx[a] = 0.0f;
    }
  }
  float ext = 0.0f, amax = 0.0f;
  for (int a = 0; a < 3; ++a) {
    ext = fmaxf(ext, mx[a] - mn[a]);
    amax = fmaxf(amax, fabsf(mn[a]));
    amax = fmaxf(amax, fabsf(mx[a]));
  }
  float fine = ext > 0.0f ? ext / (float)(kFineDim - 1) : 1.0f;
  fine = fmaxf(fine, 1e-30f);
  const float inv = 1.0f / fine;
  for (int a = 0; a < 3; ++a) {
    P.o[a] = mn[a];
    P.bmax[a] = mx[a];
  }
  P.fine = fine;
  P.inv_fine = inv;
  for (int a = 0; a < 3; ++a) P.hi_fine[a] = fine_coord(mx[a], mn[a], inv);
  P.eps = 1e-6f * (amax + (float)kFineDim * fine) + 1e-30f;
  P.level = 0;
  P.cell = fine;
}

// ---------------------------------------------------------------------------
// 3. Morton keys and the stable radix sort
// ---------------------------------------------------------------------------
__global__ void k_morton_keys(const float* __restrict__ xyz, int64_t n, const int* cs, int clouds,
                              const GridParams* __restrict__ prm, const float* __restrict__ Rt,
                              u64* __restrict__ keys, int* __restrict__ vals) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int c = cloud_of(cs, clouds, i);
  const GridParams& P = prm[c];
  float x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
  if (Rt) {
    const float* m = Rt + 12 * c;
    const float tx = fmaf(m[0], x, fmaf(m[1], y, fmaf(m[2], z, m[3])));
    const float ty = fmaf(m[4], x, fmaf(m[5], y, fmaf(m[6], z, m[7])));
    const float tz = fmaf(m[8], x, fmaf(m[9], y, fmaf(m[10], z, m[11])));
    x = tx;
    y = ty;
    z = tz;
  }
  const unsigned fx = fine_coord(x, P.o[0], P.inv_fine);
  const unsigned fy = fine_coord(y, P.o[1], P.inv_fine);
  const unsigned fz = fine_coord(z, P.o[2], P.inv_fine);
  keys[i] = ((u64)(unsigned)c << 30) | (u64)morton3(fx, fy, fz);
  vals[i] = (int)i;
}

__global__ void __launch_bounds__(kRsThreads) k_radix_hist(const u64* __restrict__ keys, int64_t n,
                                                           int shift, int* __restrict__ counts,
                                                           int nblk) {
  __shared__ int h[kRadix];
  for (int d = threadIdx.x; d < kRadix; d += kRsThreads) h[d] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kRsTile;
#pragma unroll
  for (int j = 0; j < kRsItems; ++j) {
    const int64_t i = base + j * kRsThreads + threadIdx.x;
    if (i < n) atomicAdd(&h[(int)((keys[i] >> shift) & (kRadix - 1))], 1);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < kRadix; d += kRsThreads) counts[(int64_t)d * nblk + blockIdx.x] = h[d];
}

// Per-digit prefix over the blocks: one warp per digit scans its nblk block
// counts (digit-major, contiguous) into exclusive prefixes in place and
// writes the digit's total; the scatter adds the digits' exclusive bases.
constexpr int kDigitWarps = 8;
__global__ void __launch_bounds__(kDigitWarps * 32) k_radix_digit_scan(int* __restrict__ counts,
                                                                       int nblk,
                                                                       int* __restrict__ totals) {
  const int lane = threadIdx.x & 31;
  const int d = blockIdx.x * kDigitWarps + (threadIdx.x >> 5);
  int* c = counts + (int64_t)d * nblk;
  int carry = 0;
  for (int b0 = 0; b0 < nblk; b0 += 32) {
    const int b = b0 + lane;
    const int v = b < nblk ? c[b] : 0;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (b < nblk) c[b] = carry + incl - v;
    carry += __shfl_sync(0xffffffffu, incl, 31);
  }
  if (lane == 0) totals[d] = carry;
}

// Stable scatter: each warp ranks its 256 items (index order = item j major,
// lane minor) with match_any; warps are then offset by an exclusive scan of
// the per-warp digit counts seeded with the block's global digit offsets.
__global__ void __launch_bounds__(kRsThreads) k_radix_scatter(
    const u64* __restrict__ kin, const int* __restrict__ vin, int64_t n, int shift,
    const int* __restrict__ offs, const int* __restrict__ totals, int nblk,
    u64* __restrict__ kout, int* __restrict__ vout) {
  __shared__ int wh[kRsWarps][kRadix];
  __shared__ int dbase[kRadix];  // exclusive scan of the digit totals
  __shared__ int wsum[kRsWarps];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int e = threadIdx.x; e < kRsWarps * kRadix; e += kRsThreads) (&wh[0][0])[e] = 0;
  {  // thread t owns digits [t * per, (t + 1) * per)
    constexpr int per = kRadix / kRsThreads;
    int v[per], sum = 0;
#pragma unroll
    for (int j = 0; j < per; ++j) {
      v[j] = totals[threadIdx.x * per + j];
      sum += v[j];
    }
    int incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    int run = incl - sum;
    for (int w = 0; w < warp; ++w) run += wsum[w];
#pragma unroll
    for (int j = 0; j < per; ++j) {
      dbase[threadIdx.x * per + j] = run;
      run += v[j];
    }
  }
  __syncthreads();
  const unsigned lt = (1u << lane) - 1u;
  const int64_t base = (int64_t)blockIdx.x * kRsTile + warp * (kRsTile / kRsWarps);
  u64 key[kRsItems];
  int val[kRsItems], dig[kRsItems], rnk[kRsItems];
#pragma unroll
  for (int j = 0; j < kRsItems; ++j) {
    const int64_t i = base + j * 32 + lane;
    const bool valid = i < n;
    const unsigned vmask = __ballot_sync(0xffffffffu, valid);
    int d = -1, r = 0;
    unsigned peers = 0;
    if (valid) {
      key[j] = kin[i];
      val[j] = vin[i];
      d = (int)((key[j] >> shift) & (kRadix - 1));
      peers = __match_any_sync(vmask, d);
      r = wh[warp][d] + __popc(peers & lt);
    }
    __syncwarp();
    if (valid && lane == __ffs(peers) - 1) wh[warp][d] += __popc(peers);
    __syncwarp();
    dig[j] = d;
    rnk[j] = r;
  }
  __syncthreads();
  for (int d = threadIdx.x; d < kRadix; d += kRsThreads) {
    int acc = dbase[d] + offs[(int64_t)d * nblk + blockIdx.x];
    for (int w = 0; w < kRsWarps; ++w) {
      const int t = wh[w][d];
      wh[w][d] = acc;
      acc += t;
    }
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < kRsItems; ++j) {
    if (dig[j] >= 0) {
      const int pos = wh[warp][dig[j]] + rnk[j];
      kout[pos] = key[j];
      vout[pos] = val[j];
    }
  }
}

// ---------------------------------------------------------------------------
// exclusive scan of an int array (reduce, scan partials, apply)
// ---------------------------------------------------------------------------
// int: 8 items per thread; 64-bit: 4 (keeps the chunk buffer within 48 KB)
template <typename T>
struct ScanCfg {
  static constexpr int items = sizeof(T) == 4 ? 8 : 4;
  static constexpr int chunk = kScanThreads * items;
};

template <typename T>
__device__ __forceinline__ T block_exclusive_scan(T v, T* warp_sums, T* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T x = v;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const T y = __shfl_up_sync(0xffffffffu, x, off);
    if (lane >= off) x += y;
  }
  if (lane == 31) warp_sums[warp] = x;
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
    T s = lane < nw ? warp_sums[lane] : T(0);
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const T y = __shfl_up_sync(0xffffffffu, s, off);
      if (lane >= off) s += y;
    }
    if (lane < nw) warp_sums[lane] = s;  // inclusive
  }
  __syncthreads();
  const T before = (warp > 0 ? warp_sums[warp - 1] : T(0)) + x - v;
  if (total) *total = warp_sums[(blockDim.x >> 5) - 1];
  return before;
}

template <typename T>
__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const T* __restrict__ d, int64_t L,
                                                              T* __restrict__ partial) {
  __shared__ T ws[32];
  const int64_t base = (int64_t)blockIdx.x * ScanCfg<T>::chunk;
  T s = 0;
  for (int j = 0; j < ScanCfg<T>::items; ++j) {
    const int64_t i = base + j * kScanThreads + threadIdx.x;
    if (i < L) s += d[i];
  }
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    T t = ws[threadIdx.x];
    for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
    if (threadIdx.x == 0) partial[blockIdx.x] = t;
  }
}

// exclusive scan of chunks of ScanCfg<T>::chunk values with an additive offset;
// `passes` > 1 only for the single-block scan of the partial sums
template <typename T>
__global__ void __launch_bounds__(kScanThreads) k_scan_apply(T* __restrict__ d, int64_t L,
                                                             const T* __restrict__ partial,
                                                             int passes) {
  __shared__ T buf[ScanCfg<T>::chunk];
  __shared__ T ws[32];
  __shared__ T carry_s;
  T carry = 0;
  for (int pass = 0; pass < passes; ++pass) {
    const int64_t base = ((int64_t)blockIdx.x + pass) * ScanCfg<T>::chunk;
    if (base >= L) break;
    for (int j = 0; j < ScanCfg<T>::items; ++j) {
      const int64_t i = base + j * kScanThreads + threadIdx.x;
      buf[j * kScanThreads + threadIdx.x] = i < L ? d[i] : T(0);
    }
    __syncthreads();
    T v[ScanCfg<T>::items], s = 0;
    for (int j = 0; j < ScanCfg<T>::items; ++j) {
      v[j] = buf[threadIdx.x * ScanCfg<T>::items + j];
      s += v[j];
    }
    T total;
    T run = block_exclusive_scan<T>(s, ws, &total);
    const T off = (partial ? partial[blockIdx.x] : T(0)) + carry;
    for (int j = 0; j < ScanCfg<T>::items; ++j) {
      buf[threadIdx.x * ScanCfg<T>::items + j] = run + off;
      run += v[j];
    }
    __syncthreads();
    for (int j = 0; j < ScanCfg<T>::items; ++j) {
      const int64_t i = base + j * kScanThreads + threadIdx.x;
      if (i < L) d[i] = buf[j * kScanThreads + threadIdx.x];
    }
    if (threadIdx.x == 0) carry_s = carry + total;
    __syncthreads();
    carry = carry_s;
    __syncthreads();
  }
}

size_t scan_tmp_ints(int64_t L) { return (size_t)ceil_div(L, ScanCfg<int>::chunk) + 1; }

template <typename T>
static void scan_exclusive_t(T* data, int64_t L, T* tmp, cudaStream_t s) {
  if (L <= 0) return;
  const int nb = ceil_div(L, ScanCfg<T>::chunk);
  if (nb == 1) {
    k_scan_apply<T><<<1, kScanThreads, 0, s>>>(data, L, nullptr, 1);
    note_launches(1);
    return;
  }
  note_launches(3);
  k_scan_reduce<T><<<nb, kScanThreads, 0, s>>>(data, L, tmp);
  k_scan_apply<T><<<1, kScanThreads, 0, s>>>(tmp, nb, nullptr, ceil_div(nb, ScanCfg<T>::chunk));
  k_scan_apply<T><<<nb, kScanThreads, 0, s>>>(data, L, tmp, 1);
}

void scan_exclusive(int* data, int64_t L, int* tmp, cudaStream_t s) {
  scan_exclusive_t<int>(data, L, tmp, s);
}
void scan_exclusive_i64(long long* data, int64_t L, long long* tmp, cudaStream_t s) {
  scan_exclusive_t<long long>(data, L, tmp, s);
}

static int radix_passes(int clouds) {
  int bits = 30;
  int c = 1;
  while (c < clouds) {
    c <<= 1;
    ++bits;
  }
  return (bits + kRadixBits - 1) / kRadixBits;
}

// sorts (k0, v0) using (k1, v1) as the second buffer; returns which buffer
// holds the result (0 or 1)
static int radix_sort(u64* k0, int* v0, u64* k1, int* v1, int64_t n, int passes, int* counts,
                      int* totals, int nblk, cudaStream_t s) {
  u64* ka[2] = {k0, k1};
  int* va[2] = {v0, v1};
  int cur = 0;
  for (int p = 0; p < passes; ++p) {
    const int shift = p * kRadixBits;
    k_radix_hist<<<nblk, kRsThreads, 0, s>>>(ka[cur], n, shift, counts, nblk);
    k_radix_digit_scan<<<kRadix / kDigitWarps, kDigitWarps * 32, 0, s>>>(counts, nblk, totals);
    k_radix_scatter<<<nblk, kRsThreads, 0, s>>>(ka[cur], va[cur], n, shift, counts, totals, nblk,
                                                ka[cur ^ 1], va[cur ^ 1]);
    note_launches(3);
    cur ^= 1;
  }
  return cur;
}

void radix_sort_plan(RadixPlan& p, Workspace& ws, int64_t n) {
  p.n = n;
  p.blocks = ceil_div(n > 0 ? n : 1, kRsTile);
  p.o_keys0 = ws.reserve(sizeof(u64) * (size_t)(n > 0 ? n : 1));
  p.o_keys1 = ws.reserve(sizeof(u64) * (size_t)(n > 0 ? n : 1));
  p.o_vals0 = ws.reserve(sizeof(int) * (size_t)(n > 0 ? n : 1));
  p.o_vals1 = ws.reserve(sizeof(int) * (size_t)(n > 0 ? n : 1));
  p.o_counts = ws.reserve(sizeof(int) * (size_t)kRadix * p.blocks);
  p.o_scan = ws.reserve(sizeof(int) * kRadix);  // digit totals
}

int radix_sort_pairs(const RadixPlan& p, const Workspace& ws, int bits, cudaStream_t s) {
  if (p.n <= 0) return 0;
  return radix_sort(ws.at<u64>(p.o_keys0), ws.at<int>(p.o_vals0), ws.at<u64>(p.o_keys1),
                    ws.at<int>(p.o_vals1), p.n, (bits + kRadixBits - 1) / kRadixBits,
                    ws.at<int>(p.o_counts), ws.at<int>(p.o_scan), p.blocks, s);
}

// ---------------------------------------------------------------------------
// 4. sorted points
// ---------------------------------------------------------------------------
__global__ void k_gather_sorted(const u64* __restrict__ keys, const int* __restrict__ vals, int64_t n,
                                const float* __restrict__ xyz, const GridParams* __restrict__ prm,
                                float4* __restrict__ pts) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int v = vals[i];
  const int c = (int)(keys[i] >> 30);
  const int local = v - prm[c].start;
  pts[i] = make_float4(xyz[3 * (int64_t)v], xyz[3 * (int64_t)v + 1], xyz[3 * (int64_t)v + 2],
                       __int_as_float(local));
}

// ---------------------------------------------------------------------------
// 5. level choice
// ---------------------------------------------------------------------------
// The level comes from the median, over kLevelSamples points spread evenly
// over the cloud's sorted order, of each point's k-th nearest distance among
// its 2k Morton neighbours on either side.  The samples are spread over many
// blocks (one cloud's estimate on one SM took ~39 us); one block per cloud
// then sorts them and picks the median.
constexpr int kLevelSamples = 1024;
constexpr int kLevelBlock = 128;

template <int KMAX>
__global__ void __launch_bounds__(kLevelBlock) k_level_samples(const GridParams* __restrict__ prm,
                                                               const float4* __restrict__ pts,
                                                               int k_default,
                                                               const int* __restrict__ cloud_k,
                                                               float* __restrict__ est) {
  const int cloud = blockIdx.y;
  const GridParams& P = prm[cloud];
  const int n = P.n, s0 = P.start;
  int k = cloud_k ? cloud_k[cloud] : k_default;
  k = max(1, min(k, KMAX));
  const int ns = min(kLevelSamples, n);
  const int s = blockIdx.x * kLevelBlock + threadIdx.x;  // < kLevelSamples
  float e = __int_as_float(0x7f800000);
  if (s < ns) {
    const int pos = s0 + (int)(((int64_t)s * n) / ns);
    const float4 q = pts[pos];
    const int W = 2 * k;
    TopK<KMAX> top;
    top.init(k);
    const int j0 = max(s0, pos - W), j1 = min(s0 + n - 1, pos + W);
    for (int j = j0; j <= j1; ++j) {
      const float4 p = pts[j];
      top.push(pack_key(sqdist(p.x, p.y, p.z, q.x, q.y, q.z), j));
    }
    if (top.full()) e = top.thr_d2();
  }
  est[(int64_t)cloud * kLevelSamples + s] = e;
}

// Level of each cloud: cell = fine * 2^level, the power of two nearest to
// cell_size (> 0) or to cell_scale x the median sampled k-th distance.
__global__ void __launch_bounds__(kLevelSamples) k_level_pick(GridParams* prm,
                                                              const float* __restrict__ est,
                                                              float cell_size, float cell_scale) {
  __shared__ float e[kLevelSamples];
  GridParams& P = prm[blockIdx.x];
  float target = cell_size;
  if (!(cell_size > 0.0f)) {
    e[threadIdx.x] = est[(int64_t)blockIdx.x * kLevelSamples + threadIdx.x];
    __syncthreads();
    // bitonic sort of e[] ascending
    for (int size = 2; size <= kLevelSamples; size <<= 1) {
      for (int stride = size >> 1; stride > 0; stride >>= 1) {
        const int t = threadIdx.x;
        if (t < kLevelSamples / 2) {
          const int lo = 2 * t - (t & (stride - 1));
          const int hi = lo + stride;
          const bool up = ((lo & size) == 0);
          const float a = e[lo], b = e[hi];
          if ((a > b) == up) {
            e[lo] = b;
            e[hi] = a;
          }
        }
        __syncthreads();
      }
    }
    const int ns = min(kLevelSamples, P.n);
    const float med = ns > 0 ? e[ns / 2] : __int_as_float(0x7f800000);
    const float R = isfinite(med) ? sqrtf(med) : P.fine * (float)kFineDim;
    target = (cell_scale > 0.0f ? cell_scale : kDefaultCellScale) * R;
  }
  if (threadIdx.x == 0) {
    const float ratio = target / P.fine;
    int L = ratio <= 1.0f ? 0 : (int)rintf(log2f(ratio));
    L = max(0, min(L, kFineBits));
    P.level = L;
    P.cell = ldexpf(P.fine, L);
  }
}

// ---------------------------------------------------------------------------
// 6. cell table
// ---------------------------------------------------------------------------
// Levels hashed in the table: the cloud's level L, the directory level of
// the correspondence search (L + 2) and the k-NN escalation levels (L + 3,
// + 6, + 9), each capped at 10, duplicates dropped (-1).
__device__ __forceinline__ int table_level(const GridParams& P, int slot) {
  const int add[5] = {0, 2, 3, 6, 9};
  const int lvl = min(P.level + add[slot], kFineBits);
  if (slot > 0 && lvl == min(P.level + add[slot - 1], kFineBits)) return -1;
  return lvl;
}
constexpr int kTableSlots = 5;

__device__ __forceinline__ bool same_cell(u64 a, u64 b, int L) {
  return (a >> 30) == (b >> 30) && ((unsigned)(a & 0x3fffffffu) >> (3 * L)) ==
                                       ((unsigned)(b & 0x3fffffffu) >> (3 * L));
}

__device__ __forceinline__ u64 key_cell(u64 key, int L) {
  const int c = (int)(key >> 30);
  const unsigned m = (unsigned)(key & 0x3fffffffu);
  return cell_key(L, c, (int)(compact3(m) >> L), (int)(compact3(m >> 1) >> L),
                  (int)(compact3(m >> 2) >> L));
}

__global__ void k_cells_insert(const u64* __restrict__ keys, int64_t n, const GridParams* prm,
                               CellEntry* tab, unsigned mask) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const u64 key = keys[i];
  const GridParams& P = prm[(int)(key >> 30)];
  for (int slot = 0; slot < kTableSlots; ++slot) {
    const int L = table_level(P, slot);
    if (L < 0) break;
    if (i > 0 && same_cell(keys[i - 1], key, L)) continue;
    const u64 K = key_cell(key, L);
    unsigned h = hash_key(K) & mask;
    for (unsigned probe = 0; probe <= mask; ++probe) {
      const u64 old = atomicCAS(&tab[h].key, kEmptyKey, K);
      if (old == kEmptyKey || old == K) break;
      h = (h + 1) & mask;
    }
    tab[h].start = (int)i;
    tab[h].count = 0;
  }
}

__global__ void k_cells_count(const u64* __restrict__ keys, int64_t n, const GridParams* prm,
                              CellEntry* tab, unsigned mask) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const u64 key = keys[i];
  const GridParams& P = prm[(int)(key >> 30)];
  for (int slot = 0; slot < kTableSlots; ++slot) {
    const int L = table_level(P, slot);
    if (L < 0) break;
    if (i + 1 < n && same_cell(keys[i + 1], key, L)) continue;
    const u64 K = key_cell(key, L);
    unsigned h = hash_key(K) & mask;
    for (unsigned probe = 0; probe <= mask; ++probe) {
      if (tab[h].key == K) {
        tab[h].count = (int)i - tab[h].start + 1;
        break;
      }
      h = (h + 1) & mask;
    }
  }
}

// ---------------------------------------------------------------------------
// host drivers
// ---------------------------------------------------------------------------
void grid_plan(GridPlan& p, Workspace& ws, int64_t n, int clouds) {
  p.n = n;
  p.clouds = clouds;
  // cells hashed in the table: at most min(points, cells of the level) for
  // each of its <= 5 levels (L, L+2, L+3, L+6, L+9); whatever the cloud's
  // level, that is <= 3n + 16^3 + 2^3 per cloud.  Keep the load factor <= 1/2.
  const uint64_t entries = 3 * (uint64_t)(n > 0 ? n : 1) + (uint64_t)clouds * (4096 + 8);
  const uint64_t slots = next_pow2_u32(2 * entries);
  p.mask = (unsigned)(slots - 1);
  p.radix_blocks = ceil_div(n > 0 ? n : 1, kRsTile);
  p.o_prm = ws.reserve(sizeof(GridParams) * clouds);
  p.o_pts = ws.reserve(sizeof(float4) * (size_t)(n > 0 ? n : 1));
  p.o_est = ws.reserve(sizeof(float) * kLevelSamples * (size_t)clouds);
  p.o_tab = ws.reserve(sizeof(CellEntry) * slots);
  p.o_keys0 = ws.reserve(sizeof(u64) * (size_t)(n > 0 ? n : 1));
  p.o_keys1 = ws.reserve(sizeof(u64) * (size_t)(n > 0 ? n : 1));
  p.o_vals0 = ws.reserve(sizeof(int) * (size_t)(n > 0 ? n : 1));
  p.o_vals1 = ws.reserve(sizeof(int) * (size_t)(n > 0 ? n : 1));
  p.o_counts = ws.reserve(sizeof(int) * (size_t)kRadix * p.radix_blocks);
  p.o_scan = ws.reserve(sizeof(int) * kRadix);  // digit totals
  p.o_starts = 0;
}

GridView grid_view(const GridPlan& p, const Workspace& ws) {
  GridView g;
  g.prm = ws.at<GridParams>(p.o_prm);
  g.pts = ws.at<float4>(p.o_pts);
  g.tab = ws.at<CellEntry>(p.o_tab);
  g.mask = p.mask;
  return g;
}

cil_status grid_build(const GridPlan& p, const Workspace& ws, const float* xyz,
                      const int* cloud_start_dev, const GridOptions& opt, DeviceCtx* ctx,
                      cudaStream_t s) {
  TimedRegion timer("grid_build", s);
  GridParams* prm = ws.at<GridParams>(p.o_prm);
  const int64_t n = p.n;
  note_launches(n > 0 ? 8 : 2);  // init, bbox, finalize, keys, gather, level pick, insert, count
  k_init_params<<<ceil_div(p.clouds, 128), 128, 0, s>>>(prm, p.clouds, cloud_start_dev, n);
  if (n > 0) {
    const int64_t threads = (n + 7) / 8;
    k_bbox<<<ceil_div(threads, 256), 256, 0, s>>>(xyz, n, cloud_start_dev, p.clouds, prm);
  }
  k_finalize<<<ceil_div(p.clouds, 128), 128, 0, s>>>(prm, p.clouds, ctx->err);
  const unsigned slots = p.mask + 1;
  if (cudaMemsetAsync(ws.at<CellEntry>(p.o_tab), 0xff, sizeof(CellEntry) * (size_t)slots, s) !=
      cudaSuccess)
    return CIL_ERR_CUDA;
  if (n > 0) {
    u64* k0 = ws.at<u64>(p.o_keys0);
    u64* k1 = ws.at<u64>(p.o_keys1);
    int* v0 = ws.at<int>(p.o_vals0);
    int* v1 = ws.at<int>(p.o_vals1);
    k_morton_keys<<<ceil_div(n, 256), 256, 0, s>>>(xyz, n, cloud_start_dev, p.clouds, prm, nullptr,
                                                   k0, v0);
    const int which = radix_sort(k0, v0, k1, v1, n, radix_passes(p.clouds), ws.at<int>(p.o_counts),
                                 ws.at<int>(p.o_scan), p.radix_blocks, s);
    u64* ks = which ? k1 : k0;
    int* vs = which ? v1 : v0;
    float4* pts = ws.at<float4>(p.o_pts);
    k_gather_sorted<<<ceil_div(n, 256), 256, 0, s>>>(ks, vs, n, xyz, prm, pts);
    const int kk = opt.k_est < 1 ? 1 : (opt.k_est > 32 ? 32 : opt.k_est);
    float* est = ws.at<float>(p.o_est);
    if (!(opt.cell_size > 0.0f)) {
      note_launches(1);
      const dim3 grid(kLevelSamples / kLevelBlock, p.clouds);
      CIL_FOR_K(kk, (k_level_samples<KM><<<grid, kLevelBlock, 0, s>>>(prm, pts, kk, nullptr, est)));
    }
    k_level_pick<<<p.clouds, kLevelSamples, 0, s>>>(prm, est, opt.cell_size, opt.cell_scale);
    k_cells_insert<<<ceil_div(n, 256), 256, 0, s>>>(ks, n, prm, ws.at<CellEntry>(p.o_tab), p.mask);
    k_cells_count<<<ceil_div(n, 256), 256, 0, s>>>(ks, n, prm, ws.at<CellEntry>(p.o_tab), p.mask);
  }
  return cudaGetLastError() == cudaSuccess ? CIL_OK : CIL_ERR_CUDA;
}

void order_plan(OrderPlan& p, Workspace& ws, int64_t n) {
  p.n = n;
  p.radix_blocks = ceil_div(n > 0 ? n : 1, kRsTile);
  p.o_keys0 = ws.reserve(sizeof(u64) * (size_t)(n > 0 ? n : 1));
  p.o_keys1 = ws.reserve(sizeof(u64) * (size_t)(n > 0 ? n : 1));
  p.o_vals0 = ws.reserve(sizeof(int) * (size_t)(n > 0 ? n : 1));
  p.o_vals1 = ws.reserve(sizeof(int) * (size_t)(n > 0 ? n : 1));
  p.o_counts = ws.reserve(sizeof(int) * (size_t)kRadix * p.radix_blocks);
  p.o_scan = ws.reserve(sizeof(int) * kRadix);  // digit totals
}

cil_status order_queries(const OrderPlan& p, const Workspace& ws, const float* qry,
                         const int* q_cloud_start_dev, int clouds, const GridParams* ref_prm,
                         const float* Rt_dev, int* order_out, cudaStream_t s) {
  const int64_t n = p.n;
  if (n <= 0) return CIL_OK;
  u64* k0 = ws.at<u64>(p.o_keys0);
  u64* k1 = ws.at<u64>(p.o_keys1);
  int* v0 = ws.at<int>(p.o_vals0);
  int* v1 = ws.at<int>(p.o_vals1);
  TimedRegion timer("order_queries", s);
  k_morton_keys<<<ceil_div(n, 256), 256, 0, s>>>(qry, n, q_cloud_start_dev, clouds, ref_prm, Rt_dev,
                                                 k0, v0);
  note_launches(1);
  const int which = radix_sort(k0, v0, k1, v1, n, radix_passes(clouds), ws.at<int>(p.o_counts),
                               ws.at<int>(p.o_scan), p.radix_blocks, s);
  if (cudaMemcpyAsync(order_out, which ? v1 : v0, sizeof(int) * (size_t)n, cudaMemcpyDeviceToDevice,
                      s) != cudaSuccess)
    return CIL_ERR_CUDA;
  return cudaGetLastError() == cudaSuccess ? CIL_OK : CIL_ERR_CUDA;
}

}  // namespace cil
