// pointnet.cu -- learned warm start for ICP: a PointNet-style regressor of a
// rigid transform, trained on the GPU by these kernels (no counterpart in the
// paper; it seeds the Sec. 3 point-to-plane ICP).
//
// Network (per pair b: clouds c = 2b (source) and 2b+1 (target), P points):
//   encoder  Z1 = W1 x + b1 (3->64, FP32 ALU), A1 = relu(Z1) -> bf16
//            Z2 = W2 A1 + b2 (64->128, BF16 tensor cores, FP32 accumulate)
//            Z3 = W3 A2 + b3 (128->256, BF16 tensor cores, FP32 accumulate)
//            f[c] = max over points of relu(Z3), argmax row kept for backward
//   head     h = [f_src, f_dst] (512) -> relu(W4 h + b4) (256) -> W5 . + b5 (9)
//            R = Gram-Schmidt(o[0:3], o[3:6]), t = o[6:9]
//   loss     mean over pairs of mean over source points |(R p + t) - (Rg p + tg)|^2
// The encoder runs as one persistent kernel: each block keeps W2, W3 (bf16)
// resident in shared memory and streams 128-point tiles through layer 1,
// two warp-level MMA GEMMs and a fused bias + ReLU + column max epilogue;
// the per-cloud max is combined with 64-bit atomicMax on (value, ~row) keys,
// so ties resolve to the smallest row and the result is order independent.
// Backward: the max-pool passes gradient only to the argmax row of each
// channel, so the encoder backward touches <= 256 rows per cloud and is
// recomputed from those rows in FP32 on the CUDA cores; per-cloud and
// per-pair gradient partials are reduced in a fixed order (deterministic).
#include <cuda_bf16.h>
#include <math.h>

#include "cil_host.h"
#include "cil_kernels.h"
#include "tc05.cuh"

namespace cil {

// ---------------------------------------------------------------------------
// parameter layout (FP32, in this order): W1 b1 W2 b2 W3 b3 W4 b4 W5 b5
// ---------------------------------------------------------------------------
constexpr int kH1 = 64, kH2 = 128, kH3 = 256, kH4 = 256, kOut = 9, kIn = 3;
constexpr int oW1 = 0, oB1 = oW1 + kH1 * kIn, oW2 = oB1 + kH1, oB2 = oW2 + kH2 * kH1,
              oW3 = oB2 + kH2, oB3 = oW3 + kH3 * kH2, oW4 = oB3 + kH3,
              oB4 = oW4 + kH4 * 2 * kH3, oW5 = oB4 + kH4, oB5 = oW5 + kOut * kH4,
              kNParams = oB5 + kOut;
constexpr int kEncParams = oW4;  // W1..b3 live in the encoder

constexpr int kTileP = 128;      // points per encoder tile

struct PnState {
  int max_pairs, P;
  float* params;    // FP32 master [kNParams]
  float* grad;      // [kNParams]
  float* m;         // Adam first moment
  float* v;         // Adam second moment
  __nv_bfloat16* w2b;  // [128][64]
  __nv_bfloat16* w3b;  // [256][128]
  float* w4t;       // W4 transposed [512][256]
  u64* feat_key;    // [2B][256] packed (value, ~row)
  float* h;         // [B][512]
  float* z4;        // [B][256]
  float* o;         // [B][9]
  float* dz4;       // [B][256]
  float* dout;      // [B][9]
  float* df;        // [2B][256]
  float* loss;      // [B]
  float* enc_part;  // [2B][kEncParams] per-cloud encoder gradient partials
  long long step;
  void* base;
};

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned pack_bf16x2(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const unsigned*>(&v);
}

__device__ __forceinline__ u64 feat_pack(float v, int row) {
  return ((u64)__float_as_uint(v) << 32) | (u64)(0xffffffffu - (unsigned)row);
}
__device__ __forceinline__ float feat_val(u64 k) { return __uint_as_float((unsigned)(k >> 32)); }
__device__ __forceinline__ int feat_row(u64 k) { return (int)(0xffffffffu - (unsigned)(k & 0xffffffffu)); }

// ---------------------------------------------------------------------------
// encoder forward on the 5th-generation tensor cores (tcgen05 + TMEM)
// ---------------------------------------------------------------------------
// kTcParts x 128 threads: threads r, r + 128, ... own point row r of a
// 128-point tile (warp w reads tensor-memory lanes 32 (w % 4) ..), part
// w / 4 one kTcParts-th of each layer's channels, so the CUDA-core work
// between the MMAs (layer 1, the two epilogues) is split over 4 kTcParts
// warps.  Operands live in shared memory as K-major BF16 tiles with the
// 128-byte swizzle (64-element rows); the two GEMMs accumulate in tensor
// memory (columns 0..127: layer 2, 128..383: layer 3), issued by one thread
// and completed through an mbarrier.
constexpr int kTcParts = 4;
constexpr int kTcThreads = 128 * kTcParts;
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kMbarPolls = 1u << 26;  // bounded wait (~seconds)

struct EncTcSmem {
  uint8_t a1[kTileP * 128];      // [128 rows][64 k]
  uint8_t w2[kH2 * 128];         // [128 n][64 k]
  uint8_t a2[2][kTileP * 128];   // two 64-wide k blocks of [128 rows][64 k]
  uint8_t w3[2][kH3 * 128];      // two 64-wide k blocks of [256 n][64 k]
  float w1[kH1 * kIn];
  float b1[kH1];
  float b2[kH2];
  float b3[kH3];
  float red[4 * kTcParts][32][33];  // per-warp transpose for the column max
  u64 wmax[4][kH3];              // per-warp column maxima of one tile
  uint64_t bar;
  uint32_t tmem_base;
  int abort;
};

static size_t enc_tc_smem() { return sizeof(EncTcSmem) + 1024; }

__global__ void __launch_bounds__(kTcThreads, 1) k_pn_encode_tc(
    const float* __restrict__ X, int clouds, int P, const float* __restrict__ prm,
    const __nv_bfloat16* __restrict__ w2b, const __nv_bfloat16* __restrict__ w3b,
    u64* __restrict__ feat_key, int* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // operand tiles need 1024-byte alignment (swizzle atom)
  const uint32_t raw_s = tc::smem_u32(smem_raw);
  EncTcSmem& S = *reinterpret_cast<EncTcSmem*>(smem_raw + (((raw_s + 1023u) & ~1023u) - raw_s));
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int quarter = warp & 3;  // tensor-memory lanes (tile rows) 32 quarter ..
  const int half = warp >> 2;    // which part of each layer's channels
  const int row = tid & 127;     // this thread's tile row
  if (warp == 0) {
    tc::tmem_alloc(&S.tmem_base, kTmemCols);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    tc::mbar_init(&S.bar, 1);
    tc::fence_mbar_init();
    S.abort = 0;
  }
  // resident weights, swizzled: 16-byte chunks of 8 bf16
  for (int e = tid; e < kH2 * 8; e += kTcThreads) {
    const int n = e >> 3, c = e & 7;
    *reinterpret_cast<uint4*>(S.w2 + tc::sw128_offset(n, 8 * c)) =
        *reinterpret_cast<const uint4*>(w2b + n * kH1 + 8 * c);
  }
  for (int e = tid; e < kH3 * 16; e += kTcThreads) {
    const int n = e >> 4, c = e & 15;
    *reinterpret_cast<uint4*>(S.w3[c >> 3] + tc::sw128_offset(n, 8 * (c & 7))) =
        *reinterpret_cast<const uint4*>(w3b + n * kH2 + 8 * c);
  }
  for (int e = tid; e < kH1 * kIn; e += kTcThreads) S.w1[e] = prm[oW1 + e];
  for (int e = tid; e < kH1; e += kTcThreads) S.b1[e] = prm[oB1 + e];
  for (int e = tid; e < kH2; e += kTcThreads) S.b2[e] = prm[oB2 + e];
  for (int e = tid; e < kH3; e += kTcThreads) S.b3[e] = prm[oB3 + e];
  tc::fence_async_smem();
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = S.tmem_base;
  const uint32_t lane_base = (uint32_t)(32 * quarter) << 16;
  const uint32_t id2 = tc::idesc_bf16_f32(128, kH2);
  const uint32_t id3 = tc::idesc_bf16_f32(128, kH3);
  uint32_t phase = 0;

  const int tiles_per_cloud = P / kTileP;
  const int total = clouds * tiles_per_cloud;
  for (int t = blockIdx.x; t < total; t += gridDim.x) {
    const int cloud = t / tiles_per_cloud;
    const int row0 = (t % tiles_per_cloud) * kTileP;
    // ---- layer 1 (FP32 ALU): row `row`, this part's channels -> bf16 A1 ----
    {
      const float* xp = X + ((int64_t)cloud * P + row0 + row) * 3;
      const float x = xp[0], y = xp[1], z = xp[2];
#pragma unroll
      for (int cc = 0; cc < 8 / kTcParts; ++cc) {
        const int c = (8 / kTcParts) * half + cc;
        unsigned w[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          const int ch = 8 * c + 2 * h;
          const float* wr = S.w1 + ch * 3;
          const float z0 = fmaf(wr[0], x, fmaf(wr[1], y, fmaf(wr[2], z, S.b1[ch])));
          const float z1 = fmaf(wr[3], x, fmaf(wr[4], y, fmaf(wr[5], z, S.b1[ch + 1])));
          w[h] = pack_bf16x2(fmaxf(z0, 0.0f), fmaxf(z1, 0.0f));
        }
        *reinterpret_cast<uint4*>(S.a1 + tc::sw128_offset(row, 8 * c)) =
            make_uint4(w[0], w[1], w[2], w[3]);
      }
    }
    tc::fence_async_smem();
    tc::tc_fence_before();
    __syncthreads();
    // ---- layer 2: D[0:128) = A1 [128x64] * W2^T ----
    if (tid == 0) {
      tc::tc_fence_after();
      const uint32_t a = tc::smem_u32(S.a1), b = tc::smem_u32(S.w2);
#pragma unroll
      for (int ks = 0; ks < 4; ++ks)
        tc::mma_bf16(tmem, tc::smem_desc_sw128(a + 32 * ks), tc::smem_desc_sw128(b + 32 * ks), id2,
                     ks > 0);
      tc::mma_commit(&S.bar);
    }
    bool ok = tc::mbar_wait(&S.bar, phase, kMbarPolls);
    phase ^= 1u;
    if (__syncthreads_or(!ok)) {
      if (tid == 0) atomicCAS(err, 0, (int)CIL_ERR_TIMEOUT);
      break;
    }
    tc::tc_fence_after();
    // ---- epilogue 2: bias + relu -> bf16 A2 (two 64-wide k blocks) ----
#pragma unroll 1
    for (int jj = 0; jj < 4 / kTcParts; ++jj) {
      const int j = (4 / kTcParts) * half + jj;
      float v[32];
      tc::tmem_ld32(tmem + lane_base + 32 * j, v);
      uint8_t* blk = S.a2[j >> 1];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        unsigned w[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          const int col = 32 * j + 8 * c + 2 * h;
          w[h] = pack_bf16x2(fmaxf(v[8 * c + 2 * h] + S.b2[col], 0.0f),
                             fmaxf(v[8 * c + 2 * h + 1] + S.b2[col + 1], 0.0f));
        }
        *reinterpret_cast<uint4*>(blk + tc::sw128_offset(row, (32 * j + 8 * c) & 63)) =
            make_uint4(w[0], w[1], w[2], w[3]);
      }
    }
    tc::fence_async_smem();
    tc::tc_fence_before();
    __syncthreads();
    // ---- layer 3: D[128:384) = A2 [128x128] * W3^T ----
    if (tid == 0) {
      tc::tc_fence_after();
#pragma unroll
      for (int ks = 0; ks < 8; ++ks) {
        const uint32_t a = tc::smem_u32(S.a2[ks >> 2]) + 32 * (ks & 3);
        const uint32_t b = tc::smem_u32(S.w3[ks >> 2]) + 32 * (ks & 3);
        tc::mma_bf16(tmem + kH2, tc::smem_desc_sw128(a), tc::smem_desc_sw128(b), id3, ks > 0);
      }
      tc::mma_commit(&S.bar);
    }
    ok = tc::mbar_wait(&S.bar, phase, kMbarPolls);
    phase ^= 1u;
    if (__syncthreads_or(!ok)) {
      if (tid == 0) atomicCAS(err, 0, (int)CIL_ERR_TIMEOUT);
      break;
    }
    tc::tc_fence_after();
    // ---- epilogue 3: bias + relu, column (value, row) max of the tile ----
#pragma unroll 1
    for (int jj = 0; jj < 8 / kTcParts; ++jj) {
      const int j = (8 / kTcParts) * half + jj;
      float v[32];
      tc::tmem_ld32(tmem + lane_base + kH2 + 32 * j, v);
#pragma unroll
      for (int i = 0; i < 32; ++i) S.red[warp][lane][i] = fmaxf(v[i] + S.b3[32 * j + i], 0.0f);
      __syncwarp();
      float best = S.red[warp][0][lane];
      int br = 0;
      for (int rr = 1; rr < 32; ++rr) {
        const float x = S.red[warp][rr][lane];
        if (x > best) {  // strict: ties keep the smaller row
          best = x;
          br = rr;
        }
      }
      S.wmax[quarter][32 * j + lane] = feat_pack(best, row0 + 32 * quarter + br);
      __syncwarp();
    }
    tc::tc_fence_before();
    __syncthreads();
    for (int c = tid; c < kH3; c += kTcThreads) {
      u64 m = S.wmax[0][c];
#pragma unroll
      for (int w = 1; w < 4; ++w) m = max(m, S.wmax[w][c]);
      atomicMax(feat_key + (int64_t)cloud * kH3 + c, m);
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, kTmemCols);
  }
}

// A wait on an mbarrier nothing ever arrives on, bounded like the encoder's
// waits: it gives up after `polls` polls, records CIL_ERR_TIMEOUT in the error
// word and returns (the failure path of a stalled tensor-core pipeline, made
// without stalling anything).
__global__ void k_bounded_wait_check(uint32_t polls, int* err) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    tc::fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0 && !tc::mbar_wait(&bar, 0, polls)) atomicCAS(err, 0, (int)CIL_ERR_TIMEOUT);
}

cil_status launch_bounded_wait_check(uint32_t polls, int* err, cudaStream_t s) {
  note_launches(1);
  k_bounded_wait_check<<<1, 32, 0, s>>>(polls, err);
  return cudaGetLastError() == cudaSuccess ? CIL_OK : CIL_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// head forward (+ transform output), one block per pair
// ---------------------------------------------------------------------------
__device__ void gram_schmidt3(const float a1[3], const float a2[3], float R[9]) {
  const float n1 = sqrtf(a1[0] * a1[0] + a1[1] * a1[1] + a1[2] * a1[2]);
  float b1[3] = {a1[0] / n1, a1[1] / n1, a1[2] / n1};
  const float d = b1[0] * a2[0] + b1[1] * a2[1] + b1[2] * a2[2];
  float u2[3] = {a2[0] - d * b1[0], a2[1] - d * b1[1], a2[2] - d * b1[2]};
  const float n2 = sqrtf(u2[0] * u2[0] + u2[1] * u2[1] + u2[2] * u2[2]);
  float b2[3] = {u2[0] / n2, u2[1] / n2, u2[2] / n2};
  float b3[3] = {b1[1] * b2[2] - b1[2] * b2[1], b1[2] * b2[0] - b1[0] * b2[2],
                 b1[0] * b2[1] - b1[1] * b2[0]};
  for (int i = 0; i < 3; ++i) {  // columns b1 b2 b3, row-major R
    R[3 * i] = b1[i];
    R[3 * i + 1] = b2[i];
    R[3 * i + 2] = b3[i];
  }
}

__global__ void __launch_bounds__(256) k_pn_head(const float* __restrict__ prm,
                                                 const float* __restrict__ w4t,
                                                 const u64* __restrict__ feat_key, int B,
                                                 float* __restrict__ h_out, float* __restrict__ z4_out,
                                                 float* __restrict__ o_out, double* __restrict__ T_out) {
  __shared__ float h[2 * kH3];
  __shared__ float a4[kH4];
  __shared__ float o[kOut];
  const int b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int k = tid; k < 2 * kH3; k += 256) {
    h[k] = feat_val(feat_key[(int64_t)(2 * b + k / kH3) * kH3 + (k % kH3)]);
    if (h_out) h_out[(int64_t)b * 2 * kH3 + k] = h[k];
  }
  __syncthreads();
  {
    const int c = tid;
    float z = prm[oB4 + c];
    for (int k = 0; k < 2 * kH3; ++k) z = fmaf(w4t[k * kH4 + c], h[k], z);
    if (z4_out) z4_out[(int64_t)b * kH4 + c] = z;
    a4[c] = fmaxf(z, 0.0f);
  }
  __syncthreads();
  for (int oi = warp; oi < kOut; oi += 8) {
    float s = 0.0f;
    for (int c = lane; c < kH4; c += 32) s = fmaf(prm[oW5 + oi * kH4 + c], a4[c], s);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if (lane == 0) o[oi] = s + prm[oB5 + oi];
  }
  __syncthreads();
  if (tid == 0) {
    if (o_out)
      for (int j = 0; j < kOut; ++j) o_out[(int64_t)b * kOut + j] = o[j];
    if (T_out) {
      float R[9];
      gram_schmidt3(o, o + 3, R);
      double* T = T_out + 16 * (int64_t)b;
      for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) T[4 * i + j] = (double)R[3 * i + j];
        T[4 * i + 3] = (double)o[6 + i];
      }
      T[12] = 0.0;
      T[13] = 0.0;
      T[14] = 0.0;
      T[15] = 1.0;
    }
  }
}

// ---------------------------------------------------------------------------
// loss + head backward, one block per pair
// ---------------------------------------------------------------------------
__device__ void gs_backward(const float a1[3], const float a2[3], const float dR[9], float ga1[3],
                            float ga2[3]) {
  const float n1 = sqrtf(a1[0] * a1[0] + a1[1] * a1[1] + a1[2] * a1[2]);
  float b1[3], u2[3], b2[3], g1[3], g2[3], g3[3];
  for (int i = 0; i < 3; ++i) b1[i] = a1[i] / n1;
  const float d = b1[0] * a2[0] + b1[1] * a2[1] + b1[2] * a2[2];
  for (int i = 0; i < 3; ++i) u2[i] = a2[i] - d * b1[i];
  const float n2 = sqrtf(u2[0] * u2[0] + u2[1] * u2[1] + u2[2] * u2[2]);
  for (int i = 0; i < 3; ++i) {
    b2[i] = u2[i] / n2;
    g1[i] = dR[3 * i];  // dL/d(column 0)
    g2[i] = dR[3 * i + 1];
    g3[i] = dR[3 * i + 2];
  }
  // b3 = b1 x b2:  dL/db1 += b2 x g3,  dL/db2 += g3 x b1
  g1[0] += b2[1] * g3[2] - b2[2] * g3[1];
  g1[1] += b2[2] * g3[0] - b2[0] * g3[2];
  g1[2] += b2[0] * g3[1] - b2[1] * g3[0];
  g2[0] += g3[1] * b1[2] - g3[2] * b1[1];
  g2[1] += g3[2] * b1[0] - g3[0] * b1[2];
  g2[2] += g3[0] * b1[1] - g3[1] * b1[0];
  // b2 = u2 / n2
  const float g2b2 = g2[0] * b2[0] + g2[1] * b2[1] + g2[2] * b2[2];
  float gu2[3];
  for (int i = 0; i < 3; ++i) gu2[i] = (g2[i] - g2b2 * b2[i]) / n2;
  // u2 = a2 - (b1 . a2) b1
  const float gu2b1 = gu2[0] * b1[0] + gu2[1] * b1[1] + gu2[2] * b1[2];
  float gb1[3];
  for (int i = 0; i < 3; ++i) {
    ga2[i] = gu2[i] - gu2b1 * b1[i];
    gb1[i] = g1[i] - d * gu2[i] - gu2b1 * a2[i];
  }
  // b1 = a1 / n1
  const float gb1b1 = gb1[0] * b1[0] + gb1[1] * b1[1] + gb1[2] * b1[2];
  for (int i = 0; i < 3; ++i) ga1[i] = (gb1[i] - gb1b1 * b1[i]) / n1;
}

__global__ void __launch_bounds__(256) k_pn_loss_head_bwd(
    const float* __restrict__ prm, const float* __restrict__ X, int P, int B,
    const double* __restrict__ T_gt, const float* __restrict__ z4, const float* __restrict__ o_in,
    float* __restrict__ loss, float* __restrict__ dz4_out, float* __restrict__ dout_out,
    float* __restrict__ df_out) {
  __shared__ float red[8][13];
  __shared__ float sums[13];
  __shared__ float dz4[kH4];
  __shared__ float dov[kOut];
  const int b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float o[kOut];
  for (int j = 0; j < kOut; ++j) o[j] = o_in[(int64_t)b * kOut + j];
  float R[9];
  gram_schmidt3(o, o + 3, R);
  float D[9], dt[3];
  const double* Tg = T_gt + 16 * (int64_t)b;
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) D[3 * i + j] = R[3 * i + j] - (float)Tg[4 * i + j];
    dt[i] = o[6 + i] - (float)Tg[4 * i + 3];
  }
  // per point: e = D p + dt;  accumulate |e|^2, e p^T (9), e (3)
  float acc[13];
  for (int j = 0; j < 13; ++j) acc[j] = 0.0f;
  const float* src = X + (int64_t)(2 * b) * P * 3;
  for (int p = tid; p < P; p += 256) {
    const float x = src[3 * p], y = src[3 * p + 1], z = src[3 * p + 2];
    float e[3];
    for (int i = 0; i < 3; ++i) e[i] = fmaf(D[3 * i], x, fmaf(D[3 * i + 1], y, fmaf(D[3 * i + 2], z, dt[i])));
    acc[0] += e[0] * e[0] + e[1] * e[1] + e[2] * e[2];
    for (int i = 0; i < 3; ++i) {
      acc[1 + 3 * i] += e[i] * x;
      acc[2 + 3 * i] += e[i] * y;
      acc[3 + 3 * i] += e[i] * z;
      acc[10 + i] += e[i];
    }
  }
  for (int j = 0; j < 13; ++j) {
    float v = acc[j];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (lane == 0) red[warp][j] = v;
  }
  __syncthreads();
  if (tid < 13) {
    float v = 0.0f;
    for (int w = 0; w < 8; ++w) v += red[w][tid];
    sums[tid] = v;
  }
  __syncthreads();
  if (tid == 0) {
    loss[b] = sums[0] / (float)P;
    // L_total = (1/B) sum_b (1/P) sum_p |e|^2
    const float sc = 2.0f / ((float)B * (float)P);
    float dR[9], ga1[3], ga2[3];
    for (int j = 0; j < 9; ++j) dR[j] = sc * sums[1 + j];
    gs_backward(o, o + 3, dR, ga1, ga2);
    for (int i = 0; i < 3; ++i) {
      dov[i] = ga1[i];
      dov[3 + i] = ga2[i];
      dov[6 + i] = sc * sums[10 + i];
    }
    for (int j = 0; j < kOut; ++j) dout_out[(int64_t)b * kOut + j] = dov[j];
  }
  __syncthreads();
  {
    const int c = tid;  // dA4 = W5^T do, dZ4 = dA4 * (Z4 > 0)
    float s = 0.0f;
    for (int j = 0; j < kOut; ++j) s = fmaf(prm[oW5 + j * kH4 + c], dov[j], s);
    const float d = z4[(int64_t)b * kH4 + c] > 0.0f ? s : 0.0f;
    dz4[c] = d;
    dz4_out[(int64_t)b * kH4 + c] = d;
  }
  __syncthreads();
  for (int k = tid; k < 2 * kH3; k += 256) {  // dh = W4^T dZ4
    float s = 0.0f;
    for (int c = 0; c < kH4; ++c) s = fmaf(prm[oW4 + c * 2 * kH3 + k], dz4[c], s);
    df_out[(int64_t)(2 * b + k / kH3) * kH3 + (k % kH3)] = s;
  }
}

// head weight gradients: sum over pairs in pair order (deterministic)
__global__ void k_pn_head_wgrad(const float* __restrict__ h, const float* __restrict__ z4,
                                const float* __restrict__ dz4, const float* __restrict__ dout, int B,
                                float* __restrict__ grad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int nW4 = kH4 * 2 * kH3, nW5 = kOut * kH4;
  if (i < nW4) {
    const int c = i / (2 * kH3), k = i % (2 * kH3);
    float s = 0.0f;
    for (int b = 0; b < B; ++b) s = fmaf(dz4[(int64_t)b * kH4 + c], h[(int64_t)b * 2 * kH3 + k], s);
    grad[oW4 + i] = s;
  } else if (i < nW4 + kH4) {
    const int c = i - nW4;
    float s = 0.0f;
    for (int b = 0; b < B; ++b) s += dz4[(int64_t)b * kH4 + c];
    grad[oB4 + c] = s;
  } else if (i < nW4 + kH4 + nW5) {
    const int e = i - nW4 - kH4, j = e / kH4, c = e % kH4;
    float s = 0.0f;
    for (int b = 0; b < B; ++b)
      s = fmaf(dout[(int64_t)b * kOut + j], fmaxf(z4[(int64_t)b * kH4 + c], 0.0f), s);
    grad[oW5 + e] = s;
  } else if (i < nW4 + kH4 + nW5 + kOut) {
    const int j = i - nW4 - kH4 - nW5;
    float s = 0.0f;
    for (int b = 0; b < B; ++b) s += dout[(int64_t)b * kOut + j];
    grad[oB5 + j] = s;
  }
}

// ---------------------------------------------------------------------------
// encoder backward: one block per cloud, thread = output channel of layer 3
// ---------------------------------------------------------------------------
struct EncBwdSmem {
  float g2[kH3][kH2 + 1];          // dZ2 rows per channel (reused for dZ1); padded
  __nv_bfloat16 a1[kH3][kH1 + 2];  // bf16 A1 of each channel's argmax row; padded
  float x[kH3][4];
};

__global__ void __launch_bounds__(256, 1) k_pn_encode_bwd(
    const float* __restrict__ X, int P, const float* __restrict__ prm,
    const __nv_bfloat16* __restrict__ w2b, const __nv_bfloat16* __restrict__ w3b,
    const u64* __restrict__ feat_key, const float* __restrict__ df, float* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  EncBwdSmem& S = *reinterpret_cast<EncBwdSmem*>(smem_raw);
  const int cloud = blockIdx.x, c = threadIdx.x;
  float* out = part + (int64_t)cloud * kEncParams;
  const u64 key = feat_key[(int64_t)cloud * kH3 + c];
  const float fv = feat_val(key);
  const int r = min(max(feat_row(key), 0), P - 1);
  const float gch = fv > 0.0f ? df[(int64_t)cloud * kH3 + c] : 0.0f;
  const float* xp = X + ((int64_t)cloud * P + r) * 3;
  const float x = xp[0], y = xp[1], z = xp[2];
  S.x[c][0] = x;
  S.x[c][1] = y;
  S.x[c][2] = z;
  unsigned long long pos1 = 0ull;  // bit k: Z1[k] > 0 at this row
#pragma unroll
  for (int k = 0; k < kH1; ++k) {
    const float z1 = fmaf(prm[oW1 + 3 * k], x,
                          fmaf(prm[oW1 + 3 * k + 1], y, fmaf(prm[oW1 + 3 * k + 2], z, prm[oB1 + k])));
    if (z1 > 0.0f) pos1 |= 1ull << k;
    S.a1[c][k] = __float2bfloat16_rn(fmaxf(z1, 0.0f));
  }
  // Z2 = W2b A1b + b2 ; dW3 row c = g * A2b ; dZ2 = g * W3b[c] * (Z2 > 0).
  // Four outputs at a time (each still summed over k in order): four
  // independent FMA chains, one shared-memory read of A1 for four of them.
  constexpr int kOB = 4;
#pragma unroll 1
  for (int o0 = 0; o0 < kH2; o0 += kOB) {
    float sv[kOB];
#pragma unroll
    for (int u = 0; u < kOB; ++u) sv[u] = prm[oB2 + o0 + u];
#pragma unroll 2
    for (int k0 = 0; k0 < kH1; k0 += 8) {
      // 8 weights of each row in one 16-byte load (rows of 64 bf16 are
      // 128-byte aligned)
      uint4 wv[kOB];
#pragma unroll
      for (int u = 0; u < kOB; ++u)
        wv[u] = __ldg(reinterpret_cast<const uint4*>(w2b + (o0 + u) * kH1 + k0));
#pragma unroll
      for (int h = 0; h < 8; ++h) {
        const float av = __bfloat162float(S.a1[c][k0 + h]);
#pragma unroll
        for (int u = 0; u < kOB; ++u) {
          const __nv_bfloat16* w8 = reinterpret_cast<const __nv_bfloat16*>(&wv[u]);
          sv[u] = fmaf(__bfloat162float(w8[h]), av, sv[u]);
        }
      }
    }
    float4 w3o;
    float* w3p = &w3o.x;
#pragma unroll
    for (int u = 0; u < kOB; ++u) {
      const float sz = sv[u];
      const float a2 = __bfloat162float(__float2bfloat16_rn(fmaxf(sz, 0.0f)));
      w3p[u] = gch * a2;
      S.g2[c][o0 + u] = sz > 0.0f ? gch * __bfloat162float(w3b[c * kH2 + o0 + u]) : 0.0f;
    }
    *reinterpret_cast<float4*>(out + oW3 + c * kH2 + o0) = w3o;
  }
  out[oB3 + c] = gch;
  // dA1 = W2b^T dZ2, dZ1 = dA1 * (Z1 > 0)
  float dz1[kH1];
#pragma unroll
  for (int k = 0; k < kH1; ++k) dz1[k] = 0.0f;
#pragma unroll 1
  for (int o = 0; o < kH2; ++o) {
    const float gv = S.g2[c][o];
#pragma unroll
    for (int k0 = 0; k0 < kH1; k0 += 8) {
      const uint4 wv = __ldg(reinterpret_cast<const uint4*>(w2b + o * kH1 + k0));
      const __nv_bfloat16* w8 = reinterpret_cast<const __nv_bfloat16*>(&wv);
#pragma unroll
      for (int h = 0; h < 8; ++h) dz1[k0 + h] = fmaf(__bfloat162float(w8[h]), gv, dz1[k0 + h]);
    }
  }
#pragma unroll
  for (int k = 0; k < kH1; ++k) dz1[k] = ((pos1 >> k) & 1ull) ? dz1[k] : 0.0f;
  __syncthreads();
  // dW2[o][k] = sum_c dZ2[c][o] A1[c][k],  db2[o] = sum_c dZ2[c][o]  (c in order)
  // four elements e, e + 256, ... at a time (each summed over channels in
  // order): independent chains
  static_assert((kH2 * kH1) % (4 * 256) == 0, "dW2 blocking");
  for (int e0 = threadIdx.x; e0 < kH2 * kH1; e0 += 4 * 256) {
    float sv[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    for (int cc = 0; cc < kH3; ++cc) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int e = e0 + 256 * u, o = e / kH1, k = e % kH1;
        sv[u] = fmaf(S.g2[cc][o], __bfloat162float(S.a1[cc][k]), sv[u]);
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) out[oW2 + e0 + 256 * u] = sv[u];
  }
  if (threadIdx.x < kH2) {
    float s = 0.0f;
    for (int cc = 0; cc < kH3; ++cc) s += S.g2[cc][threadIdx.x];
    out[oB2 + threadIdx.x] = s;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kH1; ++k) S.g2[c][k] = dz1[k];
  __syncthreads();
  for (int e = threadIdx.x; e < kH1 * kIn; e += 256) {
    const int o = e / kIn, j = e % kIn;
    float s = 0.0f;
    for (int cc = 0; cc < kH3; ++cc) s = fmaf(S.g2[cc][o], S.x[cc][j], s);
    out[oW1 + e] = s;
  }
  if (threadIdx.x < kH1) {
    float s = 0.0f;
    for (int cc = 0; cc < kH3; ++cc) s += S.g2[cc][threadIdx.x];
    out[oB1 + threadIdx.x] = s;
  }
}

// encoder gradient: sum of the per-cloud partials in cloud order
__global__ void k_pn_enc_reduce(const float* __restrict__ part, int clouds, float* __restrict__ grad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kEncParams) return;
  float s = 0.0f;
  for (int c = 0; c < clouds; ++c) s += part[(int64_t)c * kEncParams + i];
  grad[i] = s;
}

// Adam on the FP32 master weights, then refresh the bf16 / transposed copies
__global__ void k_pn_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                          float* __restrict__ v, float lr, float b1, float b2, float eps, float c1,
                          float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kNParams) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.0f - b1) * gi;
  const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void k_pn_refresh(const float* __restrict__ w, __nv_bfloat16* __restrict__ w2b,
                             __nv_bfloat16* __restrict__ w3b, float* __restrict__ w4t) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < kH2 * kH1) w2b[i] = __float2bfloat16_rn(w[oW2 + i]);
  if (i < kH3 * kH2) w3b[i] = __float2bfloat16_rn(w[oW3 + i]);
  if (i < kH4 * 2 * kH3) {
    const int c = i / (2 * kH3), k = i % (2 * kH3);
    w4t[k * kH4 + c] = w[oW4 + i];
  }
}

static size_t enc_bwd_smem() { return sizeof(EncBwdSmem); }

}  // namespace cil

using namespace cil;

struct cil_pointnet {
  PnState s;
  DeviceCtx* ctx;
  cudaStream_t own;
};

static cil_status pn_forward_enqueue(cil_pointnet* h, const float* clouds, int B, double* T_out,
                                     cudaStream_t s) {
  PnState& S = h->s;
  if (cudaMemsetAsync(S.feat_key, 0, sizeof(u64) * 2 * B * kH3, s) != cudaSuccess) return CIL_ERR_CUDA;
  const int tiles = 2 * B * (S.P / kTileP);
  const int grid = tiles < h->ctx->num_sms ? tiles : h->ctx->num_sms;
  {
    TimedRegion timer("k_pn_encode", s);
    note_launches(2);
    k_pn_encode_tc<<<grid, kTcThreads, enc_tc_smem(), s>>>(clouds, 2 * B, S.P, S.params, S.w2b,
                                                           S.w3b, S.feat_key, h->ctx->err);
    k_pn_head<<<B, 256, 0, s>>>(S.params, S.w4t, S.feat_key, B, S.h, S.z4, S.o, T_out);
  }
  return cudaGetLastError() == cudaSuccess ? CIL_OK : CIL_ERR_CUDA;
}

extern "C" {

int cil_pointnet_num_params(void) { return kNParams; }

cil_status cil_pointnet_create(int max_pairs, int n_points, cil_pointnet** out) {
  if (!out || max_pairs < 1 || n_points < kTileP || n_points % kTileP) return CIL_ERR_INVALID_ARG;
  cil_status st = CIL_OK;
  DeviceCtx* ctx = device_ctx(&st);
  if (!ctx) return st;
  if (cudaFuncSetAttribute(k_pn_encode_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)enc_tc_smem()) != cudaSuccess ||
      cudaFuncSetAttribute(k_pn_encode_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)enc_bwd_smem()) != cudaSuccess)
    return CIL_ERR_CUDA;
  cil_pointnet* h = new cil_pointnet();
  h->ctx = ctx;
  PnState& S = h->s;
  S.max_pairs = max_pairs;
  S.P = n_points;
  S.step = 0;
  const int B = max_pairs;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = (off + 255) & ~size_t(255);
    off = o + bytes;
    return o;
  };
  const size_t oP = take(4 * kNParams), oG = take(4 * kNParams), oM = take(4 * kNParams),
               oV = take(4 * kNParams), oW2b = take(2 * kH2 * kH1), oW3b = take(2 * kH3 * kH2),
               oW4t = take(4 * kH4 * 2 * kH3), oFK = take(8 * (size_t)2 * B * kH3),
               oH = take(4 * (size_t)B * 2 * kH3), oZ4 = take(4 * (size_t)B * kH4),
               oO = take(4 * (size_t)B * kOut), oDZ4 = take(4 * (size_t)B * kH4),
               oDO = take(4 * (size_t)B * kOut), oDF = take(4 * (size_t)2 * B * kH3),
               oL = take(4 * (size_t)B), oPart = take(4 * (size_t)2 * B * kEncParams);
  if (cudaMalloc(&S.base, off) != cudaSuccess) {
    delete h;
    return CIL_ERR_NOMEM;
  }
  char* base = static_cast<char*>(S.base);
  S.params = reinterpret_cast<float*>(base + oP);
  S.grad = reinterpret_cast<float*>(base + oG);
  S.m = reinterpret_cast<float*>(base + oM);
  S.v = reinterpret_cast<float*>(base + oV);
  S.w2b = reinterpret_cast<__nv_bfloat16*>(base + oW2b);
  S.w3b = reinterpret_cast<__nv_bfloat16*>(base + oW3b);
  S.w4t = reinterpret_cast<float*>(base + oW4t);
  S.feat_key = reinterpret_cast<u64*>(base + oFK);
  S.h = reinterpret_cast<float*>(base + oH);
  S.z4 = reinterpret_cast<float*>(base + oZ4);
  S.o = reinterpret_cast<float*>(base + oO);
  S.dz4 = reinterpret_cast<float*>(base + oDZ4);
  S.dout = reinterpret_cast<float*>(base + oDO);
  S.df = reinterpret_cast<float*>(base + oDF);
  S.loss = reinterpret_cast<float*>(base + oL);
  S.enc_part = reinterpret_cast<float*>(base + oPart);
  if (cudaMemset(S.base, 0, off) != cudaSuccess) {
    cudaFree(S.base);
    delete h;
    return CIL_ERR_CUDA;
  }
  *out = h;
  return CIL_OK;
}

void cil_pointnet_destroy(cil_pointnet* h) {
  if (!h) return;
  cudaDeviceSynchronize();
  cudaFree(h->s.base);
  delete h;
}

cil_status cil_pointnet_set_params(cil_pointnet* h, const float* params, void* stream) {
  if (!h || !params) return CIL_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  PnState& S = h->s;
  if (cudaMemcpyAsync(S.params, params, 4 * kNParams, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
      cudaMemsetAsync(S.m, 0, 4 * kNParams, s) != cudaSuccess ||
      cudaMemsetAsync(S.v, 0, 4 * kNParams, s) != cudaSuccess)
    return CIL_ERR_CUDA;
  S.step = 0;
  note_launches(1);
  k_pn_refresh<<<ceil_div(kH4 * 2 * kH3, 256), 256, 0, s>>>(S.params, S.w2b, S.w3b, S.w4t);
  return cudaGetLastError() == cudaSuccess ? CIL_OK : CIL_ERR_CUDA;
}

cil_status cil_pointnet_get_params(cil_pointnet* h, float* params, void* stream) {
  if (!h || !params) return CIL_ERR_INVALID_ARG;
  return cudaMemcpyAsync(params, h->s.params, 4 * kNParams, cudaMemcpyDeviceToDevice,
                         (cudaStream_t)stream) == cudaSuccess
             ? CIL_OK
             : CIL_ERR_CUDA;
}

cil_status cil_pointnet_forward(cil_pointnet* h, const float* clouds, int B, double* T_out,
                                float* feat_out, void* stream) {
  if (!h || !clouds || B < 1 || B > h->s.max_pairs) return CIL_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  cil_status st = pn_forward_enqueue(h, clouds, B, T_out, s);
  if (st != CIL_OK) return st;
  if (feat_out &&
      cudaMemcpyAsync(feat_out, h->s.h, 4 * (size_t)B * 2 * kH3, cudaMemcpyDeviceToDevice, s) !=
          cudaSuccess)
    return CIL_ERR_CUDA;
  return CIL_OK;
}

cil_status cil_pointnet_backward(cil_pointnet* h, const float* clouds, const double* T_gt, int B,
                                 float* loss_out, float* grad_out, void* stream) {
  if (!h || !clouds || !T_gt || B < 1 || B > h->s.max_pairs) return CIL_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  PnState& S = h->s;
  cil_status st = pn_forward_enqueue(h, clouds, B, nullptr, s);
  if (st != CIL_OK) return st;
  note_launches(4);
  k_pn_loss_head_bwd<<<B, 256, 0, s>>>(S.params, clouds, S.P, B, T_gt, S.z4, S.o, S.loss, S.dz4,
                                       S.dout, S.df);
  const int nh = kH4 * 2 * kH3 + kH4 + kOut * kH4 + kOut;
  k_pn_head_wgrad<<<ceil_div(nh, 256), 256, 0, s>>>(S.h, S.z4, S.dz4, S.dout, B, S.grad);
  {
    TimedRegion timer("k_pn_encode_bwd", s);
    k_pn_encode_bwd<<<2 * B, 256, enc_bwd_smem(), s>>>(clouds, S.P, S.params, S.w2b, S.w3b,
                                                       S.feat_key, S.df, S.enc_part);
  }
  k_pn_enc_reduce<<<ceil_div(kEncParams, 256), 256, 0, s>>>(S.enc_part, 2 * B, S.grad);
  if (loss_out &&
      cudaMemcpyAsync(loss_out, S.loss, 4 * (size_t)B, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return CIL_ERR_CUDA;
  if (grad_out &&
      cudaMemcpyAsync(grad_out, S.grad, 4 * (size_t)kNParams, cudaMemcpyDeviceToDevice, s) !=
          cudaSuccess)
    return CIL_ERR_CUDA;
  return cudaGetLastError() == cudaSuccess ? CIL_OK : CIL_ERR_CUDA;
}

cil_status cil_pointnet_adam_step(cil_pointnet* h, float lr, void* stream) {
  if (!h || !(lr >= 0.0f)) return CIL_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  PnState& S = h->s;
  S.step += 1;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float c1 = 1.0f - powf(b1, (float)S.step), c2 = 1.0f - powf(b2, (float)S.step);
  note_launches(2);
  k_pn_adam<<<ceil_div(kNParams, 256), 256, 0, s>>>(S.params, S.grad, S.m, S.v, lr, b1, b2, eps, c1,
                                                    c2);
  k_pn_refresh<<<ceil_div(kH4 * 2 * kH3, 256), 256, 0, s>>>(S.params, S.w2b, S.w3b, S.w4t);
  return cudaGetLastError() == cudaSuccess ? CIL_OK : CIL_ERR_CUDA;
}

}  // extern "C"
