// cil_host.h -- host-side internals shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/cil.h"
#include "cil_dev.cuh"

namespace cil {

// ---------------------------------------------------------------------------
// per-device context
// ---------------------------------------------------------------------------
struct DeviceCtx {
  int device = -1;
  int num_sms = 0;
  int* err = nullptr;  // device error word (cil_status value, 0 = clean)
  cudaMemPool_t pool = nullptr;
};

// Context of the current device (created on first use).  Returns nullptr and
// sets *st on failure.
DeviceCtx* device_ctx(cil_status* st);

// ---------------------------------------------------------------------------
// stream-ordered workspace: one allocation carved into 256-byte aligned parts
// ---------------------------------------------------------------------------
class Workspace {
 public:
  // reserve `bytes` and return the offset of the part
  size_t reserve(size_t bytes) {
    size_t off = (total_ + 255) & ~size_t(255);
    total_ = off + bytes;
    return off;
  }
  cil_status allocate(DeviceCtx* ctx, cudaStream_t s);
  template <typename T>
  T* at(size_t off) const {
    return reinterpret_cast<T*>(base_ + off);
  }
  void release(cudaStream_t s);
  ~Workspace();
  // bytes reserved so far
  size_t total() const { return total_; }
  // use caller-provided device memory instead of allocating; detach() must
  // run before release() or destruction so that nothing tries to free it
  void attach(void* base) { base_ = static_cast<char*>(base); }
  void detach() { base_ = nullptr; }

 private:
  char* base_ = nullptr;
  size_t total_ = 0;
  cudaStream_t stream_ = nullptr;
};

// ---------------------------------------------------------------------------
// grid build over B concatenated clouds
// ---------------------------------------------------------------------------
struct GridPlan {
  int64_t n = 0;        // total points
  int clouds = 1;
  unsigned mask = 0;    // table size - 1
  int radix_blocks = 0;
  // workspace offsets
  size_t o_prm, o_pts, o_tab, o_keys0, o_keys1, o_vals0, o_vals1, o_counts, o_scan, o_starts;
  size_t o_est;         // sampled neighbour distances of the level choice (1024 per cloud)
};

// Default multiplier on the data-driven cell edge (the median k-th neighbour
// distance of sampled points).  The level is that edge rounded to a power of
// two of the fine lattice; 1.5 was faster than 1.0 on the depth-frame,
// wavy-surface and LiDAR workloads (whole registration: 4.30 vs 4.64,
// 1.64 vs 1.72 and 3.35 vs 3.34 ms).
constexpr float kDefaultCellScale = 1.5f;

struct GridOptions {
  int k_est = 10;          // neighbourhood size the level is tuned for
  float cell_size = 0.0f;  // > 0: requested cell edge
  float cell_scale = kDefaultCellScale;  // multiplier on the data-driven size
};

// Reserve the workspace parts of a grid over `n` points in `clouds` clouds.
void grid_plan(GridPlan& p, Workspace& ws, int64_t n, int clouds);

// Enqueue the build.  `xyz` holds the concatenated clouds; `cloud_start_dev`
// (device, clouds+1 int32) their offsets (may be null when clouds == 1).
// `cloud_k_dev` (device, per-cloud neighbourhood size for the level choice)
// may be null (then opt.k_est is used).
cil_status grid_build(const GridPlan& p, const Workspace& ws, const float* xyz,
                      const int* cloud_start_dev, const GridOptions& opt, DeviceCtx* ctx,
                      cudaStream_t s);

GridView grid_view(const GridPlan& p, const Workspace& ws);

// Stable order of query points by the Morton code of their fine cell in the
// reference grid (after an optional rigid transform given per cloud as
// float[12] R|t rows on the device).  Writes `order` (global query indices).
struct OrderPlan {
  int64_t n = 0;
  int radix_blocks = 0;
  size_t o_keys0, o_keys1, o_vals0, o_vals1, o_counts, o_scan;
};
void order_plan(OrderPlan& p, Workspace& ws, int64_t n);
cil_status order_queries(const OrderPlan& p, const Workspace& ws, const float* qry,
                         const int* q_cloud_start_dev, int clouds, const GridParams* ref_prm,
                         const float* Rt_dev, int* order_out, cudaStream_t s);

// exclusive scan of int data[L] in place, `tmp` must hold scan_tmp_ints(L)
size_t scan_tmp_ints(int64_t L);
void scan_exclusive(int* data, int64_t L, int* tmp, cudaStream_t s);
void scan_exclusive_i64(long long* data, int64_t L, long long* tmp, cudaStream_t s);

int ceil_div(int64_t a, int64_t b);

// ---------------------------------------------------------------------------
// instrumentation: count of kernel launches and optional per-kernel CUDA-event
// timing on the launching stream (used by benchmarks and profiling)
// ---------------------------------------------------------------------------
void note_launches(int n);
struct TimedRegion {
  TimedRegion(const char* name, cudaStream_t s);
  ~TimedRegion();
  const char* name_;
  cudaStream_t s_;
  void* ev_ = nullptr;  // opaque pair of events when timing is on
};
unsigned next_pow2_u32(uint64_t v);

// stable LSD radix sort of (u64 key, int value) pairs on the low `bits` key
// bits, in the buffers reserved by radix_sort_plan (keys0/vals0 hold the input);
// returns which buffer pair (0 or 1) holds the result
struct RadixPlan {
  int64_t n = 0;
  int blocks = 0;
  size_t o_keys0, o_keys1, o_vals0, o_vals1, o_counts, o_scan;
};
void radix_sort_plan(RadixPlan& p, Workspace& ws, int64_t n);
int radix_sort_pairs(const RadixPlan& p, const Workspace& ws, int bits, cudaStream_t s);

}  // namespace cil
