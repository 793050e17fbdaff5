// capi.cu -- the exported C ABI (include/cil.h): argument checks, per-device
// context, stream-ordered workspaces and the enqueue sequences of each call.
#include <atomic>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "cil_host.h"
#include "cil_kernels.h"

namespace cil {

// ---------------------------------------------------------------------------
// device context
// ---------------------------------------------------------------------------
static std::mutex g_ctx_mu;
static DeviceCtx g_ctx[64];

DeviceCtx* device_ctx(cil_status* st) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    *st = CIL_ERR_CUDA;
    return nullptr;
  }
  std::lock_guard<std::mutex> lk(g_ctx_mu);
  DeviceCtx& c = g_ctx[dev];
  if (c.device == dev) return &c;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    *st = CIL_ERR_CUDA;
    return nullptr;
  }
  int* err = nullptr;
  if (cudaMalloc(&err, sizeof(int)) != cudaSuccess) {
    *st = CIL_ERR_NOMEM;
    return nullptr;
  }
  if (cudaMemset(err, 0, sizeof(int)) != cudaSuccess) {
    *st = CIL_ERR_CUDA;
    return nullptr;
  }
  cudaMemPoolProps props = {};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  cudaMemPool_t pool = nullptr;
  if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
    *st = CIL_ERR_CUDA;
    return nullptr;
  }
  uint64_t keep = ~0ull;  // keep freed blocks cached in the pool
  cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  c.num_sms = sms;
  c.err = err;
  c.pool = pool;
  c.device = dev;
  return &c;
}

// allocations left to fail (cil_test_fail_next_allocations)
static std::atomic<int> g_fail_allocs{0};

cil_status Workspace::allocate(DeviceCtx* ctx, cudaStream_t s) {
  stream_ = s;
  if (total_ == 0) total_ = 256;
  for (int f = g_fail_allocs.load(); f > 0; f = g_fail_allocs.load())
    if (g_fail_allocs.compare_exchange_weak(f, f - 1)) return CIL_ERR_NOMEM;
  if (cudaMallocFromPoolAsync(reinterpret_cast<void**>(&base_), total_, ctx->pool, s) !=
      cudaSuccess) {
    base_ = nullptr;
    cudaGetLastError();
    return CIL_ERR_NOMEM;
  }
  return CIL_OK;
}

void Workspace::release(cudaStream_t s) {
  if (base_) cudaFreeAsync(base_, s);
  base_ = nullptr;
}

Workspace::~Workspace() {
  if (base_) cudaFreeAsync(base_, stream_);
}

// ---------------------------------------------------------------------------
// instrumentation
// ---------------------------------------------------------------------------
static std::atomic<long long> g_launches{0};
static std::atomic<int> g_timing{0};
static std::mutex g_timing_mu;
struct TimedRecord {
  std::string name;
  cudaEvent_t a, b;
};
static std::vector<TimedRecord> g_records;

void note_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

TimedRegion::TimedRegion(const char* name, cudaStream_t s) : name_(name), s_(s) {
  if (!g_timing.load(std::memory_order_relaxed)) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
  cudaEvent_t* ev = new cudaEvent_t[2];
  if (cudaEventCreate(&ev[0]) != cudaSuccess || cudaEventCreate(&ev[1]) != cudaSuccess) {
    delete[] ev;
    return;
  }
  cudaEventRecord(ev[0], s);
  ev_ = ev;
}

TimedRegion::~TimedRegion() {
  if (!ev_) return;
  cudaEvent_t* ev = static_cast<cudaEvent_t*>(ev_);
  cudaEventRecord(ev[1], s_);
  std::lock_guard<std::mutex> lk(g_timing_mu);
  g_records.push_back({name_, ev[0], ev[1]});
  delete[] ev;
}

static cil_status read_error_word(DeviceCtx* ctx, cudaStream_t s, bool clear) {
  int v = 0;
  if (cudaMemcpyAsync(&v, ctx->err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return CIL_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return CIL_ERR_CUDA;
  if (v != 0 && clear) {
    if (cudaMemsetAsync(ctx->err, 0, sizeof(int), s) != cudaSuccess) return CIL_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return CIL_ERR_CUDA;
  }
  return (cil_status)v;
}

static bool bad_count(int64_t n) { return n < 0 || n > (int64_t)0x7fffffff; }

static GridOptions grid_options(const cil_params* prm, int k) {
  GridOptions o;
  o.k_est = k;
  if (prm) {
    o.cell_size = prm->cell_size > 0.0f ? prm->cell_size : 0.0f;
    o.cell_scale = prm->cell_scale > 0.0f ? prm->cell_scale : kDefaultCellScale;
  }
  return o;
}

static int block_of(const cil_params* prm) { return prm && prm->block ? prm->block : 128; }
static int topk_of(const cil_params* prm) {
  return prm && prm->topk >= 0 && prm->topk <= 3 ? prm->topk : 0;
}

}  // namespace cil

using namespace cil;

extern "C" {

const char* cil_status_string(cil_status s) {
  switch (s) {
    case CIL_OK: return "CIL_OK";
    case CIL_ERR_INVALID_ARG: return "CIL_ERR_INVALID_ARG";
    case CIL_ERR_CUDA: return "CIL_ERR_CUDA";
    case CIL_ERR_NONFINITE: return "CIL_ERR_NONFINITE";
    case CIL_ERR_CAPACITY: return "CIL_ERR_CAPACITY";
    case CIL_ERR_DEGENERATE: return "CIL_ERR_DEGENERATE";
    case CIL_ERR_TIMEOUT: return "CIL_ERR_TIMEOUT";
    case CIL_ERR_NOMEM: return "CIL_ERR_NOMEM";
  }
  return "CIL_ERR_UNKNOWN";
}

void cil_timing_enable(int on) { g_timing.store(on ? 1 : 0); }

int64_t cil_launch_count(void) { return g_launches.load(); }

void cil_test_fail_next_allocations(int count) { g_fail_allocs.store(count > 0 ? count : 0); }

cil_status cil_check_bounded_wait(unsigned polls, void* stream) {
  cil_status st = CIL_OK;
  DeviceCtx* ctx = device_ctx(&st);
  if (!ctx) return st;
  cudaStream_t s = (cudaStream_t)stream;
  if ((st = launch_bounded_wait_check(polls, ctx->err, s)) != CIL_OK) return st;
  return read_error_word(ctx, s, true);
}

cil_status cil_timing_read(const char* name, double* total_ms, int64_t* launches) {
  if (!name || !total_ms || !launches) return CIL_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_timing_mu);
  double tot = 0.0;
  int64_t cnt = 0;
  for (auto& r : g_records) {
    if (r.name != name) continue;
    if (cudaEventSynchronize(r.b) != cudaSuccess) return CIL_ERR_CUDA;
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) return CIL_ERR_CUDA;
    tot += ms;
    ++cnt;
  }
  *total_ms = tot;
  *launches = cnt;
  return CIL_OK;
}

void cil_timing_reset(void) {
  std::lock_guard<std::mutex> lk(g_timing_mu);
  for (auto& r : g_records) {
    cudaEventSynchronize(r.b);
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  g_records.clear();
}

cil_status cil_sync_status(void* stream) {
  cil_status st = CIL_OK;
  DeviceCtx* ctx = device_ctx(&st);
  if (!ctx) return st;
  return read_error_word(ctx, (cudaStream_t)stream, true);
}

cil_status cil_knn_ex(const float* ref, int64_t n_ref, const float* qry, int64_t n_qry, int k,
                      int32_t* out_idx, float* out_d2, const cil_params* params, void* stream) {
  if (k < 1 || k > CIL_MAX_K || bad_count(n_ref) || bad_count(n_qry)) return CIL_ERR_INVALID_ARG;
  if (n_qry == 0) return CIL_OK;
  if (!qry || !out_idx || (n_ref > 0 && !ref)) return CIL_ERR_INVALID_ARG;
  cil_status st = CIL_OK;
  DeviceCtx* ctx = device_ctx(&st);
  if (!ctx) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const bool self = (qry == ref && n_qry == n_ref);
  Workspace ws;
  GridPlan gp;
  grid_plan(gp, ws, n_ref, 1);
  OrderPlan op;
  size_t o_order = 0;
  if (!self) {
    order_plan(op, ws, n_qry);
    o_order = ws.reserve(sizeof(int) * (size_t)n_qry);
  }
  if ((st = ws.allocate(ctx, s)) != CIL_OK) return st;
  if ((st = grid_build(gp, ws, ref, nullptr, grid_options(params, k), ctx, s)) != CIL_OK) return st;
  const GridView g = grid_view(gp, ws);
  int* order = nullptr;
  if (!self) {
    order = ws.at<int>(o_order);
    if ((st = order_queries(op, ws, qry, nullptr, 1, g.prm, nullptr, order, s)) != CIL_OK) return st;
  }
  st = launch_knn(g, qry, n_qry, order, k, out_idx, out_d2, block_of(params), s, topk_of(params));
  ws.release(s);
  return st;
}

cil_status cil_knn(const float* ref, int64_t n_ref, const float* qry, int64_t n_qry, int k,
                   int32_t* out_idx, float* out_d2, void* stream) {
  return cil_knn_ex(ref, n_ref, qry, n_qry, k, out_idx, out_d2, nullptr, stream);
}

cil_status cil_estimate_normals_ex(const float* xyz, int64_t n, int k, const float* viewpoint,
                                   float* out_normals, float* out_curvature,
                                   const cil_params* params, void* stream) {
  if (k < 1 || k > CIL_MAX_K || bad_count(n) || !viewpoint) return CIL_ERR_INVALID_ARG;
  if (n == 0) return CIL_OK;
  if (!xyz || !out_normals) return CIL_ERR_INVALID_ARG;
  cil_status st = CIL_OK;
  DeviceCtx* ctx = device_ctx(&st);
  if (!ctx) return st;
  cudaStream_t s = (cudaStream_t)stream;
  Workspace ws;
  GridPlan gp;
  grid_plan(gp, ws, n, 1);
  if ((st = ws.allocate(ctx, s)) != CIL_OK) return st;
  if ((st = grid_build(gp, ws, xyz, nullptr, grid_options(params, k), ctx, s)) != CIL_OK) return st;
  st = launch_normals(grid_view(gp, ws), 1, n, k, nullptr, viewpoint, xyz, out_normals,
                      out_curvature, block_of(params), s, nullptr, topk_of(params));
  ws.release(s);
  return st;
}

cil_status cil_estimate_normals(const float* xyz, int64_t n, int k, const float* viewpoint,
                                float* out_normals, float* out_curvature, void* stream) {
  return cil_estimate_normals_ex(xyz, n, k, viewpoint, out_normals, out_curvature, nullptr, stream);
}

cil_status cil_knn_hybrid(const float* ref, int64_t n_ref, const float* qry, int64_t n_qry, int k,
                          float r, int32_t* out_idx, float* out_d2, void* stream) {
  if (k < 1 || k > CIL_MAX_K || bad_count(n_ref) || bad_count(n_qry) || !(r >= 0.0f) ||
      !isfinite(r))
    return CIL_ERR_INVALID_ARG;
  if (n_qry == 0) return CIL_OK;
  if (!qry || !out_idx || (n_ref > 0 && !ref)) return CIL_ERR_INVALID_ARG;
  cil_status st = CIL_OK;
  DeviceCtx* ctx = device_ctx(&st);
  if (!ctx) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const bool self = (qry == ref && n_qry == n_ref);
  Workspace ws;
  GridPlan gp;
  grid_plan(gp, ws, n_ref, 1);
  OrderPlan op;
  size_t o_order = 0;
  if (!self) {
    order_plan(op, ws, n_qry);
    o_order = ws.reserve(sizeof(int) * (size_t)n_qry);
  }
  if ((st = ws.allocate(ctx, s)) != CIL_OK) return st;
  if ((st = grid_build(gp, ws, ref, nullptr, grid_options(nullptr, k), ctx, s)) != CIL_OK) return st;
  const GridView g = grid_view(gp, ws);
  int* order = nullptr;
  if (!self) {
    order = ws.at<int>(o_order);
    if ((st = order_queries(op, ws, qry, nullptr, 1, g.prm, nullptr, order, s)) != CIL_OK) return st;
  }
  st = launch_knn_hybrid(g, qry, n_qry, order, k, r, out_idx, out_d2, s);
  ws.release(s);
  return st;
}

cil_status cil_estimate_normals_radius(const float* xyz, int64_t n, float r, const float* viewpoint,
                                       float* out_normals, float* out_curvature,
                                       int32_t* out_counts, void* stream) {
  if (bad_count(n) || !viewpoint || !(r > 0.0f) || !isfinite(r)) return CIL_ERR_INVALID_ARG;
  if (n == 0) return CIL_OK;
  if (!xyz || !out_normals) return CIL_ERR_INVALID_ARG;
  cil_status st = CIL_OK;
  DeviceCtx* ctx = device_ctx(&st);
  if (!ctx) return st;
  cudaStream_t s = (cudaStream_t)stream;
  Workspace ws;
  GridPlan gp;
  grid_plan(gp, ws, n, 1);
  if ((st = ws.allocate(ctx, s)) != CIL_OK) return st;
  GridOptions opt;
  opt.k_est = 10;
  opt.cell_size = r;
  if ((st = grid_build(gp, ws, xyz, nullptr, opt, ctx, s)) != CIL_OK) return st;
  st = launch_normals_radius(grid_view(gp, ws), n, r, viewpoint, out_normals, out_curvature,
                             out_counts, s);
  ws.release(s);
  return st;
}

// Shared body of cil_icp and cil_icp_sums (sums_out: host, or null).
static cil_status icp_impl(const float* src, int64_t n_src, const float* dst,
                           const float* dst_normals, int64_t n_dst, const double* T_init,
                           int max_iters, float max_corr_dist, const cil_icp_options* opt,
                           double* T_out, cil_icp_report* rep, double* sums_out, void* stream) {
  IcpOptions o;
  if (opt) {
    if (opt->metric < CIL_METRIC_POINT_TO_PLANE || opt->metric > CIL_METRIC_COMBINED ||
        opt->association < CIL_ASSOC_NEAREST || opt->association > CIL_ASSOC_PROJECTIVE)
      return CIL_ERR_INVALID_ARG;
    o.metric = opt->metric;
    o.association = opt->association;
    if (o.metric == CIL_METRIC_COMBINED) {
      if (!(opt->w_point >= 0.0f && opt->w_point < INFINITY && opt->w_plane >= 0.0f &&
            opt->w_plane < INFINITY))
        return CIL_ERR_INVALID_ARG;
      o.w_point = opt->w_point;
      o.w_plane = opt->w_plane;
    }
    if (o.association == CIL_ASSOC_PROJECTIVE) {
      if (!opt->pixel_map || opt->width <= 0 || opt->height <= 0 ||
          !(fabsf(opt->fx) < INFINITY && fabsf(opt->fy) < INFINITY && fabsf(opt->cx) < INFINITY &&
            fabsf(opt->cy) < INFINITY))
        return CIL_ERR_INVALID_ARG;
      o.pixel_map = opt->pixel_map;
      o.width = opt->width;
      o.height = opt->height;
      o.fx = opt->fx;
      o.fy = opt->fy;
      o.cx = opt->cx;
      o.cy = opt->cy;
    }
  }
  const bool need_normals = o.metric != CIL_METRIC_POINT_TO_POINT;
  if (bad_count(n_src) || bad_count(n_dst) || max_iters < 0 || !(max_corr_dist >= 0.0f) || !T_out ||
      !rep)
    return CIL_ERR_INVALID_ARG;
  if ((n_src > 0 && !src) || (n_dst > 0 && (!dst || (need_normals && !dst_normals))))
    return CIL_ERR_INVALID_ARG;
  cil_status st = CIL_OK;
  DeviceCtx* ctx = device_ctx(&st);
  if (!ctx) return st;
  cudaStream_t s = (cudaStream_t)stream;
  Workspace ws;
  GridPlan gp;
  grid_plan(gp, ws, n_dst, 1);
  IcpPlan ip;
  const int64_t counts[1] = {n_src};
  icp_plan(ip, ws, counts, 1);
  const size_t o_out = ws.reserve(sizeof(double) * 16 + sizeof(cil_icp_report));
  const size_t n_sums = (size_t)(max_iters + 1) * (kIcpQ + 1);
  const size_t o_sums = sums_out ? ws.reserve(sizeof(double) * n_sums) : 0;
  if ((st = ws.allocate(ctx, s)) != CIL_OK) return st;
  if (sums_out) {
    o.sums = ws.at<double>(o_sums);
    if (cudaMemsetAsync(o.sums, 0, sizeof(double) * n_sums, s) != cudaSuccess) return CIL_ERR_CUDA;
  }
  GridOptions gopt = grid_options(nullptr, 10);
  if ((st = grid_build(gp, ws, dst, nullptr, gopt, ctx, s)) != CIL_OK) return st;
  if ((st = icp_run(ip, ws, grid_view(gp, ws), src, nullptr, dst, need_normals ? dst_normals : nullptr,
                    nullptr, T_init, max_iters, nullptr, max_corr_dist, ctx, s, &o)) != CIL_OK)
    return st;
  double* Td = ws.at<double>(o_out);
  cil_icp_report* rd = reinterpret_cast<cil_icp_report*>(Td + 16);
  if ((st = icp_export(ip, ws, Td, rd, s)) != CIL_OK) return st;
  struct {
    double T[16];
    cil_icp_report r;
  } h;
  if (cudaMemcpyAsync(&h, Td, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess) return CIL_ERR_CUDA;
  if (sums_out && cudaMemcpyAsync(sums_out, o.sums, sizeof(double) * n_sums,
                                  cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return CIL_ERR_CUDA;
  ws.release(s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return CIL_ERR_CUDA;
  for (int j = 0; j < 16; ++j) T_out[j] = h.T[j];
  *rep = h.r;
  cil_status dev = read_error_word(ctx, s, true);
  if (dev != CIL_OK) return dev;
  return CIL_OK;
}

cil_status cil_icp(const float* src, int64_t n_src, const float* dst, const float* dst_normals,
                   int64_t n_dst, const double* T_init, int max_iters, float max_corr_dist,
                   const cil_icp_options* opt, double* T_out, cil_icp_report* rep, void* stream) {
  return icp_impl(src, n_src, dst, dst_normals, n_dst, T_init, max_iters, max_corr_dist, opt,
                  T_out, rep, nullptr, stream);
}

cil_status cil_icp_sums(const float* src, int64_t n_src, const float* dst,
                        const float* dst_normals, int64_t n_dst, const double* T_init,
                        int max_iters, float max_corr_dist, const cil_icp_options* opt,
                        double* T_out, cil_icp_report* rep, double* sums_out, void* stream) {
  if (!sums_out) return CIL_ERR_INVALID_ARG;
  return icp_impl(src, n_src, dst, dst_normals, n_dst, T_init, max_iters, max_corr_dist, opt,
                  T_out, rep, sums_out, stream);
}

// Shared body of cil_segment (normals given) and cil_smooth_segment (normals
// computed here from the same k-NN lists that define the graph: one search).
static cil_status segment_impl(const float* xyz, const float* normals_in, const float* viewpoint,
                               int64_t n, int k, float theta, float radius, float* out_normals,
                               int32_t* out_labels, int64_t* out_count, void* stream) {
  if (k < 1 || k > CIL_MAX_K || bad_count(n) || !out_count || !(theta >= 0.0f) ||
      !(theta < INFINITY) || !(radius >= 0.0f) || !(radius < INFINITY))
    return CIL_ERR_INVALID_ARG;
  *out_count = 0;
  if (n == 0) return CIL_OK;
  if (!xyz || (!normals_in && !viewpoint) || !out_labels) return CIL_ERR_INVALID_ARG;
  cil_status st = CIL_OK;
  DeviceCtx* ctx = device_ctx(&st);
  if (!ctx) return st;
  cudaStream_t s = (cudaStream_t)stream;
  Workspace ws;
  GridPlan gp;
  grid_plan(gp, ws, n, 1);
  const size_t o_idx = ws.reserve(sizeof(int) * (size_t)n * (size_t)k);
  const size_t o_parent = ws.reserve(sizeof(int) * (size_t)n);
  const size_t o_count = ws.reserve(sizeof(unsigned long long));
  const bool own_normals = !normals_in && !out_normals;
  const size_t o_nrm = own_normals ? ws.reserve(sizeof(float) * 3 * (size_t)n) : 0;
  if ((st = ws.allocate(ctx, s)) != CIL_OK) return st;
  if ((st = grid_build(gp, ws, xyz, nullptr, grid_options(nullptr, k), ctx, s)) != CIL_OK) return st;
  int* idx = ws.at<int>(o_idx);
  const float* nrm = normals_in;
  if (normals_in) {
    st = launch_knn(grid_view(gp, ws), xyz, n, nullptr, k, idx, nullptr, block_of(nullptr), s);
  } else {
    float* nout = own_normals ? ws.at<float>(o_nrm) : out_normals;
    st = launch_normals(grid_view(gp, ws), 1, n, k, nullptr, viewpoint, xyz, nout, nullptr,
                        block_of(nullptr), s, idx);
    nrm = nout;
  }
  if (st != CIL_OK) return st;
  // the thresholds as FP32 values, the same rounding the oracle applies
  const float cos_t = (float)cos((double)theta);
  const float r2 = radius > 0.0f ? (float)((double)radius * (double)radius) : 0.0f;
  unsigned long long* count = ws.at<unsigned long long>(o_count);
  if ((st = launch_segment(idx, k, xyz, nrm, n, grid_view(gp, ws).pts, cos_t, r2,
                           ws.at<int>(o_parent), out_labels, count, ctx->err, s)) != CIL_OK)
    return st;
  unsigned long long c = 0;
  if (cudaMemcpyAsync(&c, count, sizeof(c), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return CIL_ERR_CUDA;
  ws.release(s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return CIL_ERR_CUDA;
  *out_count = (int64_t)c;
  return read_error_word(ctx, s, true);
}

cil_status cil_segment(const float* xyz, const float* normals, int64_t n, int k, float theta,
                       float radius, int32_t* out_labels, int64_t* out_count, void* stream) {
  if (n > 0 && !normals) return CIL_ERR_INVALID_ARG;
  return segment_impl(xyz, normals, nullptr, n, k, theta, radius, nullptr, out_labels, out_count,
                      stream);
}

cil_status cil_smooth_segment(const float* xyz, int64_t n, int k, const float* viewpoint,
                              float theta, float radius, float* out_normals, int32_t* out_labels,
                              int64_t* out_count, void* stream) {
  if (!viewpoint) return CIL_ERR_INVALID_ARG;
  return segment_impl(xyz, nullptr, viewpoint, n, k, theta, radius, out_normals, out_labels,
                      out_count, stream);
}

cil_status cil_icp_point_to_plane(const float* src, int64_t n_src, const float* dst,
                                  const float* dst_normals, int64_t n_dst, const double* T_init,
                                  int max_iters, float max_corr_dist, double* T_out,
                                  cil_icp_report* rep, void* stream) {
  if (n_dst > 0 && !dst_normals) return CIL_ERR_INVALID_ARG;
  return cil_icp(src, n_src, dst, dst_normals, n_dst, T_init, max_iters, max_corr_dist, nullptr,
                 T_out, rep, stream);
}

cil_status cil_register_pair(const float* src, int64_t n_src, const float* dst, int64_t n_dst, int k,
                             const float* viewpoint, const double* T_init, int max_iters,
                             float max_corr_dist, float* out_normals, double* T_out,
                             cil_icp_report* rep, const cil_params* params, void* stream) {
  if (bad_count(n_src) || bad_count(n_dst) || k < 1 || k > CIL_MAX_K || max_iters < 0 ||
      !(max_corr_dist >= 0.0f) || !viewpoint || !T_out || !rep)
    return CIL_ERR_INVALID_ARG;
  if ((n_src > 0 && !src) || (n_dst > 0 && !dst)) return CIL_ERR_INVALID_ARG;
  cil_status st = CIL_OK;
  DeviceCtx* ctx = device_ctx(&st);
  if (!ctx) return st;
  cudaStream_t s = (cudaStream_t)stream;
  Workspace ws;
  GridPlan gp;
  grid_plan(gp, ws, n_dst, 1);
  IcpPlan ip;
  const int64_t counts[1] = {n_src};
  icp_plan(ip, ws, counts, 1);
  size_t o_nrm = 0;
  if (!out_normals) o_nrm = ws.reserve(sizeof(float) * 3 * (size_t)(n_dst > 0 ? n_dst : 1));
  if ((st = ws.allocate(ctx, s)) != CIL_OK) return st;
  float* nrm = out_normals ? out_normals : ws.at<float>(o_nrm);
  GridOptions gopt = grid_options(params, k);
  if ((st = grid_build(gp, ws, dst, nullptr, gopt, ctx, s)) != CIL_OK) return st;
  const GridView g = grid_view(gp, ws);
  if ((st = launch_normals(g, 1, n_dst, k, nullptr, viewpoint, dst, nrm, nullptr, block_of(params),
                           s, nullptr, topk_of(params))) != CIL_OK)
    return st;
  if ((st = icp_run(ip, ws, g, src, nullptr, dst, nrm, T_init, nullptr, max_iters, nullptr, max_corr_dist,
                    ctx, s)) != CIL_OK)
    return st;
  st = icp_export(ip, ws, T_out, rep, s);
  ws.release(s);
  return st;
}

}  // extern "C"
