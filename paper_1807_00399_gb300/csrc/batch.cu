// batch.cu -- registration of many independent cloud pairs in one graph launch.
//
// A cil_batch handle owns a device workspace sized for its pair sizes.  A run
// enqueues, for all B pairs at once:
//   grid build over the concatenated targets (cloud id above the Morton bits,
//   one search level per cloud), k-NN PCA normals of every target point, and
//   the ICP rounds of every pair (three launches per round over all pairs'
//   tiles, see icp.cu) with the final RMSE pass.
// The sequence is captured once per set of buffer pointers into a CUDA graph
// and replayed with a single cudaGraphLaunch on the caller's stream.
//
// Fallback after a warm-started run (the learned warm start keeps plain ICP
// from the identity as its fallback): the pairs whose final RMSE is at or
// above a threshold (or undefined) are marked on the device, re-registered
// from the identity over the same target grid and normals (only their tiles
// are launched), and each keeps the better of its two results.
#include <stdlib.h>

#include <vector>

#include "cil_host.h"
#include "cil_kernels.h"

namespace cil {

struct BatchHandle {
  int B = 0;
  int device = -1;
  cil_batch_params prm;
  std::vector<int64_t> n_src, n_dst;
  int64_t tot_src = 0, tot_dst = 0;
  Workspace ws;
  GridPlan gp;
  IcpPlan ip;
  size_t o_src_start = 0, o_dst_start = 0, o_nrm = 0, o_active = 0, o_fb_tiles = 0;
  const float* last_normals = nullptr;  // normals of the last run (null: o_nrm)
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  const void* key[7] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  int launches_per_run = 0;
  DeviceCtx* ctx = nullptr;
};

static cil_status enqueue_batch(BatchHandle* h, const float* src, const float* dst,
                                const double* T_init, double* T_out, cil_icp_report* rep,
                                float* normals, cudaStream_t s) {
  int* dst_start = h->ws.at<int>(h->o_dst_start);
  int* src_start = h->ws.at<int>(h->o_src_start);
  float* nrm = normals ? normals : h->ws.at<float>(h->o_nrm);
  GridOptions opt;
  opt.k_est = h->prm.k;
  opt.cell_size = h->prm.tune.cell_size > 0.0f ? h->prm.tune.cell_size : 0.0f;
  opt.cell_scale = h->prm.tune.cell_scale > 0.0f ? h->prm.tune.cell_scale : kDefaultCellScale;
  cil_status st = grid_build(h->gp, h->ws, dst, dst_start, opt, h->ctx, s);
  if (st != CIL_OK) return st;
  const GridView g = grid_view(h->gp, h->ws);
  const int block = h->prm.tune.block ? h->prm.tune.block : 128;
  const int topk = h->prm.tune.topk >= 0 && h->prm.tune.topk <= 3 ? h->prm.tune.topk : 0;
  if ((st = launch_normals(g, h->B, h->tot_dst, h->prm.k, nullptr, h->prm.viewpoint, dst, nrm,
                           nullptr, block, s, nullptr, topk)) != CIL_OK)
    return st;
  if ((st = icp_run(h->ip, h->ws, g, src, src_start, dst, nrm, T_init, nullptr, h->prm.iters, nullptr,
                    h->prm.max_corr_dist, h->ctx, s)) != CIL_OK)
    return st;
  return icp_export(h->ip, h->ws, T_out, rep, s);
}

// Pairs to re-register: final RMSE not below `thr` (NaN included); counts
// their tiles.  One block.
__global__ void k_fallback_select(const cil_icp_report* __restrict__ rep, int B, double thr,
                                  const int* __restrict__ src_start, int* __restrict__ active,
                                  unsigned* __restrict__ n_tiles) {
  unsigned t = 0;
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    const bool redo = !(rep[b].rmse < thr);
    active[b] = redo ? 1 : 0;
    if (redo) t += (unsigned)((src_start[b + 1] - src_start[b] + kIcpThreads - 1) / kIcpThreads);
  }
  atomicAdd(n_tiles, t);
}

// Keep the better result of each re-registered pair: the identity-started
// one replaces the first when its RMSE is smaller, or when the first has none.
// used[b]: 0 not re-registered, 1 re-registered and the first result kept,
// 2 replaced.
__global__ void k_fallback_merge(const IcpPairState* __restrict__ st, int B,
                                 const int* __restrict__ active, double* __restrict__ T_out,
                                 cil_icp_report* __restrict__ rep, int* __restrict__ used) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  int u = 0;
  if (active[b]) {
    const IcpPairState& S = st[b];
    const double r0 = rep[b].rmse, r1 = S.rmse;
    const bool better = (r1 < r0) || (isnan(r0) && !isnan(r1));
    u = better ? 2 : 1;
    if (better) {
      for (int j = 0; j < 16; ++j) T_out[16 * b + j] = S.T[j];
      cil_icp_report r;
      r.rmse = S.rmse;
      r.n_inliers = S.n_inl;
      r.iters_done = S.iters;
      r.status = S.status;
      rep[b] = r;
    }
  }
  if (used) used[b] = u;
}

}  // namespace cil

using namespace cil;

struct cil_batch {
  BatchHandle h;
};

extern "C" {

cil_status cil_icp_batch_create(const int64_t* n_src, const int64_t* n_dst, int B,
                                const cil_batch_params* params, cil_batch** out) {
  if (!out || !n_src || !n_dst || !params || B < 1 || params->k < 1 || params->k > CIL_MAX_K ||
      params->iters < 0 || !(params->max_corr_dist >= 0.0f))
    return CIL_ERR_INVALID_ARG;
  *out = nullptr;
  int64_t ts = 0, td = 0;
  for (int b = 0; b < B; ++b) {
    if (n_src[b] < 0 || n_dst[b] < 0) return CIL_ERR_INVALID_ARG;
    ts += n_src[b];
    td += n_dst[b];
  }
  if (ts > 0x7fffffff || td > 0x7fffffff) return CIL_ERR_INVALID_ARG;
  cil_status st = CIL_OK;
  DeviceCtx* ctx = device_ctx(&st);
  if (!ctx) return st;
  cil_batch* hb = new cil_batch();
  BatchHandle* h = &hb->h;
  h->B = B;
  h->ctx = ctx;
  h->device = ctx->device;
  h->prm = *params;
  h->n_src.assign(n_src, n_src + B);
  h->n_dst.assign(n_dst, n_dst + B);
  h->tot_src = ts;
  h->tot_dst = td;
  grid_plan(h->gp, h->ws, td, B);
  icp_plan(h->ip, h->ws, n_src, B);
  h->o_src_start = h->ws.reserve(sizeof(int) * (B + 1));
  h->o_dst_start = h->ws.reserve(sizeof(int) * (B + 1));
  h->o_nrm = h->ws.reserve(sizeof(float) * 3 * (size_t)(td > 0 ? td : 1));
  h->o_active = h->ws.reserve(sizeof(int) * B);
  h->o_fb_tiles = h->ws.reserve(sizeof(unsigned));
  if (cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    delete hb;
    return CIL_ERR_CUDA;
  }
  if ((st = h->ws.allocate(ctx, h->cap_stream)) != CIL_OK) {
    cudaStreamDestroy(h->cap_stream);
    delete hb;
    return st;
  }
  std::vector<int> ss(B + 1), ds(B + 1);
  ss[0] = ds[0] = 0;
  for (int b = 0; b < B; ++b) {
    ss[b + 1] = ss[b] + (int)n_src[b];
    ds[b + 1] = ds[b] + (int)n_dst[b];
  }
  if (cudaMemcpyAsync(h->ws.at<int>(h->o_src_start), ss.data(), sizeof(int) * (B + 1),
                      cudaMemcpyHostToDevice, h->cap_stream) != cudaSuccess ||
      cudaMemcpyAsync(h->ws.at<int>(h->o_dst_start), ds.data(), sizeof(int) * (B + 1),
                      cudaMemcpyHostToDevice, h->cap_stream) != cudaSuccess ||
      cudaStreamSynchronize(h->cap_stream) != cudaSuccess) {
    cil_icp_batch_destroy(hb);
    return CIL_ERR_CUDA;
  }
  *out = hb;
  return CIL_OK;
}

cil_status cil_icp_batch_run(cil_batch* hb, const float* src_cat, const float* dst_cat,
                             const double* T_init, double* T_out, cil_icp_report* rep,
                             float* normals_out, void* stream) {
  if (!hb || !T_out || !rep || (hb->h.tot_src > 0 && !src_cat) || (hb->h.tot_dst > 0 && !dst_cat))
    return CIL_ERR_INVALID_ARG;
  BatchHandle* h = &hb->h;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != h->device) return CIL_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const void* key[7] = {src_cat, dst_cat, T_init, T_out, rep, normals_out, (const void*)1};
  bool same = h->exec != nullptr;
  for (int j = 0; j < 7 && same; ++j) same = (key[j] == h->key[j]);
  if (!same) {
    if (h->exec) {
      cudaGraphExecDestroy(h->exec);
      h->exec = nullptr;
    }
    if (h->graph) {
      cudaGraphDestroy(h->graph);
      h->graph = nullptr;
    }
    const int64_t c0 = cil_launch_count();
    if (cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      return CIL_ERR_CUDA;
    cil_status st = enqueue_batch(h, src_cat, dst_cat, T_init, T_out, rep, normals_out,
                                  h->cap_stream);
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(h->cap_stream, &graph);
    if (st != CIL_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    if (ce != cudaSuccess) return CIL_ERR_CUDA;
    // kernels counted while capturing run on every replay, not now
    h->launches_per_run = (int)(cil_launch_count() - c0);
    note_launches(-h->launches_per_run);
    if (cudaGraphInstantiate(&h->exec, graph, 0) != cudaSuccess) {
      cudaGraphDestroy(graph);
      return CIL_ERR_CUDA;
    }
    h->graph = graph;
    for (int j = 0; j < 7; ++j) h->key[j] = key[j];
  }
  if (cudaGraphLaunch(h->exec, s) != cudaSuccess) return CIL_ERR_CUDA;
  note_launches(h->launches_per_run);
  h->last_normals = normals_out;
  return CIL_OK;
}

cil_status cil_icp_batch_fallback(cil_batch* hb, const float* src_cat, const float* dst_cat,
                                  double rmse_threshold, double* T_out, cil_icp_report* rep,
                                  int32_t* used_out, void* stream) {
  if (!hb || !T_out || !rep || (hb->h.tot_src > 0 && !src_cat) || (hb->h.tot_dst > 0 && !dst_cat) ||
      !(rmse_threshold >= 0.0))
    return CIL_ERR_INVALID_ARG;
  BatchHandle* h = &hb->h;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != h->device) return CIL_ERR_INVALID_ARG;
  if (!h->exec) return CIL_ERR_INVALID_ARG;  // no run to fall back from
  cudaStream_t s = (cudaStream_t)stream;
  int* active = h->ws.at<int>(h->o_active);
  unsigned* fb_tiles = h->ws.at<unsigned>(h->o_fb_tiles);
  const int* src_start = h->ws.at<int>(h->o_src_start);
  if (cudaMemsetAsync(fb_tiles, 0, sizeof(unsigned), s) != cudaSuccess) return CIL_ERR_CUDA;
  note_launches(1);
  k_fallback_select<<<1, 1024, 0, s>>>(rep, h->B, rmse_threshold, src_start, active, fb_tiles);
  unsigned n_tiles = 0;
  if (cudaMemcpyAsync(&n_tiles, fb_tiles, sizeof(unsigned), cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return CIL_ERR_CUDA;
  if (n_tiles > 0) {
    const float* nrm = h->last_normals ? h->last_normals : h->ws.at<float>(h->o_nrm);
    cil_status st = icp_run(h->ip, h->ws, grid_view(h->gp, h->ws), src_cat, src_start, dst_cat,
                            nrm, nullptr, nullptr, h->prm.iters, nullptr, h->prm.max_corr_dist,
                            h->ctx, s, nullptr, active, (int)n_tiles);
    if (st != CIL_OK) return st;
  }
  note_launches(1);
  k_fallback_merge<<<ceil_div(h->B, 128), 128, 0, s>>>(icp_state(h->ip, h->ws), h->B, active, T_out,
                                                      rep, used_out);
  return cudaGetLastError() == cudaSuccess ? CIL_OK : CIL_ERR_CUDA;
}

void cil_icp_batch_destroy(cil_batch* hb) {
  if (!hb) return;
  BatchHandle* h = &hb->h;
  if (h->exec) cudaGraphExecDestroy(h->exec);
  if (h->graph) cudaGraphDestroy(h->graph);
  cudaDeviceSynchronize();
  if (h->cap_stream) {
    h->ws.release(h->cap_stream);
    cudaStreamSynchronize(h->cap_stream);
    cudaStreamDestroy(h->cap_stream);
  }
  delete hb;
}

}  // extern "C"
