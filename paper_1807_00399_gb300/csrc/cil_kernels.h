// cil_kernels.h -- host launchers of the query, normals, ICP and radius kernels.
#pragma once

#include "cil_host.h"

namespace cil {

// topk_layout: 0 = by k, 1 = register list, 2 = shared-memory heap (the
// results do not depend on it)
cil_status launch_knn(const GridView& g, const float* qry, int64_t nq, const int* order, int k,
                      int* out_idx, float* out_d2, int block, cudaStream_t s, int topk_layout = 0);

// viewpoints: vp_dev (device float[3 * clouds]) or, when null, vp_host[3]
// out_idx (optional, single cloud): the k neighbour indices of every point,
// row-major (n, k), ascending (d2, index), -1 past the cloud's size -- the
// lists the normals used
cil_status launch_normals(const GridView& g, int clouds, int64_t n, int k, const float* vp_dev,
                          const float* vp_host, const float* xyz, float* out_n, float* out_c,
                          int block, cudaStream_t s, int* out_idx = nullptr,
                          int topk_layout = 0);

cil_status launch_knn_hybrid(const GridView& g, const float* qry, int64_t nq, const int* order,
                             int k, float r, int* out_idx, float* out_d2, cudaStream_t s);
cil_status launch_normals_radius(const GridView& g, int64_t n, float r, const float* vp_host,
                                 float* out_n, float* out_c, int* out_cnt, cudaStream_t s);

// a bounded mbarrier wait that times out (pointnet.cu; failure-path check)
cil_status launch_bounded_wait_check(uint32_t polls, int* err, cudaStream_t s);

// connected-component segmentation over k-NN edges (segment.cu): labels =
// smallest index of each component, count = number of components; `sorted`
// (optional): the grid's sorted points, whose order the union pass follows
cil_status launch_segment(const int* knn_idx, int k, const float* xyz, const float* nrm, int64_t n,
                          const float4* sorted, float cos_t, float r2, int* parent,
                          int32_t* labels, unsigned long long* count, int* err, cudaStream_t s);

// ---------------------------------------------------------------------------
// point-to-plane ICP over B pairs (B = 1 for a single registration)
// ---------------------------------------------------------------------------
struct Mat4 {
  double m[16];
};

// Metric and correspondence search of an ICP run (CIL_METRIC_*, CIL_ASSOC_*;
// the pixel map is the target's organised image for projective association).
struct IcpOptions {
  int metric = CIL_METRIC_POINT_TO_PLANE;
  float w_point = 0.0f, w_plane = 1.0f;
  int association = CIL_ASSOC_NEAREST;
  const int* pixel_map = nullptr;  // device int32[height][width]: target index or -1
  int width = 0, height = 0;
  float fx = 0.0f, fy = 0.0f, cx = 0.0f, cy = 0.0f;
  double* sums = nullptr;  // device [pairs][rounds][kIcpQ + 1]: each round's sums and inlier
                           // count as the round close sees them, or null (not recorded)
};

struct IcpPairState {
  double T[16];     // current transform (source -> target), row-major
  double rmse;      // final point-to-plane RMSE
  long long n_inl;  // final inlier count
  float Rt[12];     // T as float rows [R | t] for the association passes
  float Rt_prev[12];  // the previous round's Rt (certificates of unchanged neighbours)
  int has_prev;     // Rt_prev holds a round's transform
  float dmax2;      // squared rejection distance
  float ref[3];     // reference point of the pair (point-to-point sums are about it)
  int tile_begin, tile_end;
  int grp_begin;    // first tile group of the pair (groups of kIcpGroup tiles)
  int n_grp;        // tile groups of the pair
  int tiles_done;   // tile groups of the current round reduced
  int status;       // CIL_OK or CIL_ERR_DEGENERATE
  int iters;        // rounds requested
};

struct IcpPlan {
  int pairs = 1;
  int64_t n_src = 0;
  int n_tiles = 0;
  int tile = 0;     // source points per tile
  int n_groups = 0;  // tile groups over all pairs
  size_t o_state, o_order, o_src_sorted, o_tile_off, o_rt, o_part_s, o_part_c, o_part_n;
  size_t o_grp_s, o_grp_c, o_grp_n, o_grp_done;
  size_t o_corr, o_lbd, o_queue, o_qc;
  OrderPlan order;
};

constexpr int kIcpThreads = 256;  // source points per tile (one per thread)
constexpr int kIcpQ = 28;  // 21 (H upper) + 6 (g) + 1 (sum r^2)
constexpr int kIcpGroup = 32;  // tiles reduced together before the round's solve

// Reserve workspace; `src_counts` host array of per-pair source sizes.
void icp_plan(IcpPlan& p, Workspace& ws, const int64_t* src_counts, int pairs);

// Enqueue: order the sources, initialise per-pair state from T_init (device
// double[16 * pairs], or host double[16] for one pair, or both null =
// identity) and run all rounds plus the final RMSE pass (three launches per
// round).  `src_start_dev`: device int[pairs+1] (null for one pair).
// `active_dev` (device int[pairs], or null = all): pairs with 0 get no tiles;
// `n_tiles_active` is then the tile count of the active pairs (launch size).
cil_status icp_run(const IcpPlan& p, const Workspace& ws, const GridView& tgt,
                   const float* src, const int* src_start_dev, const float* dst,
                   const float* dst_normals,
                   const double* T_init_dev, const double* T_init_host, int iters,
                   const float* dmax_dev, float dmax, DeviceCtx* ctx, cudaStream_t s,
                   const IcpOptions* opt = nullptr, const int* active_dev = nullptr,
                   int n_tiles_active = -1);

IcpPairState* icp_state(const IcpPlan& p, const Workspace& ws);

// copy results of pair b to T_out (device double[16]) and rep (device)
cil_status icp_export(const IcpPlan& p, const Workspace& ws, double* T_out_dev,
                      cil_icp_report* rep_dev, cudaStream_t s);

}  // namespace cil
