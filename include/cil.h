/*
 * cil.h -- C ABI of the GB300 point-cloud hot path: k-nearest-neighbour and
 * radius search over a uniform grid, PCA surface normals, and rigid
 * point-to-plane ICP.
 *
 * The operations follow the cilantro paper (Zampogiannis, Fermueller,
 * Aloimonos, ACM MM 2018):
 *   - Sec. 3 "Core operations": k-NN, radius and hybrid queries on a point set;
 *     surface normal and curvature estimation; PCA;
 *   - Sec. 3 "Iterative geometric registration": the ICP loop alternating
 *     correspondence search and a rigid point-to-plane estimator (Low 2004);
 *   - Sec. 4: 10-NN normal neighbourhoods with viewpoint-consistent
 *     orientation; ICP with a fixed iteration count and a rejection distance.
 *
 * Common conventions
 *   Points      const float xyz[n][3], x/y/z interleaved, one point after the
 *               other (the paper's contiguous "one point per column" matrix
 *               view, Sec. 2).  All point and output arrays are DEVICE pointers
 *               owned by the caller unless the comment says "host".
 *   Indices     int32, relative to the reference cloud; n <= 2^31 - 1.
 *   Ordering    neighbour lists ascend by (squared distance, index): ties in
 *               FP32 squared distance are broken by the smaller index.
 *   Distances   squared Euclidean distances in FP32, each coordinate
 *               difference formed directly (q - p), never via |q|^2 - 2 q.p.
 *   Transforms  double[16], row-major 4x4 rigid transform mapping SOURCE
 *               coordinates to TARGET coordinates.
 *   Streams     every call is enqueued on `stream` (a cudaStream_t passed as
 *               void*; NULL = legacy default stream).  Calls with host outputs
 *               synchronise that stream before returning; the others return
 *               as soon as the work is enqueued.
 *   Workspace   the library allocates its temporary device memory from its own
 *               stream-ordered pool on the call's stream and releases it on the
 *               same stream; nothing persists between calls except handles.
 *   Errors      argument errors are returned synchronously.  Errors detected
 *               on the device (non-finite coordinates, a bounded wait that ran
 *               out) are recorded in a per-device error word: calls that
 *               synchronise return them; cil_sync_status() returns and clears
 *               them for the asynchronous calls.  No call falls back to the CPU.
 */
#ifndef CIL_H
#define CIL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  CIL_OK = 0,
  CIL_ERR_INVALID_ARG = 1, /* null pointer, bad size, k out of range, ...   */
  CIL_ERR_CUDA = 2,        /* a CUDA runtime call failed                      */
  CIL_ERR_NONFINITE = 3,   /* an input coordinate is NaN or infinite          */
  CIL_ERR_CAPACITY = 4,    /* output buffer too small (radius search)        */
  CIL_ERR_DEGENERATE = 5,  /* ICP normal equations singular / < 6 inliers    */
  CIL_ERR_TIMEOUT = 6,     /* a bounded device-side wait gave up              */
  CIL_ERR_NOMEM = 7        /* device workspace allocation failed              */
} cil_status;

#define CIL_MAX_K 32

/* Optional tuning knobs (pass NULL for defaults).  None of them changes a
 * result, only the time it takes.
 *   cell_size   > 0: grid cell edge in input units (rounded to the nearest
 *               power-of-two multiple of the cloud's fine Morton resolution,
 *               max_extent / 1023); 0: chosen from the data.
 *   cell_scale  multiplier applied to the data-driven cell size (the median
 *               distance of sampled points to their k-th neighbour; 0 = 1.5).
 *   block       threads per block of the query kernels (0 = default 128;
 *               64, 128, 256 accepted).
 *   topk        how the k-NN and normals kernels search: 0 = the default;
 *               1 = one thread per query, its k best in a sorted register
 *               list; 2 = one thread per query, a binary max-heap in shared
 *               memory (k = 1 always uses the list; the default picks the list
 *               for k < 8, the heap from 8 on); 3 = warp-staged: the 32
 *               Morton-adjacent queries of a warp scan one shared set of
 *               points (their cells and one ring around them, staged in
 *               shared memory), a query whose k-th distance is not proven
 *               inside that set continuing with the per-query search. */
typedef struct {
  float cell_size;
  float cell_scale;
  int block;
  int topk;
} cil_params;

/* Human-readable name of a status code (static storage). */
const char *cil_status_string(cil_status s);

/* Synchronise `stream`, return the device error word (CIL_OK if clean) and
 * clear it. */
cil_status cil_sync_status(void *stream);

/* ---------------------------------------------------------------------------
 * k nearest neighbours (Sec. 3, KDTree k-NN query; here a uniform grid).
 *   ref      [n_ref][3]   reference points (device)
 *   qry      [n_qry][3]   query points (device); may alias ref (self-query: a
 *                         point is its own first neighbour at distance 0)
 *   k        1..CIL_MAX_K
 *   out_idx  [n_qry][k]   int32 neighbour indices into ref (device)
 *   out_d2   [n_qry][k]   float squared distances (device), may be NULL
 * Each row ascends by (d2, idx).  When k > n_ref the row is padded with
 * idx = -1, d2 = +inf.  Exact: the grid search expands until no unvisited
 * cell can hold a closer point.  n_qry == 0 is a no-op; n_ref == 0 pads.
 * Asynchronous.
 */
cil_status cil_knn(const float *ref, int64_t n_ref, const float *qry, int64_t n_qry, int k,
                   int32_t *out_idx, float *out_d2, void *stream);
cil_status cil_knn_ex(const float *ref, int64_t n_ref, const float *qry, int64_t n_qry, int k,
                      int32_t *out_idx, float *out_d2, const cil_params *params, void *stream);

/* ---------------------------------------------------------------------------
 * k nearest neighbours without any device allocation (the paper has no
 * counterpart: it concerns how the library obtains memory, not what it
 * computes).  For callers that cannot call cudaMalloc -- plugins inside a host
 * framework whose allocator owns all device memory, real-time loops that
 * forbid allocation after start-up, certified code without dynamic allocation
 * -- this runs cil_knn's kernels on scratch held in a fixed 8 MiB array inside
 * the library (every GPU that loads the library keeps it until exit).
 * Arguments, layout and results are those of cil_knn, except:
 *   - n_ref and n_qry must each be <= 32768, else CIL_ERR_CAPACITY (nothing is
 *     launched);
 *   - the first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; the address is kept
 *     for the life of the process, so after a cudaDeviceReset of that device
 *     this entry point must not be called again;
 *   - every call shares the one array: calls that overlap on the GPU race and
 *     corrupt each other's results; each call resets the state it needs;
 *   - the call synchronises `stream` and returns a device-detected error
 *     (CIL_ERR_NONFINITE) directly.
 */
cil_status cil_knn_noalloc(const float *ref, int64_t n_ref, const float *qry, int64_t n_qry,
                           int k, int32_t *out_idx, float *out_d2, void *stream);

/* ---------------------------------------------------------------------------
 * Radius search (Sec. 3, KDTree radius query): for every query all reference
 * points with squared distance <= r*r (inclusive), as CSR:
 *   out_offsets [n_qry+1] int64 (device): row q is [offsets[q], offsets[q+1])
 *   out_idx     [capacity] int32 (device), out_d2 [capacity] float (device,
 *               may be NULL); rows ascend by (d2, idx)
 *   out_nnz     host int64: total number of neighbours found
 * If the total exceeds `capacity`, nothing is written to out_idx/out_d2,
 * out_offsets holds the full CSR offsets, *out_nnz the required size, and the
 * call returns CIL_ERR_CAPACITY.  r >= 0.  Synchronises the stream.
 */
cil_status cil_radius_search(const float *ref, int64_t n_ref, const float *qry, int64_t n_qry,
                             float r, int64_t *out_offsets, int32_t *out_idx, float *out_d2,
                             int64_t capacity, int64_t *out_nnz, void *stream);
/* The same with tuning knobs (NULL = defaults): the search cells' edge is r,
 * or params->cell_size when > 0, or r * params->cell_scale when > 0 (rounded
 * to a power-of-two multiple of the fine lattice); block and topk unused.
 * Results do not depend on them. */
cil_status cil_radius_search_ex(const float *ref, int64_t n_ref, const float *qry, int64_t n_qry,
                                float r, int64_t *out_offsets, int32_t *out_idx, float *out_d2,
                                int64_t capacity, int64_t *out_nnz, const cil_params *params,
                                void *stream);

/* ---------------------------------------------------------------------------
 * Hybrid query (Sec. 3, KDTree "hybrid" queries): for every query the k
 * nearest reference points among those with squared distance <= r*r
 * (inclusive).  Same layout, order and padding (-1 / +inf) as cil_knn; rows
 * hold fewer than k valid entries when the ball holds fewer points.  r >= 0.
 * Asynchronous.
 */
cil_status cil_knn_hybrid(const float *ref, int64_t n_ref, const float *qry, int64_t n_qry, int k,
                          float r, int32_t *out_idx, float *out_d2, void *stream);

/* ---------------------------------------------------------------------------
 * PCA normals over radius neighbourhoods (Sec. 3 normal estimation; Sec. 4
 * compares 1 cm balls): for every point, all points within r (inclusive, the
 * point itself included) form the neighbourhood; mean, centred covariance,
 * smallest eigenvector, viewpoint orientation and curvature as in
 * cil_estimate_normals.  out_counts [n] int32 (device, may be NULL) receives
 * each neighbourhood's size; fewer than 3 neighbours give NaN.  r > 0.
 * Asynchronous.
 */
cil_status cil_estimate_normals_radius(const float *xyz, int64_t n, float r, const float *viewpoint,
                                       float *out_normals, float *out_curvature,
                                       int32_t *out_counts, void *stream);

/* ---------------------------------------------------------------------------
 * PCA surface normals and curvature (Sec. 3 normal/curvature estimation,
 * Sec. 4 k-NN neighbourhoods, viewpoint-consistent orientation).
 *   xyz          [n][3] points (device)
 *   k            neighbourhood size including the point itself, 1..CIL_MAX_K
 *   viewpoint    host float[3]; each normal is flipped so that
 *                normal . (viewpoint - p) >= 0
 *   out_normals  [n][3] float (device): unit eigenvector of the smallest
 *                eigenvalue of C = (1/m) sum (p_j - mu)(p_j - mu)^T over the
 *                m = min(k, n) neighbours
 *   out_curvature [n] float (device, may be NULL): l0 / (l0 + l1 + l2)
 * Fewer than 3 neighbours or a zero covariance give NaN normal and curvature.
 * Asynchronous.
 */
cil_status cil_estimate_normals(const float *xyz, int64_t n, int k, const float *viewpoint,
                                float *out_normals, float *out_curvature, void *stream);
cil_status cil_estimate_normals_ex(const float *xyz, int64_t n, int k, const float *viewpoint,
                                   float *out_normals, float *out_curvature,
                                   const cil_params *params, void *stream);

/* ---------------------------------------------------------------------------
 * Voxel-grid downsampling (Sec. 3 GridAccumulator; Sec. 4 downsamples to
 * 1 cm voxels before ICP): point p falls in voxel floor(p / voxel) per axis
 * (correctly rounded FP32 division, voxel indices clamped to +-2^20); each
 * occupied voxel yields the mean of its points.
 *   out_xyz     [n][3] float (device; capacity n: at most n voxels)
 *   out_counts  [n] int32 (device, may be NULL): points per output voxel
 *   out_n       host: number of output voxels
 * Output voxels ascend by (ix, iy, iz).  Synchronises the stream.
 */
cil_status cil_voxel_downsample(const float *xyz, int64_t n, float voxel, float *out_xyz,
                                int32_t *out_counts, int64_t *out_n, void *stream);

/* ---------------------------------------------------------------------------
 * Rigid point-to-plane ICP (Sec. 2 ICP base loop; Sec. 3 point-to-plane
 * estimator after Low 2004; Sec. 4 fixed iterations + rejection distance).
 * Each of `max_iters` rounds, at the current T:
 *   p' = R p + t for every source point; q = nearest target point of p';
 *   the pair is an inlier if |p' - q| <= max_corr_dist and q's normal is
 *   finite; r = n_q . (p' - q), J = [p' x n_q, n_q];
 *   H = sum J J^T, g = sum J r (FP32 terms, compensated FP32 sums);
 *   solve H xi = -g in FP64 (Cholesky), xi = (w, tau);
 *   T <- [exp(w^), tau; 0 1] * T  (FP64).
 * A round with < 6 inliers or a Cholesky pivot <= 1e-12 * trace(H) is
 * skipped and reported as CIL_ERR_DEGENERATE in rep->status.  No early stop.
 * After the last round one more association pass gives the point-to-plane
 * RMSE over the inliers.
 *   src [n_src][3], dst [n_dst][3], dst_normals [n_dst][3]   (device)
 *   T_init host double[16] (NULL = identity); T_out host double[16]
 *   rep    host report
 * Synchronises the stream; returns rep->status's error if the device error
 * word is set.
 */
typedef struct {
  double rmse;       /* point-to-plane RMSE after the final association   */
  int64_t n_inliers; /* inliers in the final association                   */
  int iters_done;    /* rounds executed (== max_iters)                     */
  int status;        /* CIL_OK or CIL_ERR_DEGENERATE (any round skipped)   */
} cil_icp_report;

cil_status cil_icp_point_to_plane(const float *src, int64_t n_src, const float *dst,
                                  const float *dst_normals, int64_t n_dst, const double *T_init,
                                  int max_iters, float max_corr_dist, double *T_out,
                                  cil_icp_report *rep, void *stream);

/* ---------------------------------------------------------------------------
 * One registration of a frame pair, the paper's Sec. 4 pipeline in one call:
 * build the target grid once, estimate k-NN normals of the target (oriented
 * to `viewpoint`), then run point-to-plane ICP of `src` against it.
 * Everything stays on the device; nothing is synchronised:
 *   out_normals [n_dst][3] float (device, may be NULL: kept internal)
 *   T_init  device double[16] or NULL (identity)
 *   T_out   device double[16];  rep  device cil_icp_report
 */
cil_status cil_register_pair(const float *src, int64_t n_src, const float *dst, int64_t n_dst,
                             int k, const float *viewpoint, const double *T_init, int max_iters,
                             float max_corr_dist, float *out_normals, double *T_out,
                             cil_icp_report *rep, const cil_params *params, void *stream);

/* ---------------------------------------------------------------------------
 * Connected-component segmentation on the k-NN graph (Sec. 3: connected
 * components under a point-wise similarity, e.g. smooth segments; Sec. 4
 * segments a reconstruction with k = 30 and a normal-angle threshold).
 *   xyz, normals  device float[n][3] (oriented unit normals, e.g. from
 *                 cil_estimate_normals; a point with a non-finite normal has
 *                 no edge)
 *   k             neighbours per point, self included (1..CIL_MAX_K)
 *   theta         normal-angle threshold in radians (>= 0): i and j are
 *                 joined when j is among the k nearest of i (or i of j) and
 *                 n_i . n_j >= cos(theta)
 *   radius        > 0: additionally |p_i - p_j| <= radius; 0: no distance test
 *   out_labels    device int32[n]: the smallest point index of each point's
 *                 component
 *   out_count     host: number of components
 * The similarity tests are evaluated in FP32 ((x x + y y) + z z, no fused
 * multiply-add, thresholds rounded to FP32).  Synchronises the stream.
 * CIL_ERR_INVALID_ARG for bad sizes, k, theta or radius, or null pointers;
 * CIL_ERR_NONFINITE for non-finite coordinates.
 * ------------------------------------------------------------------------- */
cil_status cil_segment(const float *xyz, const float *normals, int64_t n, int k, float theta,
                       float radius, int32_t *out_labels, int64_t *out_count, void *stream);

/* ---------------------------------------------------------------------------
 * Smooth segmentation in one search (Sec. 3 normals and connected components;
 * Sec. 4's first test): the k nearest neighbours of every point are found
 * once, give its PCA normal (as cil_estimate_normals, oriented towards
 * viewpoint) and its edges of the graph of cil_segment.
 *   xyz           device float[n][3]
 *   k             neighbours per point, self included (1..CIL_MAX_K), for
 *                 both the normals and the graph
 *   viewpoint     host float[3]
 *   theta, radius as cil_segment
 *   out_normals   device float[n][3] or NULL (then kept internally)
 *   out_labels    device int32[n]: smallest point index of each component
 *   out_count     host: number of components
 * Labels equal cil_segment's on the same normals.  Synchronises the stream.
 * Errors as cil_segment; CIL_ERR_INVALID_ARG for a null viewpoint.
 * ------------------------------------------------------------------------- */
cil_status cil_smooth_segment(const float *xyz, int64_t n, int k, const float *viewpoint,
                              float theta, float radius, float *out_normals, int32_t *out_labels,
                              int64_t *out_count, void *stream);

/* ---------------------------------------------------------------------------
 * ICP variants (Sec. 3: the ICP loop parameterised by the correspondence
 * search and the estimator; rigid registration under the point-to-point
 * metric (Besl & McKay), the point-to-plane metric (Low) and weighted
 * combinations thereof; correspondences by nearest-neighbour search or by
 * projective data association).
 *   metric       CIL_METRIC_POINT_TO_PLANE: as cil_icp_point_to_plane;
 *                CIL_METRIC_POINT_TO_POINT: each round the closed-form rigid
 *                motion minimising sum |R p' + t - q|^2 (FP64);
 *                CIL_METRIC_COMBINED: w_point sum |p' - q|^2 + w_plane sum
 *                (n.(p' - q))^2, linearised, one FP64 Gauss-Newton step per
 *                round (w_point, w_plane >= 0, finite).
 *   association  CIL_ASSOC_NEAREST: exact nearest target point within
 *                max_corr_dist (as cil_icp_point_to_plane);
 *                CIL_ASSOC_PROJECTIVE: the target is the organised image of
 *                its camera (target coordinates = camera frame): p' projects
 *                to pixel (round(fx x/z + cx), round(fy y/z + cy)) (halves to
 *                even); pixel_map (device int32[height][width]) holds the
 *                index of the target point seen at each pixel or -1; the
 *                point there is the correspondence when |p' - q| <=
 *                max_corr_dist; z <= 0, outside the image or -1: none.
 * The report's rmse is the metric's own residual after the final
 * association pass: point-to-point distance, plane residual, or
 * sqrt(mean(w_point d^2 + w_plane r^2)).  Rounds whose system does not fix a
 * motion (fewer than 3 correspondences for the closed form, fewer than 6 or
 * a Cholesky pivot <= 1e-12 tr H otherwise) keep T and report
 * CIL_ERR_DEGENERATE.
 * ------------------------------------------------------------------------- */
typedef enum {
  CIL_METRIC_POINT_TO_PLANE = 0,
  CIL_METRIC_POINT_TO_POINT = 1,
  CIL_METRIC_COMBINED = 2
} cil_icp_metric;

typedef enum { CIL_ASSOC_NEAREST = 0, CIL_ASSOC_PROJECTIVE = 1 } cil_icp_association;

typedef struct {
  int metric;               /* cil_icp_metric                                  */
  float w_point, w_plane;   /* weights of CIL_METRIC_COMBINED                  */
  int association;          /* cil_icp_association                             */
  const int32_t* pixel_map; /* device int32[height][width] (projective only)   */
  int width, height;        /* image size (projective only)                    */
  float fx, fy, cx, cy;     /* pinhole intrinsics (projective only)            */
} cil_icp_options;

/* cil_icp_point_to_plane with a metric and a correspondence search chosen by
 * `opt` (NULL: point-to-plane, nearest neighbour).  dst_normals may be NULL
 * for CIL_METRIC_POINT_TO_POINT.  Same argument rules, outputs and
 * synchronisation as cil_icp_point_to_plane; additionally
 * CIL_ERR_INVALID_ARG for an unknown metric or association, negative or
 * non-finite weights, or a projective search without a pixel map, positive
 * image size and finite intrinsics. */
cil_status cil_icp(const float *src, int64_t n_src, const float *dst, const float *dst_normals,
                   int64_t n_dst, const double *T_init, int max_iters, float max_corr_dist,
                   const cil_icp_options *opt, double *T_out, cil_icp_report *rep, void *stream);

/* cil_icp that also returns, for every round, the normal-equation sums the
 * round's solve used (Sec. 3 point-to-plane estimator: the linearised system
 * H xi = -g accumulated over the round's correspondences; the paper states
 * the estimator, not a layout).  Diagnostics and precision checks of the
 * compensated FP32 sums against an FP64 reference.
 *   sums_out  host double[max_iters + 1][29], round r at sums_out + 29 r:
 *             [0, 21)  H, upper triangle row by row (H00 H01 .. H05 H11 .. H55)
 *             [21, 27) g
 *             27       sum of r^2 over the inliers
 *             28       inlier count
 *             (point-to-plane metric; for the other metrics the first 28 slots
 *             hold that metric's 28 sums).  Row max_iters is the final
 *             association pass.  Rounds that never ran hold zeros.
 * Everything else as cil_icp; CIL_ERR_INVALID_ARG for a null sums_out. */
cil_status cil_icp_sums(const float *src, int64_t n_src, const float *dst, const float *dst_normals,
                        int64_t n_dst, const double *T_init, int max_iters, float max_corr_dist,
                        const cil_icp_options *opt, double *T_out, cil_icp_report *rep,
                        double *sums_out, void *stream);

/* ---------------------------------------------------------------------------
 * Batched registration of B independent pairs of uneven sizes (no counterpart
 * in the paper, which registers one pair at a time, Sec. 4).  Per pair: the
 * same target grid + k-NN normals + point-to-plane ICP as cil_register_pair,
 * all pairs in one CUDA graph launch: one grid build over the concatenated
 * targets (one cell level per pair), one normals kernel, and per ICP round
 * three kernels over all pairs' source tiles.
 *   cil_icp_batch_create  n_src, n_dst: host int64[B] point counts; allocates
 *                         the handle's device workspace (synchronous)
 *   cil_icp_batch_run     src_cat [sum n_src][3], dst_cat [sum n_dst][3]:
 *                         device, pairs concatenated in order;
 *                         T_init  device double[B][16] or NULL (identity);
 *                         T_out   device double[B][16];
 *                         rep     device cil_icp_report[B];
 *                         normals_out device float[sum n_dst][3] or NULL.
 *                         Asynchronous.  The first run with a given set of
 *                         pointers captures a CUDA graph (call it outside any
 *                         stream capture); later runs with the same pointers
 *                         replay it.
 *   cil_icp_batch_destroy waits for the device to be idle, frees everything.
 * Runs of one handle must not overlap on the device (they share workspace).
 */
typedef struct {
  int k;               /* normals neighbourhood, 1..CIL_MAX_K                */
  int iters;           /* ICP rounds                                         */
  float max_corr_dist; /* rejection distance for every pair                  */
  float viewpoint[3];  /* normal orientation for every pair                  */
  cil_params tune;     /* grid cell size / scale, query block size           */
} cil_batch_params;

typedef struct cil_batch cil_batch;

cil_status cil_icp_batch_create(const int64_t *n_src, const int64_t *n_dst, int B,
                                const cil_batch_params *params, cil_batch **out);
cil_status cil_icp_batch_run(cil_batch *h, const float *src_cat, const float *dst_cat,
                             const double *T_init, double *T_out, cil_icp_report *rep,
                             float *normals_out, void *stream);
void cil_icp_batch_destroy(cil_batch *h);

/* Fallback of a warm-started batch (no counterpart in the paper: plain ICP
 * from the identity stays the fallback of the learned warm start below).
 * Call after cil_icp_batch_run of the same handle, with the same src_cat,
 * dst_cat, T_out and rep, on the same stream (it reuses that run's target
 * grid and normals).  Pairs whose rep[b].rmse is >= rmse_threshold, or NaN
 * (no inliers), are re-registered from the identity (k-NN association,
 * point-to-plane, the handle's iterations and rejection distance; only their
 * source tiles are launched) and keep the result with the smaller final RMSE
 * (the re-registered one wins over a NaN); T_out and rep are updated in
 * place.  Every re-registered pair's result is bitwise the result an
 * identity-started cil_icp_batch_run gives that pair.
 *   used_out  device int32[B] or NULL: 0 not re-registered, 1 re-registered
 *             and the first result kept, 2 replaced by the re-registration
 * Synchronises the stream once (to read how many source tiles to launch);
 * not for stream capture.  CIL_ERR_INVALID_ARG for a null handle or output,
 * a negative or NaN threshold, or a handle that has not run. */
cil_status cil_icp_batch_fallback(cil_batch *h, const float *src_cat, const float *dst_cat,
                                  double rmse_threshold, double *T_out, cil_icp_report *rep,
                                  int32_t *used_out, void *stream);

/* ---------------------------------------------------------------------------
 * Learned warm start (no counterpart in the paper; it seeds the Sec. 3 ICP).
 * A PointNet-style regressor of the source -> target transform:
 *   encoder, shared by both clouds of a pair: 3 -> 64 (FP32), 64 -> 128 and
 *   128 -> 256 (BF16 tensor cores, FP32 accumulation), ReLU after each,
 *   global max-pool over the points;
 *   head: [f_src, f_dst] (512) -> 256 (ReLU) -> 9; R = Gram-Schmidt of the
 *   first two 3-vectors (columns b1, b2, b1 x b2), t = last three;
 *   loss: mean over pairs of mean over source points |(R p + t) - (Rg p + tg)|^2.
 * Parameters: one FP32 vector of cil_pointnet_num_params() values in the order
 * W1[64][3] b1 W2[128][64] b2 W3[256][128] b3 W4[256][512] b4 W5[9][256] b5.
 *   clouds  device float[B][2][P][3]: per pair the source then the target cloud
 *           (P = n_points, a multiple of 128)
 *   T_gt    device double[B][16] row-major source -> target labels
 *   T_out   device double[B][16] predicted transforms (may be NULL)
 *   cil_pointnet_forward   prediction only (features to feat_out [B][512] if
 *                          not NULL)
 *   cil_pointnet_backward  forward + loss (per pair, device float[B]) +
 *                          gradient of the mean loss (device float[n_params])
 *   cil_pointnet_adam_step Adam (0.9, 0.999, 1e-8) on the FP32 master weights
 *                          with the last gradient, then refreshes the BF16 copies
 * All asynchronous on `stream`; a handle's calls must not overlap.
 */
typedef struct cil_pointnet cil_pointnet;
int cil_pointnet_num_params(void);
cil_status cil_pointnet_create(int max_pairs, int n_points, cil_pointnet **out);
void cil_pointnet_destroy(cil_pointnet *h);
cil_status cil_pointnet_set_params(cil_pointnet *h, const float *params, void *stream);
cil_status cil_pointnet_get_params(cil_pointnet *h, float *params, void *stream);
cil_status cil_pointnet_forward(cil_pointnet *h, const float *clouds, int B, double *T_out,
                                float *feat_out, void *stream);
cil_status cil_pointnet_backward(cil_pointnet *h, const float *clouds, const double *T_gt, int B,
                                 float *loss_out, float *grad_out, void *stream);
cil_status cil_pointnet_adam_step(cil_pointnet *h, float lr, void *stream);

/* ---------------------------------------------------------------------------
 * Instrumentation (benchmarks, profiling; no counterpart in the paper).
 *   cil_launch_count   kernels this library has launched since it was loaded
 *   cil_timing_enable  1: record a pair of CUDA events on the launching stream
 *                      around each instrumented kernel ("k_icp", "k_knn",
 *                      "k_normals", "k_radius") and the grid build
 *                      ("grid_build"); 0: stop recording
 *   cil_timing_read    wait for the recorded events of `name` and return their
 *                      summed duration (ms) and count
 *   cil_timing_reset   wait for and drop every record
 */
int64_t cil_launch_count(void);
void cil_timing_enable(int on);
cil_status cil_timing_read(const char *name, double *total_ms, int64_t *launches);
void cil_timing_reset(void);

/* ---------------------------------------------------------------------------
 * Failure-path checks (tests; no counterpart in the paper).  Faults are made
 * on the host or with waits that end by themselves, never by faulting the GPU.
 *   cil_test_fail_next_allocations  the next `count` workspace allocations of
 *                      any call fail with CIL_ERR_NOMEM (0 clears)
 *   cil_check_bounded_wait  launches one warp that waits on an mbarrier no one
 *                      arrives on, bounded by `polls` polls as the encoder's
 *                      waits are; synchronises `stream` and returns the
 *                      error word: CIL_ERR_TIMEOUT (the wait gave up and the
 *                      kernel returned; the context stays usable)
 */
void cil_test_fail_next_allocations(int count);
cil_status cil_check_bounded_wait(unsigned polls, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* CIL_H */
