// noalloc.cu -- k-nearest-neighbour search that allocates no device memory.
//
// cil_knn takes its temporary buffers (grid, sort keys, query order) from a
// stream-ordered pool.  Some callers cannot allocate at all: plugins running
// inside a host framework whose own allocator owns all device memory, real-
// time loops that forbid allocation once started (an allocation can block or
// fail under fragmentation), and certified code that allows no dynamic
// allocation after initialisation.  cil_knn_noalloc runs the same kernels on
// scratch that lives in a fixed-size device array inside the library itself.
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library holds it (kNoAllocScratchBytes) until the process exits.  Host code
// cannot use the array's name as a device address (it is a host-side stand-in
// for the symbol), so the first call on each device looks the address up with
// cudaGetSymbolAddress while that device is current; make that first call
// before any stream capture.  All calls share the one array: calls that
// overlap on the GPU (other streams, other host threads) race and corrupt each
// other's results.  What must start from a known state (the cell table, the
// error word) is reset by every call.
#include <mutex>

#include "cil_host.h"
#include "cil_kernels.h"

namespace cil {

constexpr int64_t kNoAllocMaxPoints = 32768;          // per reference and per query set
constexpr size_t kNoAllocScratchBytes = 8u << 20;     // 8 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];
static __device__ int g_noalloc_err;

struct NoAllocDevice {
  int device = -1;
  int num_sms = 0;
  void* scratch = nullptr;  // device address of g_noalloc_scratch
  int* err = nullptr;       // device address of g_noalloc_err
};
static std::mutex g_noalloc_mu;
static NoAllocDevice g_noalloc_dev[64];

// once per device, with that device current: resolve the symbols' addresses
static cil_status noalloc_setup(NoAllocDevice* out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return CIL_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  NoAllocDevice& d = g_noalloc_dev[dev];
  if (d.device != dev) {
    void* scratch = nullptr;
    void* err = nullptr;
    int sms = 0;
    if (cudaGetSymbolAddress(&scratch, g_noalloc_scratch) != cudaSuccess) return CIL_ERR_CUDA;
    if (cudaGetSymbolAddress(&err, g_noalloc_err) != cudaSuccess) return CIL_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return CIL_ERR_CUDA;
    d.scratch = scratch;
    d.err = static_cast<int*>(err);
    d.num_sms = sms;
    d.device = dev;
  }
  *out = d;
  return CIL_OK;
}

// keeps the workspace pointed at the static array for the scope, and detaches
// it on every exit path so nothing ever tries to free the array
struct AttachGuard {
  Workspace& ws;
  AttachGuard(Workspace& w, void* base) : ws(w) { ws.attach(base); }
  ~AttachGuard() { ws.detach(); }
};

}  // namespace cil

using namespace cil;

extern "C" cil_status cil_knn_noalloc(const float* ref, int64_t n_ref, const float* qry,
                                      int64_t n_qry, int k, int32_t* out_idx, float* out_d2,
                                      void* stream) {
  if (k < 1 || k > CIL_MAX_K || n_ref < 0 || n_qry < 0) return CIL_ERR_INVALID_ARG;
  if (n_ref > kNoAllocMaxPoints || n_qry > kNoAllocMaxPoints) return CIL_ERR_CAPACITY;
  if (n_qry == 0) return CIL_OK;
  if (!qry || !out_idx || (n_ref > 0 && !ref)) return CIL_ERR_INVALID_ARG;
  NoAllocDevice d;
  cil_status st = noalloc_setup(&d);
  if (st != CIL_OK) return st;
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
  if (ws.total() > kNoAllocScratchBytes) return CIL_ERR_CAPACITY;
  AttachGuard guard(ws, d.scratch);
  if (cudaMemsetAsync(d.err, 0, sizeof(int), s) != cudaSuccess) return CIL_ERR_CUDA;
  DeviceCtx ctx;
  ctx.device = d.device;
  ctx.num_sms = d.num_sms;
  ctx.err = d.err;
  ctx.pool = nullptr;
  GridOptions opt;
  opt.k_est = k;
  if ((st = grid_build(gp, ws, ref, nullptr, opt, &ctx, s)) != CIL_OK) return st;
  const GridView g = grid_view(gp, ws);
  int* order = nullptr;
  if (!self) {
    order = ws.at<int>(o_order);
    if ((st = order_queries(op, ws, qry, nullptr, 1, g.prm, nullptr, order, s)) != CIL_OK) return st;
  }
  if ((st = launch_knn(g, qry, n_qry, order, k, out_idx, out_d2, 128, s)) != CIL_OK) return st;
  int v = 0;
  if (cudaMemcpyAsync(&v, d.err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return CIL_ERR_CUDA;
  return v ? (cil_status)v : CIL_OK;
}
