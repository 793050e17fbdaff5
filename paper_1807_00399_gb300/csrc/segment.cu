// segment.cu -- connected-component segmentation on the k-NN graph (Sec. 3:
// connected components under a point-wise similarity, e.g. smooth segments;
// Sec. 4 segments an apartment-scale reconstruction with k = 30 and a
// normal-angle threshold).
//
// Graph: {i, j} for every j among the k nearest neighbours of i (self
// included, so k - 1 others), kept when the oriented normals' angle is at
// most theta (n_i . n_j >= cos theta) and, with a radius r > 0, the points
// are at most r apart.  The two tests decide integers from floating point, so
// they are evaluated in FP32 with a fixed operation order and no fused
// multiply-add ((x x + y y) + z z), the order the oracle uses.
// Components by a concurrent union-find: a root is hooked with an atomic
// compare-and-swap onto a smaller index of the other set, so parents always
// have smaller indices than their children, every find terminates, and each
// component ends with its smallest index as root -- the label, independent of
// the order in which edges were processed.
#include "cil_host.h"
#include "cil_kernels.h"

namespace cil {

constexpr int kSegThreads = 256;
constexpr int kUnionSteps = 1 << 20;  // a union needs far fewer; the cap only bounds the loop
constexpr int kSegFirst = 3;           // list entries joined before the compression pass

__device__ __forceinline__ int parent_of(const int* parent, int x) {
  return *reinterpret_cast<const volatile int*>(parent + x);
}

// root of x, halving the path on the way (each write replaces a parent by an
// ancestor, so concurrent finds and unions stay consistent)
__device__ __forceinline__ int find_root(int* parent, int x) {
  for (;;) {
    const int p = parent_of(parent, x);
    if (p == x) return x;
    const int gp = parent_of(parent, p);
    if (gp == p) return p;
    *reinterpret_cast<volatile int*>(parent + x) = gp;
    x = gp;
  }
}

// Join the sets of a (a member of this thread's set, not necessarily its
// root) and b (j's root).  Only a root is ever re-parented, and only onto a
// smaller index, so parent pointers always decrease (no cycle can form, every
// walk ends) and each component ends with its smallest index as root; the
// node a root is hooked under need not be a root itself.  Returns a member of
// the merged set.
__device__ __forceinline__ int unite(int* parent, int a, int b, int* err) {
  for (int step = 0; a != b; ++step) {
    if (step == kUnionSteps) {
      atomicCAS(err, 0, (int)CIL_ERR_TIMEOUT);
      return a;
    }
    const int lo = min(a, b), hi = max(a, b);
    const int old = atomicCAS(parent + hi, hi, lo);
    if (old == hi) return lo;
    // hi is no longer a root: continue from its root (a smaller index)
    if (hi == a) a = find_root(parent, old);
    else b = find_root(parent, old);
  }
  return a;
}

__device__ __forceinline__ float dot3_rn(float ax, float ay, float az, float bx, float by, float bz) {
  return __fadd_rn(__fadd_rn(__fmul_rn(ax, bx), __fmul_rn(ay, by)), __fmul_rn(az, bz));
}

__global__ void k_seg_init(int* parent, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) parent[i] = (int)i;
}

// One thread per point i, one union per kept edge among list entries
// [m0, m1).  ra tracks a member of i's set (its parent to begin with); an
// edge whose far end hangs directly below ra (or is ra) is skipped with one
// load, which after a compression pass is nearly every edge inside a grown
// component.
__global__ void __launch_bounds__(kSegThreads) k_seg_union(const int* __restrict__ idx, int k,
                                                           int m0, int m1,
                                                           const float* __restrict__ xyz,
                                                           const float* __restrict__ nrm, int64_t n,
                                                           const float4* __restrict__ sorted,
                                                           float cos_t, float r2, int* parent,
                                                           int* err) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  // points in the grid's Morton order: a warp's points are a compact blob
  // whose neighbour lists overlap, so their normals and parents hit in L1
  const int64_t i = sorted ? (int64_t)__float_as_int(__ldg(sorted + t).w) : t;
  const float nx = __ldg(nrm + 3 * i), ny = __ldg(nrm + 3 * i + 1), nz = __ldg(nrm + 3 * i + 2);
  const float px = __ldg(xyz + 3 * i), py = __ldg(xyz + 3 * i + 1), pz = __ldg(xyz + 3 * i + 2);
  int ra = parent_of(parent, (int)i);
  for (int m = m0; m < m1; ++m) {
    const int j = __ldg(idx + i * k + m);
    if (j < 0 || j == (int)i) continue;
    const float dot = dot3_rn(nx, ny, nz, __ldg(nrm + 3 * (int64_t)j),
                              __ldg(nrm + 3 * (int64_t)j + 1), __ldg(nrm + 3 * (int64_t)j + 2));
    if (!(isfinite(dot) && dot >= cos_t)) continue;
    if (r2 > 0.0f) {
      const float dx = __fsub_rn(px, __ldg(xyz + 3 * (int64_t)j));
      const float dy = __fsub_rn(py, __ldg(xyz + 3 * (int64_t)j + 1));
      const float dz = __fsub_rn(pz, __ldg(xyz + 3 * (int64_t)j + 2));
      if (!(dot3_rn(dx, dy, dz, dx, dy, dz) <= r2)) continue;
    }
    if (j == ra) continue;
    const int pj = parent_of(parent, j);
    if (pj == ra) continue;
    const int rb = pj == j ? j : find_root(parent, pj);
    ra = unite(parent, ra, rb, err);
  }
}

// every point straight below its root (no union runs meanwhile)
__global__ void k_seg_compress(int* parent, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) parent[i] = find_root(parent, (int)i);
}

__global__ void k_seg_labels(int* parent, int64_t n, int32_t* labels, unsigned long long* count) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int roots = 0;
  if (i < n) {
    const int r = find_root(parent, (int)i);
    labels[i] = r;
    roots = r == (int)i;
  }
  const int c = __syncthreads_count(roots);
  if (threadIdx.x == 0 && c) atomicAdd(count, (unsigned long long)c);
}

cil_status launch_segment(const int* knn_idx, int k, const float* xyz, const float* nrm, int64_t n,
                          const float4* sorted, float cos_t, float r2, int* parent, int32_t* labels,
                          unsigned long long* count, int* err, cudaStream_t s) {
  TimedRegion timer("segment", s);
  note_launches(5);
  const int blocks = ceil_div(n, kSegThreads);
  k_seg_init<<<blocks, kSegThreads, 0, s>>>(parent, n);
  // the nearest few edges first (mostly distinct small trees, little
  // contention), every point then straight below its root, then the rest
  const int mA = k < kSegFirst ? k : kSegFirst;
  k_seg_union<<<blocks, kSegThreads, 0, s>>>(knn_idx, k, 0, mA, xyz, nrm, n, sorted, cos_t, r2,
                                             parent, err);
  k_seg_compress<<<blocks, kSegThreads, 0, s>>>(parent, n);
  k_seg_union<<<blocks, kSegThreads, 0, s>>>(knn_idx, k, mA, k, xyz, nrm, n, sorted, cos_t, r2,
                                             parent, err);
  if (cudaMemsetAsync(count, 0, sizeof(unsigned long long), s) != cudaSuccess) return CIL_ERR_CUDA;
  k_seg_labels<<<blocks, kSegThreads, 0, s>>>(parent, n, labels, count);
  return cudaGetLastError() == cudaSuccess ? CIL_OK : CIL_ERR_CUDA;
}

}  // namespace cil
