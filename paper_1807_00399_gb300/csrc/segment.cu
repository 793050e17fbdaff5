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
// Components by a concurrent union-find: every root is hooked onto the
// smaller of two roots with an atomic compare-and-swap, so parents always
// have smaller indices than their children, every find terminates, and each
// component ends with its smallest index as root -- the label, independent of
// the order in which edges were processed.
#include "cil_host.h"
#include "cil_kernels.h"

namespace cil {

constexpr int kSegThreads = 256;
constexpr int kUnionSteps = 1 << 20;  // a union needs far fewer; the cap only bounds the loop

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

__device__ __forceinline__ void unite(int* parent, int a, int b, int* err) {
  int ra = find_root(parent, a), rb = find_root(parent, b);
  for (int step = 0; ra != rb; ++step) {
    if (step == kUnionSteps) {
      atomicCAS(err, 0, (int)CIL_ERR_TIMEOUT);
      return;
    }
    if (ra > rb) {
      const int t = ra;
      ra = rb;
      rb = t;
    }
    const int old = atomicCAS(parent + rb, rb, ra);
    if (old == rb) return;
    rb = find_root(parent, old);  // rb was hooked meanwhile: go on from its root
    ra = find_root(parent, ra);
  }
}

__device__ __forceinline__ float dot3_rn(float ax, float ay, float az, float bx, float by, float bz) {
  return __fadd_rn(__fadd_rn(__fmul_rn(ax, bx), __fmul_rn(ay, by)), __fmul_rn(az, bz));
}

__global__ void k_seg_init(int* parent, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) parent[i] = (int)i;
}

__global__ void __launch_bounds__(kSegThreads) k_seg_union(const int* __restrict__ idx, int k,
                                                           const float* __restrict__ xyz,
                                                           const float* __restrict__ nrm, int64_t n,
                                                           float cos_t, float r2, int* parent,
                                                           int* err) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float nx = __ldg(nrm + 3 * i), ny = __ldg(nrm + 3 * i + 1), nz = __ldg(nrm + 3 * i + 2);
  const float px = __ldg(xyz + 3 * i), py = __ldg(xyz + 3 * i + 1), pz = __ldg(xyz + 3 * i + 2);
  for (int m = 0; m < k; ++m) {
    const int j = __ldg(idx + i * k + m);
    if (j < 0 || j == (int)i) continue;
    const float dot = dot3_rn(nx, ny, nz, __ldg(nrm + 3 * (int64_t)j), __ldg(nrm + 3 * (int64_t)j + 1),
                              __ldg(nrm + 3 * (int64_t)j + 2));
    if (!(isfinite(dot) && dot >= cos_t)) continue;
    if (r2 > 0.0f) {
      const float dx = __fsub_rn(px, __ldg(xyz + 3 * (int64_t)j));
      const float dy = __fsub_rn(py, __ldg(xyz + 3 * (int64_t)j + 1));
      const float dz = __fsub_rn(pz, __ldg(xyz + 3 * (int64_t)j + 2));
      if (!(dot3_rn(dx, dy, dz, dx, dy, dz) <= r2)) continue;
    }
    unite(parent, (int)i, j, err);
  }
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
                          float cos_t, float r2, int* parent, int32_t* labels,
                          unsigned long long* count, int* err, cudaStream_t s) {
  TimedRegion timer("segment", s);
  note_launches(3);
  const int blocks = ceil_div(n, kSegThreads);
  k_seg_init<<<blocks, kSegThreads, 0, s>>>(parent, n);
  k_seg_union<<<blocks, kSegThreads, 0, s>>>(knn_idx, k, xyz, nrm, n, cos_t, r2, parent, err);
  if (cudaMemsetAsync(count, 0, sizeof(unsigned long long), s) != cudaSuccess) return CIL_ERR_CUDA;
  k_seg_labels<<<blocks, kSegThreads, 0, s>>>(parent, n, labels, count);
  return cudaGetLastError() == cudaSuccess ? CIL_OK : CIL_ERR_CUDA;
}

}  // namespace cil
