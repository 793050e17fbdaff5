// cil_dev.cuh -- device-side building blocks of the grid index and searches.
//
// Spatial index (replaces the paper's kd-tree, Sec. 3 "KDTree"):
//   * every cloud gets a cubic "fine" lattice over its bounding box with
//     1024 cells on the longest axis (fine = max_extent / 1023);
//   * points are sorted (stable LSD radix sort) by the 30-bit Morton code of
//     their fine cell, with the cloud id above bit 30 in batched mode;
//   * a search grid of level L uses cells of edge fine * 2^L; each such cell is
//     a Morton prefix, hence a contiguous run of the sorted points;
//   * an open-addressing hash table maps (cloud, cell x, y, z) -> (start, count).
// Searches visit cells in growing Chebyshev shells around the query's cell and
// stop only when no unvisited cell can hold a closer point (exact results).
#pragma once

#include <type_traits>
#include <cuda_runtime.h>
#include <stdint.h>

namespace cil {

typedef unsigned long long u64;

constexpr u64 kEmptyKey = ~0ull;
constexpr int kFineBits = 10;          // fine lattice: 1024 cells per axis
constexpr int kFineDim = 1 << kFineBits;

// Per-cloud parameters, written on the device by the grid build.
struct GridParams {
  float o[3];          // origin = bounding-box minimum
  float fine;          // fine cell edge
  float inv_fine;      // 1 / fine
  float eps;           // absolute slack for cell-boundary tests
  float bmax[3];       // bounding-box maximum
  int hi_fine[3];      // fine cell index of bmax per axis (<= 1023)
  int level;           // search-grid level: cell edge = fine * 2^level
  float cell;          // fine * 2^level
  int n;               // points of this cloud
  int start;           // offset of this cloud in the concatenated arrays
  unsigned bbox_enc[6];// order-preserving integer encodings (min x,y,z, max x,y,z)
  int nonfinite;       // number of non-finite coordinates seen
  int pad[3];
};

struct __align__(16) CellEntry {
  u64 key;
  int start;
  int count;
};

// Read-only view of a built grid (passed by value to kernels).
struct GridView {
  const GridParams* prm;  // [n_clouds]
  const float4* pts;      // sorted points: x, y, z, local index (int bits)
  const CellEntry* tab;   // hash table of the k-NN level
  unsigned mask;          // table size - 1 (power of two)
};

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned float_to_ordered(float f) {
  unsigned u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ordered_to_float(unsigned u) {
  return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

// spread the low 10 bits of v so that bit i lands on bit 3i
__device__ __forceinline__ unsigned spread3(unsigned v) {
  v &= 0x3ffu;
  v = (v | (v << 16)) & 0x030000ffu;
  v = (v | (v << 8)) & 0x0300f00fu;
  v = (v | (v << 4)) & 0x030c30c3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}
__device__ __forceinline__ unsigned compact3(unsigned v) {
  v &= 0x09249249u;
  v = (v | (v >> 2)) & 0x030c30c3u;
  v = (v | (v >> 4)) & 0x0300f00fu;
  v = (v | (v >> 8)) & 0x030000ffu;
  v = (v | (v >> 16)) & 0x000003ffu;
  return v;
}
__device__ __forceinline__ unsigned morton3(unsigned x, unsigned y, unsigned z) {
  return spread3(x) | (spread3(y) << 1) | (spread3(z) << 2);
}

// fine lattice coordinate of one axis (clamped into [0, 1023]);
// NaN maps to 0, so corrupt inputs never index out of range
__device__ __forceinline__ int fine_coord(float v, float o, float inv_fine) {
  float f = floorf((v - o) * inv_fine);
  f = fminf(fmaxf(f, 0.0f), (float)(kFineDim - 1));
  return (int)f;
}

// Cell-key hash on 32-bit arithmetic: fold the key's high word into the low
// one with a Fibonacci multiplier, then the "lowbias32" integer mixer
// (xorshift-multiply rounds, C. Wellons' hash-prospector).
__device__ __forceinline__ unsigned hash_key(u64 k) {
  unsigned h = (unsigned)k ^ ((unsigned)(k >> 32) * 0x9E3779B1u);
  h ^= h >> 16;
  h *= 0x7FEB352Du;
  h ^= h >> 15;
  h *= 0x846CA68Bu;
  h ^= h >> 16;
  return h;
}

// hash-table key of a cell: level (4 bits), cloud (11 bits), z, y, x (10 bits each)
__device__ __forceinline__ u64 cell_key(int level, int cloud, int x, int y, int z) {
  return ((u64)(unsigned)level << 41) | ((u64)(unsigned)cloud << 30) | ((u64)(unsigned)z << 20) |
         ((u64)(unsigned)y << 10) | (u64)(unsigned)x;
}

// levels searched by k-NN queries: the cloud's level and up to three coarser
// ones (x8 cell edge each), all hashed in the k-NN table
constexpr int kEscalateStep = 3;
constexpr int kRingCap = 3;  // rings searched at one level before escalating
__device__ __forceinline__ int next_level(int lvl) { return min(lvl + kEscalateStep, kFineBits); }

__device__ __forceinline__ bool table_lookup(const CellEntry* tab, unsigned mask, u64 K, int& start,
                                             int& count) {
  unsigned h = hash_key(K) & mask;
  for (unsigned probe = 0; probe <= mask; ++probe) {
    const int4 v = __ldg(reinterpret_cast<const int4*>(tab + h));
    const u64 key = (u64)(unsigned)v.x | ((u64)(unsigned)v.y << 32);
    if (key == K) {
      start = v.z;
      count = v.w;
      return true;
    }
    if (key == kEmptyKey) return false;
    h = (h + 1) & mask;
  }
  return false;
}

__device__ __forceinline__ bool cell_lookup(const GridView& g, u64 K, int& start, int& count) {
  return table_lookup(g.tab, g.mask, K, start, count);
}

// squared distance of two points from exact per-axis differences
__device__ __forceinline__ float sqdist(float px, float py, float pz, float qx, float qy, float qz) {
  const float dx = px - qx, dy = py - qy, dz = pz - qz;
  return fmaf(dz, dz, fmaf(dy, dy, dx * dx));
}

// (squared distance, index) packed so that unsigned order == lexicographic order
// (squared distances are >= 0, whose IEEE bit patterns are monotone)
__device__ __forceinline__ u64 pack_key(float d2, int idx) {
  return ((u64)__float_as_uint(d2) << 32) | (u64)(unsigned)idx;
}
__device__ __forceinline__ float key_d2(u64 k) { return __uint_as_float((unsigned)(k >> 32)); }
__device__ __forceinline__ int key_idx(u64 k) { return (int)(unsigned)(k & 0xffffffffu); }

// Visit the points [s, s + n) of the sorted array in chunks of W whose loads
// are issued together (the loop is otherwise bound by load latency).
template <int W = 4, class F>
__device__ __forceinline__ void for_points(const float4* pts, int s, int n, F&& fn) {
  const int e = s + n;
  for (int j = s; j < e; j += W) {
    float4 p[W];
#pragma unroll
    for (int u = 0; u < W; ++u)
      if (j + u < e) p[u] = __ldg(pts + j + u);
#pragma unroll
    for (int u = 0; u < W; ++u)
      if (j + u < e) fn(p[u], j + u);
  }
}

// squared distance from q to the box [lo, hi] (per axis), 0 inside
__device__ __forceinline__ float box_d2(const float q[3], const float lo[3], const float hi[3]) {
  float s = 0.0f;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float d = fmaxf(fmaxf(lo[a] - q[a], q[a] - hi[a]), 0.0f);
    s = fmaf(d, d, s);
  }
  return s;
}

// Geometry of one cloud's search grid at its level, in registers.
struct CellFrame {
  float o[3];
  float c;      // cell edge
  float eps;
  int hi[3];    // largest occupied-range cell index per axis
  int level;
  int cloud;

  __device__ __forceinline__ void load(const GridParams& P, int cloud_id) {
    load_level(P, cloud_id, P.level, P.cell);
  }
  __device__ __forceinline__ void load_level(const GridParams& P, int cloud_id, int lvl, float cell) {
    o[0] = P.o[0];
    o[1] = P.o[1];
    o[2] = P.o[2];
    c = cell;
    eps = P.eps;
    level = lvl;
    hi[0] = P.hi_fine[0] >> level;
    hi[1] = P.hi_fine[1] >> level;
    hi[2] = P.hi_fine[2] >> level;
    cloud = cloud_id;
  }
  __device__ __forceinline__ int cell_of(float v, int a, float inv_fine) const {
    int f = fine_coord(v, o[a], inv_fine) >> level;
    return min(f, hi[a]);
  }
  // squared distance from q to the cells [lo_c, hi_c] (inclusive indices),
  // padded by eps
  __device__ __forceinline__ float range_d2(const float q[3], const int lo_c[3],
                                            const int hi_c[3]) const {
    float lo[3], hh[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      lo[a] = fmaf((float)lo_c[a], c, o[a]) - eps;
      hh[a] = fmaf((float)(hi_c[a] + 1), c, o[a]) + eps;
    }
    return box_d2(q, lo, hh);
  }
  // squared distance from q to the part of the grid outside the explored cube
  // [e0, e1] (cell indices, may exceed the grid); +inf when nothing is left
  __device__ __forceinline__ float unexplored_d2(const float q[3], const int e0[3],
                                                 const int e1[3]) const {
    float best = __int_as_float(0x7f800000);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      int lo_c[3] = {0, 0, 0};
      int hi_c[3] = {hi[0], hi[1], hi[2]};
      if (e0[a] > 0) {  // slab below the explored cube on axis a
        hi_c[a] = e0[a] - 1;
        best = fminf(best, range_d2(q, lo_c, hi_c));
        hi_c[a] = hi[a];
      }
      if (e1[a] < hi[a]) {  // slab above
        lo_c[a] = e1[a] + 1;
        best = fminf(best, range_d2(q, lo_c, hi_c));
      }
    }
    return best;
  }
};

// Iterate (x, y, z) over every cell of the Chebyshev shell of radius r around
// (cx, cy, cz) that lies in the grid.  Rows on the shell's faces are walked
// cell by cell, interior rows contribute their two end cells (stride 2r).
// Written as a loop header/footer pair so the body stays inline and all search
// state stays in registers; `continue` in the body skips to the next cell.
#define CIL_SHELL_FOR(f, cx, cy, cz, r, x, y, z)                                      \
  for (int z = max((cz) - (r), 0), z##_end = min((cz) + (r), (f).hi[2]); z <= z##_end; ++z) \
    for (int y = max((cy) - (r), 0), y##_end = min((cy) + (r), (f).hi[1]); y <= y##_end; ++y) \
      for (int x##_edge = (z == (cz) - (r)) || (z == (cz) + (r)) || (y == (cy) - (r)) ||      \
                          (y == (cy) + (r)),                                                \
               x = x##_edge ? max((cx) - (r), 0) : (cx) - (r),                              \
               x##_end = x##_edge ? min((cx) + (r), (f).hi[0]) : (cx) + (r),               \
               x##_step = x##_edge ? 1 : 2 * (r);                                           \
           x <= x##_end; x += x##_step)                                                     \
        if (x >= 0 && x <= (f).hi[0])

// ---------------------------------------------------------------------------
// register top-k: sorted ascending array of packed (d2, idx) keys
// ---------------------------------------------------------------------------
template <int KMAX>
struct TopK {
  u64 v[KMAX];
  u64 thr;  // == v[k-1]: a candidate enters only if its key is smaller
  int k;

  __device__ __forceinline__ void init(int kk) {
    k = kk;
#pragma unroll
    for (int j = 0; j < KMAX; ++j) v[j] = kEmptyKey;
    thr = kEmptyKey;
  }
  // branch-free insertion into the ascending list (selects, no predicated
  // stores, so the array stays in registers).  The whole KMAX-slot list stays
  // sorted, so its first k slots are the k smallest keys seen; thr = v[k-1].
  __device__ __forceinline__ void push(u64 key) {
    if (key < thr) {
#pragma unroll
      for (int j = KMAX - 1; j > 0; --j) {
        const u64 prev = v[j - 1];
        const u64 cur = v[j];
        v[j] = (key < prev) ? prev : ((key < cur) ? key : cur);
      }
      v[0] = (key < v[0]) ? key : v[0];
      if (k == KMAX) {
        thr = v[KMAX - 1];
      } else {
        u64 t = v[0];
#pragma unroll
        for (int j = 1; j < KMAX; ++j) t = (j < k) ? v[j] : t;
        thr = t;
      }
    }
  }
  __device__ __forceinline__ bool full() const { return thr != kEmptyKey; }
  __device__ __forceinline__ float thr_d2() const { return key_d2(thr); }
  __device__ __forceinline__ void bind(u64*, int) {}
  __device__ __forceinline__ void finish() {}
  // slot j (a compile-time index in unrolled loops): ascending order
  __device__ __forceinline__ u64 key_at(int j) const { return v[j]; }
};

// The k smallest keys as a binary max-heap in shared memory (this thread's
// slot j at h[j * stride], so the lanes of a warp touch consecutive words).
// A key below the root replaces it and sifts down: at most log2(k) levels of
// two loads and one store, where the register list above shifts all KMAX
// slots with integer selects -- for large k that shifting saturates the
// integer pipe.  Keys are unique (the index fills the low word), so the set
// of the k smallest is well defined; heap order is not ascending until
// finish() sorts it.
template <int KMAX>
struct TopKHeap {
  u64* h;
  u64 thr;  // the root once k keys are held, else kEmptyKey
  int stride, k, cnt;

  __device__ __forceinline__ void bind(u64* base, int st) {
    h = base;
    stride = st;
  }
  __device__ __forceinline__ void init(int kk) {
    k = kk;
    cnt = 0;
    thr = kEmptyKey;
  }
  __device__ __forceinline__ u64 at(int j) const { return h[j * stride]; }
  __device__ __forceinline__ void put(int j, u64 x) { h[j * stride] = x; }
  // place `key` at the root of the heap h[0, n) and restore heap order
  __device__ __forceinline__ void sift_down(u64 key, int n) {
    int j = 0;
    for (;;) {
      int c = 2 * j + 1;
      if (c >= n) break;
      u64 cv = at(c);
      if (c + 1 < n) {
        const u64 c2 = at(c + 1);
        if (c2 > cv) {
          cv = c2;
          ++c;
        }
      }
      if (cv <= key) break;
      put(j, cv);
      j = c;
    }
    put(j, key);
  }
  __device__ __forceinline__ void push(u64 key) {
    if (key >= thr) return;
    if (cnt < k) {
      int j = cnt++;
      while (j > 0) {
        const int p = (j - 1) >> 1;
        const u64 pv = at(p);
        if (pv >= key) break;
        put(j, pv);
        j = p;
      }
      put(j, key);
      if (cnt == k) thr = at(0);
    } else {
      sift_down(key, k);
      thr = at(0);
    }
  }
  __device__ __forceinline__ bool full() const { return thr != kEmptyKey; }
  __device__ __forceinline__ float thr_d2() const { return key_d2(thr); }
  // ascending order in place (heap sort of the cnt held keys)
  __device__ __forceinline__ void finish() {
    for (int e = cnt - 1; e > 0; --e) {
      const u64 top = at(0);
      const u64 last = at(e);
      put(e, top);
      sift_down(last, e);
    }
  }
  __device__ __forceinline__ u64 key_at(int j) const { return j < cnt ? at(j) : kEmptyKey; }
};

// Register list for small k, shared-memory heap from kHeapFromK on (a block
// of B threads then needs B * KMAX * 8 bytes of dynamic shared memory).
constexpr int kHeapFromK = 8;
template <int KMAX>
using TopKFor = typename std::conditional<(KMAX >= kHeapFromK), TopKHeap<KMAX>, TopK<KMAX>>::type;
template <int KMAX>
constexpr int topk_smem_per_thread() {
  return KMAX >= kHeapFromK ? KMAX * (int)sizeof(u64) : 0;
}

// Top-k layout picked at run time (a tuning axis; results do not depend on
// it): 0 = by k as TopKFor, 1 = register list, 2 = shared-memory heap.
template <int KMAX, bool HEAP>
using TopKSel = typename std::conditional<HEAP, TopKHeap<KMAX>, TopK<KMAX>>::type;
constexpr bool topk_heap(int kmax, int layout) {
  return layout == 2 || (layout != 1 && kmax >= kHeapFromK);
}

// Exact k nearest neighbours of q among the points of cloud `cloud`.
// Rings of cells are searched at the cloud's level; a search that has not
// proved its k-th distance after kRingCap rings (sparse regions, queries far
// from the cloud) restarts at an 8x coarser level, up to the level whose one
// cell spans the whole cloud, so every query visits at most a few hundred
// cells per level.
template <int KMAX, class Top>
__device__ __forceinline__ void grid_knn(const GridView& g, int cloud, const float q[3], Top& top,
                                         int* visited_cells = nullptr) {
  const GridParams& P = g.prm[cloud];
  const float inv_fine = P.inv_fine;
  int nvis = 0;
  for (int lvl = P.level;; lvl = next_level(lvl)) {
    CellFrame f;
    f.load_level(P, cloud, lvl, ldexpf(P.fine, lvl));
    const int cx = f.cell_of(q[0], 0, inv_fine);
    const int cy = f.cell_of(q[1], 1, inv_fine);
    const int cz = f.cell_of(q[2], 2, inv_fine);
    const int rmax = max(max(max(cx, f.hi[0] - cx), max(cy, f.hi[1] - cy)), max(cz, f.hi[2] - cz));
    const int rcap = lvl >= kFineBits ? rmax : min(rmax, kRingCap);
    top.init(top.k);
    bool done = false;
    for (int r = 0; r <= rcap; ++r) {
      CIL_SHELL_FOR(f, cx, cy, cz, r, x, y, z) {
        if (top.full()) {
          const int c3[3] = {x, y, z};
          if (f.range_d2(q, c3, c3) * (1.0f - 1e-6f) > top.thr_d2()) continue;
        }
        int s, n;
        if (!cell_lookup(g, cell_key(lvl, cloud, x, y, z), s, n)) continue;
        ++nvis;
        for_points(g.pts, s, n, [&](const float4& p, int) {
          top.push(pack_key(sqdist(p.x, p.y, p.z, q[0], q[1], q[2]), __float_as_int(p.w)));
        });
      }
      if (r == rmax) {
        done = true;  // the explored cube holds the whole cloud
        break;
      }
      if (top.full()) {
        const int e0[3] = {cx - r, cy - r, cz - r};
        const int e1[3] = {cx + r, cy + r, cz + r};
        if (top.thr_d2() < f.unexplored_d2(q, e0, e1) * (1.0f - 1e-6f)) {
          done = true;
          break;
        }
      }
    }
    if (done || lvl >= kFineBits) break;
  }
  if (visited_cells) *visited_cells = nvis;
}

// Exact k nearest neighbours of q among the points within squared distance r2
// (inclusive): the search, the pruning and the stopping bound all use
// min(current k-th distance, r2); levels escalate as in grid_knn.
template <int KMAX, class Top>
__device__ __forceinline__ void grid_knn_within(const GridView& g, int cloud, const float q[3],
                                                float r2, Top& top) {
  const GridParams& P = g.prm[cloud];
  const float inv_fine = P.inv_fine;
  for (int lvl = P.level;; lvl = next_level(lvl)) {
    CellFrame f;
    f.load_level(P, cloud, lvl, ldexpf(P.fine, lvl));
    const int cx = f.cell_of(q[0], 0, inv_fine);
    const int cy = f.cell_of(q[1], 1, inv_fine);
    const int cz = f.cell_of(q[2], 2, inv_fine);
    const int rmax = max(max(max(cx, f.hi[0] - cx), max(cy, f.hi[1] - cy)), max(cz, f.hi[2] - cz));
    const int rcap = lvl >= kFineBits ? rmax : min(rmax, kRingCap);
    top.init(top.k);
    bool done = false;
    for (int r = 0; r <= rcap; ++r) {
      CIL_SHELL_FOR(f, cx, cy, cz, r, x, y, z) {
        const float lim = top.full() ? fminf(top.thr_d2(), r2) : r2;
        const int c3[3] = {x, y, z};
        if (f.range_d2(q, c3, c3) * (1.0f - 1e-6f) > lim) continue;
        int s, n;
        if (!cell_lookup(g, cell_key(lvl, cloud, x, y, z), s, n)) continue;
        for_points(g.pts, s, n, [&](const float4& p, int) {
          const float d2 = sqdist(p.x, p.y, p.z, q[0], q[1], q[2]);
          if (d2 <= r2) top.push(pack_key(d2, __float_as_int(p.w)));
        });
      }
      if (r == rmax) {
        done = true;
        break;
      }
      const float lim = top.full() ? fminf(top.thr_d2(), r2) : r2;
      const int e0[3] = {cx - r, cy - r, cz - r};
      const int e1[3] = {cx + r, cy + r, cz + r};
      if (lim < f.unexplored_d2(q, e0, e1) * (1.0f - 1e-6f)) {
        done = true;
        break;
      }
    }
    if (done || lvl >= kFineBits) break;
  }
}

// Exact nearest neighbour of q within squared distance dmax2 (inclusive).
// Returns the packed key, or kEmptyKey when no point lies within dmax2.
__device__ __forceinline__ u64 grid_nn(const GridView& g, int cloud, const float q[3], float dmax2) {
  const GridParams& P = g.prm[cloud];
  CellFrame f;
  f.load(P, cloud);
  const float inv_fine = P.inv_fine;
  const int cx = f.cell_of(q[0], 0, inv_fine);
  const int cy = f.cell_of(q[1], 1, inv_fine);
  const int cz = f.cell_of(q[2], 2, inv_fine);
  const int rmax = max(max(max(cx, f.hi[0] - cx), max(cy, f.hi[1] - cy)), max(cz, f.hi[2] - cz));
  u64 best = kEmptyKey;
  float lim = dmax2;  // min(best d2, dmax2)
  for (int r = 0; r <= rmax; ++r) {
    {
      // the whole shell lies farther than the limit: nothing left to find
      const int e0[3] = {cx - r + 1, cy - r + 1, cz - r + 1};
      const int e1[3] = {cx + r - 1, cy + r - 1, cz + r - 1};
      if (r > 0 && f.unexplored_d2(q, e0, e1) * (1.0f - 1e-6f) > lim) break;
    }
    CIL_SHELL_FOR(f, cx, cy, cz, r, x, y, z) {
      const int c3[3] = {x, y, z};
      if (f.range_d2(q, c3, c3) * (1.0f - 1e-6f) > lim) continue;
      int s, n;
      if (!cell_lookup(g, cell_key(P.level, cloud, x, y, z), s, n)) continue;
      for_points(g.pts, s, n, [&](const float4& p, int) {
        const float d2 = sqdist(p.x, p.y, p.z, q[0], q[1], q[2]);
        if (d2 <= dmax2) {
          const u64 key = pack_key(d2, __float_as_int(p.w));
          if (key < best) {
            best = key;
            lim = fminf(lim, d2);
          }
        }
      });
    }
  }
  return best;
}

// ---------------------------------------------------------------------------
// compensated FP32 summation (error-free TwoSum transformation)
// ---------------------------------------------------------------------------
struct KSum {
  float s, c;
  __device__ __forceinline__ void zero() { s = c = 0.0f; }
  __device__ __forceinline__ void add(float x) {
    const float t = __fadd_rn(s, x);
    const float bp = __fsub_rn(t, s);
    const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(x, bp));
    s = t;
    c = __fadd_rn(c, e);
  }
  __device__ __forceinline__ void merge(float s2, float c2) {
    add(s2);
    c = __fadd_rn(c, c2);
  }
};

// Host-side dispatch of a kernel template on the smallest compiled register
// top-k capacity KM >= k (k in 1..32).
#define CIL_FOR_K(k, CALL)          \
  do {                              \
    if ((k) <= 1) {                 \
      constexpr int KM = 1;         \
      CALL;                         \
    } else if ((k) <= 4) {          \
      constexpr int KM = 4;         \
      CALL;                         \
    } else if ((k) <= 8) {          \
      constexpr int KM = 8;         \
      CALL;                         \
    } else if ((k) <= 10) {         \
      constexpr int KM = 10;        \
      CALL;                         \
    } else if ((k) <= 16) {         \
      constexpr int KM = 16;        \
      CALL;                         \
    } else if ((k) <= 24) {         \
      constexpr int KM = 24;        \
      CALL;                         \
    } else {                        \
      constexpr int KM = 32;        \
      CALL;                         \
    }                               \
  } while (0)

}  // namespace cil
