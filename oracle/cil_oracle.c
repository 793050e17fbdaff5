/*
 * cil_oracle.c -- plain FP64 CPU oracle for the point-cloud hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or calls
 * this file; only the test-suite, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header, table or helper with the CUDA
 * library.
 *
 * Every routine is the plain definition of what the method computes, written
 * for readability rather than speed (the only concession is a thread-parallel
 * loop over independent queries):
 *
 *   oracle_knn          k nearest neighbours by exhaustive search
 *                       (Sec. 3, "KDTree ... k-NN, radius, and hybrid queries")
 *   oracle_knn_kdtree   the same result through a kd-tree (Sec. 2 bundles
 *                       nanoflann for kd-tree queries); validated against the
 *                       exhaustive search by the tests, used for large inputs
 *   oracle_radius       all neighbours within a radius by exhaustive search
 *                       (Sec. 3, radius queries)
 *   oracle_sym3_eigen   cyclic Jacobi eigen-decomposition of a symmetric 3x3
 *   oracle_normals      PCA surface normal + curvature from each point's kNN
 *                       covariance, oriented towards a viewpoint
 *                       (Sec. 3 "surface normal and curvature estimation",
 *                       "Principal Component Analysis"; Sec. 4 10-NN
 *                       neighbourhoods and viewpoint-consistent orientation)
 *   oracle_icp          rigid point-to-plane ICP: alternate nearest-neighbour
 *                       correspondences (with a rejection distance) and a
 *                       linearised point-to-plane Gauss-Newton step, for a
 *                       fixed number of iterations (Sec. 2 ICP base loop,
 *                       Sec. 3 rigid point-to-plane estimator after Low 2004,
 *                       Sec. 4 fixed iteration count and rejection threshold)
 *
 * Conventions shared with the public C-ABI (but not its code): points are
 * float[N][3] interleaved; input floats are promoted exactly to double and all
 * arithmetic is FP64; neighbour lists are ordered by (squared distance, index)
 * ascending; missing neighbours (k > n_ref) are padded with index -1 and
 * distance +inf; the rigid transform is a row-major 4x4 double matrix mapping
 * source coordinates to target coordinates.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

/* ------------------------------------------------------------------------- */
/* thread-parallel loop over [0, n) in contiguous chunks                      */
/* ------------------------------------------------------------------------- */
typedef void (*range_fn)(void *ctx, int64_t lo, int64_t hi, int tid);

typedef struct {
  range_fn fn;
  void *ctx;
  int64_t lo, hi;
  int tid;
} range_job;

static void *range_worker(void *arg) {
  range_job *j = (range_job *)arg;
  j->fn(j->ctx, j->lo, j->hi, j->tid);
  return NULL;
}

int oracle_default_threads(void) {
  long c = sysconf(_SC_NPROCESSORS_ONLN);
  return c > 0 ? (int)c : 1;
}

static int clamp_threads(int nt) {
  if (nt <= 0) nt = oracle_default_threads();
  if (nt > 256) nt = 256;
  return nt;
}

static void parallel_for(int64_t n, int nthreads, range_fn fn, void *ctx) {
  nthreads = clamp_threads(nthreads);
  if (n < 2 * (int64_t)nthreads || nthreads == 1) {
    fn(ctx, 0, n, 0);
    return;
  }
  pthread_t th[256];
  range_job jobs[256];
  for (int t = 0; t < nthreads; ++t) {
    jobs[t].fn = fn;
    jobs[t].ctx = ctx;
    jobs[t].lo = n * t / nthreads;
    jobs[t].hi = n * (t + 1) / nthreads;
    jobs[t].tid = t;
    pthread_create(&th[t], NULL, range_worker, &jobs[t]);
  }
  for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
}

/* ------------------------------------------------------------------------- */
/* squared Euclidean distance in FP64 between two float[3] points             */
/* ------------------------------------------------------------------------- */
static double dist2(const float *a, const float *b) {
  double dx = (double)a[0] - (double)b[0];
  double dy = (double)a[1] - (double)b[1];
  double dz = (double)a[2] - (double)b[2];
  return dx * dx + dy * dy + dz * dz;
}

/* (d2, idx) lexicographic "less than" */
static int pair_less(double da, int64_t ia, double db, int64_t ib) {
  return da < db || (da == db && ia < ib);
}

/* Insert (d, i) into the sorted list (len entries, capacity k). */
static void topk_insert(double *d, int32_t *idx, int *len, int k, double dn, int32_t in) {
  int n = *len;
  if (n == k && !pair_less(dn, in, d[k - 1], idx[k - 1])) return;
  int pos = (n < k) ? n : k - 1;
  while (pos > 0 && pair_less(dn, in, d[pos - 1], idx[pos - 1])) {
    d[pos] = d[pos - 1];
    idx[pos] = idx[pos - 1];
    --pos;
  }
  d[pos] = dn;
  idx[pos] = in;
  if (n < k) *len = n + 1;
}

static void pad_topk(double *d, int32_t *idx, int len, int k) {
  for (int j = len; j < k; ++j) {
    d[j] = INFINITY;
    idx[j] = -1;
  }
}

/* ------------------------------------------------------------------------- */
/* kNN by exhaustive search                                                   */
/* ------------------------------------------------------------------------- */
typedef struct {
  const float *ref, *qry;
  int64_t n_ref;
  int k;
  int32_t *out_idx;
  double *out_d2;
} knn_ctx;

static void knn_range(void *vctx, int64_t lo, int64_t hi, int tid) {
  (void)tid;
  knn_ctx *c = (knn_ctx *)vctx;
  for (int64_t q = lo; q < hi; ++q) {
    double *d = c->out_d2 + q * c->k;
    int32_t *ix = c->out_idx + q * c->k;
    int len = 0;
    for (int64_t i = 0; i < c->n_ref; ++i)
      topk_insert(d, ix, &len, c->k, dist2(c->qry + 3 * q, c->ref + 3 * i), (int32_t)i);
    pad_topk(d, ix, len, c->k);
  }
}

int oracle_knn(const float *ref, int64_t n_ref, const float *qry, int64_t n_qry, int k,
               int32_t *out_idx, double *out_d2, int n_threads) {
  if (k <= 0 || n_ref < 0 || n_qry < 0) return 1;
  knn_ctx c = {ref, qry, n_ref, k, out_idx, out_d2};
  parallel_for(n_qry, n_threads, knn_range, &c);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* kd-tree (exact kNN; a faster route to the same answer for big inputs)       */
/* ------------------------------------------------------------------------- */
typedef struct {
  int32_t lo, hi;    /* range in the permutation */
  int32_t left, right; /* child nodes or -1 */
  int axis;
  double split;
} kd_node;

typedef struct {
  const float *pts;
  int32_t *perm;
  kd_node *nodes;
  int32_t n_nodes, cap;
} kd_tree;

static const float *kd_pt(const kd_tree *t, int32_t j) { return t->pts + 3 * (int64_t)t->perm[j]; }

/* quickselect on perm[lo,hi) so that perm[mid] holds the median along axis */
static void kd_select(kd_tree *t, int32_t lo, int32_t hi, int32_t mid, int axis) {
  while (hi - lo > 1) {
    double pivot = kd_pt(t, lo + (hi - lo) / 2)[axis];
    int32_t i = lo, j = hi - 1;
    while (i <= j) {
      while (kd_pt(t, i)[axis] < pivot) ++i;
      while (kd_pt(t, j)[axis] > pivot) --j;
      if (i <= j) {
        int32_t tmp = t->perm[i];
        t->perm[i] = t->perm[j];
        t->perm[j] = tmp;
        ++i;
        --j;
      }
    }
    if (mid <= j) hi = j + 1;
    else if (mid >= i) lo = i;
    else return;
  }
}

static int32_t kd_build(kd_tree *t, int32_t lo, int32_t hi) {
  int32_t id = t->n_nodes++;
  kd_node *nd = &t->nodes[id];
  nd->lo = lo;
  nd->hi = hi;
  nd->left = nd->right = -1;
  nd->axis = 0;
  nd->split = 0;
  if (hi - lo <= 8) return id;
  double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int32_t j = lo; j < hi; ++j)
    for (int a = 0; a < 3; ++a) {
      double v = kd_pt(t, j)[a];
      if (v < mn[a]) mn[a] = v;
      if (v > mx[a]) mx[a] = v;
    }
  int axis = 0;
  for (int a = 1; a < 3; ++a)
    if (mx[a] - mn[a] > mx[axis] - mn[axis]) axis = a;
  if (mx[axis] - mn[axis] <= 0) return id; /* all points coincide: keep as leaf */
  int32_t mid = lo + (hi - lo) / 2;
  kd_select(t, lo, hi, mid, axis);
  double split = kd_pt(t, mid)[axis];
  int32_t l = kd_build(t, lo, mid);
  int32_t r = kd_build(t, mid, hi);
  nd = &t->nodes[id];
  nd->axis = axis;
  nd->split = split;
  nd->left = l;
  nd->right = r;
  return id;
}

static int kd_init(kd_tree *t, const float *pts, int64_t n) {
  t->pts = pts;
  t->perm = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  t->cap = (int32_t)(2 * n / 4 + 64);
  t->nodes = (kd_node *)malloc(sizeof(kd_node) * (size_t)t->cap * 2);
  t->cap *= 2;
  t->n_nodes = 0;
  if (!t->perm || !t->nodes) return 1;
  for (int64_t i = 0; i < n; ++i) t->perm[i] = (int32_t)i;
  if (n > 0) kd_build(t, 0, (int32_t)n);
  return 0;
}

static void kd_free(kd_tree *t) {
  free(t->perm);
  free(t->nodes);
}

/* Points on the left child have coordinate <= split, on the right >= split.
 * A subtree is skipped only when the squared distance to its half-space is
 * strictly above the current k-th distance (with a relative margin), so ties
 * that the exhaustive search would see are never pruned away. */
static void kd_knn(const kd_tree *t, int32_t node, const float *q, double *d, int32_t *ix, int *len,
                   int k) {
  const kd_node *nd = &t->nodes[node];
  if (nd->left < 0) {
    for (int32_t j = nd->lo; j < nd->hi; ++j) topk_insert(d, ix, len, k, dist2(q, kd_pt(t, j)), t->perm[j]);
    return;
  }
  double diff = (double)q[nd->axis] - nd->split;
  int32_t near = diff <= 0 ? nd->left : nd->right;
  int32_t far = diff <= 0 ? nd->right : nd->left;
  kd_knn(t, near, q, d, ix, len, k);
  double worst = (*len < k) ? INFINITY : d[k - 1];
  if (diff * diff <= worst * (1.0 + 1e-12)) kd_knn(t, far, q, d, ix, len, k);
}

typedef struct {
  const kd_tree *t;
  const float *qry;
  int k;
  int32_t *out_idx;
  double *out_d2;
} kdq_ctx;

static void kdq_range(void *vctx, int64_t lo, int64_t hi, int tid) {
  (void)tid;
  kdq_ctx *c = (kdq_ctx *)vctx;
  for (int64_t q = lo; q < hi; ++q) {
    double *d = c->out_d2 + q * c->k;
    int32_t *ix = c->out_idx + q * c->k;
    int len = 0;
    if (c->t->n_nodes > 0) kd_knn(c->t, 0, c->qry + 3 * q, d, ix, &len, c->k);
    pad_topk(d, ix, len, c->k);
  }
}

int oracle_knn_kdtree(const float *ref, int64_t n_ref, const float *qry, int64_t n_qry, int k,
                      int32_t *out_idx, double *out_d2, int n_threads) {
  if (k <= 0 || n_ref < 0 || n_qry < 0 || n_ref > INT32_MAX) return 1;
  kd_tree t;
  if (kd_init(&t, ref, n_ref)) {
    kd_free(&t);
    return 2;
  }
  kdq_ctx c = {&t, qry, k, out_idx, out_d2};
  parallel_for(n_qry, n_threads, kdq_range, &c);
  kd_free(&t);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* radius search by exhaustive search: CSR output, rows sorted by (d2, idx)    */
/* Two calls: with out_idx == NULL only the per-row counts are written to      */
/* offsets[1..n_qry] (offsets[0] = 0, prefix-summed); then a second call fills */
/* idx/d2 using those offsets.                                                 */
/* ------------------------------------------------------------------------- */
typedef struct {
  const float *ref, *qry;
  int64_t n_ref;
  double r2;
  int64_t *offsets;
  int32_t *out_idx;
  double *out_d2;
} rad_ctx;

static int cmp_pair(const void *a, const void *b) {
  const double *x = (const double *)a, *y = (const double *)b;
  if (x[0] < y[0]) return -1;
  if (x[0] > y[0]) return 1;
  return (x[1] < y[1]) ? -1 : (x[1] > y[1]);
}

static void rad_range(void *vctx, int64_t lo, int64_t hi, int tid) {
  (void)tid;
  rad_ctx *c = (rad_ctx *)vctx;
  for (int64_t q = lo; q < hi; ++q) {
    if (!c->out_idx) {
      int64_t cnt = 0;
      for (int64_t i = 0; i < c->n_ref; ++i)
        if (dist2(c->qry + 3 * q, c->ref + 3 * i) <= c->r2) ++cnt;
      c->offsets[q + 1] = cnt;
    } else {
      int64_t b = c->offsets[q], e = c->offsets[q + 1];
      double *tmp = (double *)malloc(sizeof(double) * 2 * (size_t)(e - b + 1));
      int64_t m = 0;
      for (int64_t i = 0; i < c->n_ref && m < e - b; ++i) {
        double d = dist2(c->qry + 3 * q, c->ref + 3 * i);
        if (d <= c->r2) {
          tmp[2 * m] = d;
          tmp[2 * m + 1] = (double)i;
          ++m;
        }
      }
      qsort(tmp, (size_t)m, 2 * sizeof(double), cmp_pair);
      for (int64_t j = 0; j < m; ++j) {
        c->out_d2[b + j] = tmp[2 * j];
        c->out_idx[b + j] = (int32_t)tmp[2 * j + 1];
      }
      free(tmp);
    }
  }
}

int oracle_radius(const float *ref, int64_t n_ref, const float *qry, int64_t n_qry, double r,
                  int64_t *offsets, int32_t *out_idx, double *out_d2, int n_threads) {
  if (r < 0 || n_ref < 0 || n_qry < 0) return 1;
  rad_ctx c = {ref, qry, n_ref, r * r, offsets, out_idx, out_d2};
  if (!out_idx) {
    offsets[0] = 0;
    parallel_for(n_qry, n_threads, rad_range, &c);
    for (int64_t q = 0; q < n_qry; ++q) offsets[q + 1] += offsets[q];
  } else {
    parallel_for(n_qry, n_threads, rad_range, &c);
  }
  return 0;
}

/* ------------------------------------------------------------------------- */
/* symmetric 3x3 eigen-decomposition by cyclic Jacobi rotations               */
/* C given as (c00, c01, c02, c11, c12, c22).  Eigenvalues ascending; the      */
/* eigenvector of evals[j] is column j of evecs (row-major 3x3).               */
/* ------------------------------------------------------------------------- */
int oracle_sym3_eigen(const double *Cu, double *evals, double *evecs) {
  double a[3][3] = {{Cu[0], Cu[1], Cu[2]}, {Cu[1], Cu[3], Cu[4]}, {Cu[2], Cu[4], Cu[5]}};
  double v[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  double fro = 0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) fro += a[i][j] * a[i][j];
  fro = sqrt(fro);
  for (int sweep = 0; sweep < 64; ++sweep) {
    double off = sqrt(2.0 * (a[0][1] * a[0][1] + a[0][2] * a[0][2] + a[1][2] * a[1][2]));
    if (off <= 1e-15 * fro || off == 0.0) break;
    for (int p = 0; p < 2; ++p)
      for (int q = p + 1; q < 3; ++q) {
        if (a[p][q] == 0.0) continue;
        /* rotation that annihilates a[p][q] */
        double theta = (a[q][q] - a[p][p]) / (2.0 * a[p][q]);
        double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        for (int r = 0; r < 3; ++r) { /* A <- A J */
          double arp = a[r][p], arq = a[r][q];
          a[r][p] = c * arp - s * arq;
          a[r][q] = s * arp + c * arq;
        }
        for (int r = 0; r < 3; ++r) { /* A <- J^T A */
          double apr = a[p][r], aqr = a[q][r];
          a[p][r] = c * apr - s * aqr;
          a[q][r] = s * apr + c * aqr;
        }
        for (int r = 0; r < 3; ++r) { /* V <- V J */
          double vrp = v[r][p], vrq = v[r][q];
          v[r][p] = c * vrp - s * vrq;
          v[r][q] = s * vrp + c * vrq;
        }
      }
  }
  int ord[3] = {0, 1, 2};
  for (int i = 0; i < 3; ++i)
    for (int j = i + 1; j < 3; ++j)
      if (a[ord[j]][ord[j]] < a[ord[i]][ord[i]]) {
        int tmp = ord[i];
        ord[i] = ord[j];
        ord[j] = tmp;
      }
  for (int j = 0; j < 3; ++j) {
    evals[j] = a[ord[j]][ord[j]];
    for (int r = 0; r < 3; ++r) evecs[3 * r + j] = v[r][ord[j]];
  }
  return 0;
}

/* ------------------------------------------------------------------------- */
/* PCA normals + curvature from kNN neighbourhoods                            */
/*   neighbourhood: the k nearest points of p (p itself included)             */
/*   mean mu = (1/n) sum p_j,  C = (1/n) sum (p_j - mu)(p_j - mu)^T           */
/*   normal = eigenvector of the smallest eigenvalue, flipped so that          */
/*            normal . (viewpoint - p) >= 0                                    */
/*   curvature (surface variation) = l0 / (l0 + l1 + l2)                       */
/*   fewer than 3 neighbours or a zero covariance -> NaN normal and curvature */
/* ------------------------------------------------------------------------- */
typedef struct {
  const float *xyz;
  const int32_t *nbr;
  int k;
  const double *vp;
  double *normals, *curv, *evals;
} nrm_ctx;

static void nrm_range(void *vctx, int64_t lo, int64_t hi, int tid) {
  (void)tid;
  nrm_ctx *c = (nrm_ctx *)vctx;
  for (int64_t i = lo; i < hi; ++i) {
    const int32_t *nb = c->nbr + i * c->k;
    int n = 0;
    double mu[3] = {0, 0, 0};
    for (int j = 0; j < c->k; ++j) {
      if (nb[j] < 0) continue;
      const float *p = c->xyz + 3 * (int64_t)nb[j];
      for (int a = 0; a < 3; ++a) mu[a] += (double)p[a];
      ++n;
    }
    double *nout = c->normals + 3 * i;
    double ev[3] = {NAN, NAN, NAN};
    if (n >= 3) {
      for (int a = 0; a < 3; ++a) mu[a] /= n;
      double C[6] = {0, 0, 0, 0, 0, 0};
      for (int j = 0; j < c->k; ++j) {
        if (nb[j] < 0) continue;
        const float *p = c->xyz + 3 * (int64_t)nb[j];
        double e0 = p[0] - mu[0], e1 = p[1] - mu[1], e2 = p[2] - mu[2];
        C[0] += e0 * e0;
        C[1] += e0 * e1;
        C[2] += e0 * e2;
        C[3] += e1 * e1;
        C[4] += e1 * e2;
        C[5] += e2 * e2;
      }
      for (int m = 0; m < 6; ++m) C[m] /= n;
      double vec[9];
      oracle_sym3_eigen(C, ev, vec);
      double tr = ev[0] + ev[1] + ev[2];
      if (tr > 0) {
        double nx = vec[0], ny = vec[3], nz = vec[6];
        const float *p = c->xyz + 3 * i;
        double s = nx * (c->vp[0] - p[0]) + ny * (c->vp[1] - p[1]) + nz * (c->vp[2] - p[2]);
        if (s < 0) {
          nx = -nx;
          ny = -ny;
          nz = -nz;
        }
        nout[0] = nx;
        nout[1] = ny;
        nout[2] = nz;
        c->curv[i] = ev[0] / tr;
      } else {
        nout[0] = nout[1] = nout[2] = NAN;
        c->curv[i] = NAN;
      }
    } else {
      nout[0] = nout[1] = nout[2] = NAN;
      c->curv[i] = NAN;
    }
    if (c->evals)
      for (int a = 0; a < 3; ++a) c->evals[3 * i + a] = ev[a];
  }
}

int oracle_normals(const float *xyz, int64_t n, int k, const double *viewpoint, double *normals,
                   double *curvature, double *evals, int use_kdtree, int n_threads) {
  if (k <= 0 || n < 0) return 1;
  int32_t *nbr = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n * k + 1));
  double *d2 = (double *)malloc(sizeof(double) * (size_t)(n * k + 1));
  if (!nbr || !d2) {
    free(nbr);
    free(d2);
    return 2;
  }
  int rc = use_kdtree ? oracle_knn_kdtree(xyz, n, xyz, n, k, nbr, d2, n_threads)
                      : oracle_knn(xyz, n, xyz, n, k, nbr, d2, n_threads);
  if (rc == 0) {
    nrm_ctx c = {xyz, nbr, k, viewpoint, normals, curvature, evals};
    parallel_for(n, n_threads, nrm_range, &c);
  }
  free(nbr);
  free(d2);
  return rc;
}

/* normals for a subset of points (the neighbourhood is still searched over    */
/* the whole cloud); used for sampled checks on large clouds                  */
int oracle_normals_subset(const float *xyz, int64_t n, const int64_t *sel, int64_t n_sel, int k,
                          const double *viewpoint, double *normals, double *curvature,
                          double *evals, int use_kdtree, int n_threads) {
  if (k <= 0 || n < 0 || n_sel < 0) return 1;
  float *q = (float *)malloc(sizeof(float) * 3 * (size_t)(n_sel + 1));
  int32_t *nbr = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n_sel * k + 1));
  double *d2 = (double *)malloc(sizeof(double) * (size_t)(n_sel * k + 1));
  if (!q || !nbr || !d2) {
    free(q);
    free(nbr);
    free(d2);
    return 2;
  }
  for (int64_t s = 0; s < n_sel; ++s)
    for (int a = 0; a < 3; ++a) q[3 * s + a] = xyz[3 * sel[s] + a];
  int rc = use_kdtree ? oracle_knn_kdtree(xyz, n, q, n_sel, k, nbr, d2, n_threads)
                      : oracle_knn(xyz, n, q, n_sel, k, nbr, d2, n_threads);
  if (rc == 0) {
    /* evaluate each selected point with its own neighbour list; the viewpoint
       test uses the selected point's own coordinates */
    for (int64_t s = 0; s < n_sel; ++s) {
      /* build a tiny local cloud = the neighbours, then reuse nrm_range on it
         with the query placed at index 0 for the orientation test */
      float *loc = (float *)malloc(sizeof(float) * 3 * (size_t)(k + 1));
      int32_t *lnb = (int32_t *)malloc(sizeof(int32_t) * (size_t)k);
      for (int a = 0; a < 3; ++a) loc[a] = q[3 * s + a];
      for (int j = 0; j < k; ++j) {
        int32_t g = nbr[s * k + j];
        if (g < 0) {
          lnb[j] = -1;
          continue;
        }
        for (int a = 0; a < 3; ++a) loc[3 * (j + 1) + a] = xyz[3 * (int64_t)g + a];
        lnb[j] = j + 1;
      }
      nrm_ctx lc = {loc, lnb, k, viewpoint, normals + 3 * s, curvature + s, evals ? evals + 3 * s : NULL};
      nrm_range(&lc, 0, 1, 0);
      free(loc);
      free(lnb);
    }
  }
  free(q);
  free(nbr);
  free(d2);
  return rc;
}

/* ------------------------------------------------------------------------- */
/* rigid point-to-plane ICP                                                   */
/* ------------------------------------------------------------------------- */
/* status bits reported by oracle_icp (same meaning as the library's report) */
#define ORACLE_ICP_DEGENERATE 5

typedef struct {
  const float *src, *dst, *dst_n;
  int64_t n_src, n_dst;
  const kd_tree *tree; /* NULL: exhaustive nearest-neighbour search */
  double R[9], t[3];
  double dmax2;
  /* per-thread accumulators: H (6x6 upper), g (6), sum r^2, count */
  double (*H)[36];
  double (*g)[6];
  double *r2;
  int64_t *cnt;
} icp_ctx;

/* Exhaustive nearest neighbour of a double-precision (transformed) point. */
static void nearest_d(const icp_ctx *c, const double *p, int32_t *best_i, double *best_d) {
  int32_t bi = -1;
  double bd = INFINITY;
  for (int64_t i = 0; i < c->n_dst; ++i) {
    const float *q = c->dst + 3 * i;
    double dx = p[0] - q[0], dy = p[1] - q[1], dz = p[2] - q[2];
    double d = dx * dx + dy * dy + dz * dz;
    if (pair_less(d, i, bd, bi)) {
      bd = d;
      bi = (int32_t)i;
    }
  }
  *best_i = bi;
  *best_d = bd;
}

/* kd-tree nearest neighbour for a double-precision query point */
static void kd_nn_d(const kd_tree *t, int32_t node, const double *q, double *bd, int32_t *bi) {
  const kd_node *nd = &t->nodes[node];
  if (nd->left < 0) {
    for (int32_t j = nd->lo; j < nd->hi; ++j) {
      const float *p = kd_pt(t, j);
      double dx = q[0] - p[0], dy = q[1] - p[1], dz = q[2] - p[2];
      double d = dx * dx + dy * dy + dz * dz;
      if (pair_less(d, t->perm[j], *bd, *bi)) {
        *bd = d;
        *bi = t->perm[j];
      }
    }
    return;
  }
  double diff = q[nd->axis] - nd->split;
  int32_t near = diff <= 0 ? nd->left : nd->right;
  int32_t far = diff <= 0 ? nd->right : nd->left;
  kd_nn_d(t, near, q, bd, bi);
  if (diff * diff <= *bd * (1.0 + 1e-12)) kd_nn_d(t, far, q, bd, bi);
}

static void icp_range(void *vctx, int64_t lo, int64_t hi, int tid) {
  icp_ctx *c = (icp_ctx *)vctx;
  double *H = c->H[tid], *g = c->g[tid];
  for (int64_t i = lo; i < hi; ++i) {
    const float *ps = c->src + 3 * i;
    /* p' = R p + t */
    double p[3];
    for (int a = 0; a < 3; ++a)
      p[a] = c->R[3 * a] * ps[0] + c->R[3 * a + 1] * ps[1] + c->R[3 * a + 2] * ps[2] + c->t[a];
    int32_t j;
    double d2;
    if (c->tree) {
      j = -1;
      d2 = INFINITY;
      if (c->tree->n_nodes > 0) kd_nn_d(c->tree, 0, p, &d2, &j);
    } else {
      nearest_d(c, p, &j, &d2);
    }
    /* reject: no neighbour, farther than the rejection distance, or no normal */
    if (j < 0 || !(d2 <= c->dmax2)) continue;
    const float *q = c->dst + 3 * (int64_t)j;
    const float *nq = c->dst_n + 3 * (int64_t)j;
    double n[3] = {nq[0], nq[1], nq[2]};
    if (!isfinite(n[0]) || !isfinite(n[1]) || !isfinite(n[2])) continue;
    /* residual r = n . (p' - q);  Jacobian J = [p' x n, n] */
    double r = n[0] * (p[0] - q[0]) + n[1] * (p[1] - q[1]) + n[2] * (p[2] - q[2]);
    double J[6] = {p[1] * n[2] - p[2] * n[1], p[2] * n[0] - p[0] * n[2], p[0] * n[1] - p[1] * n[0],
                   n[0], n[1], n[2]};
    for (int a = 0; a < 6; ++a) {
      for (int b = 0; b < 6; ++b) H[6 * a + b] += J[a] * J[b];
      g[a] += J[a] * r;
    }
    c->r2[tid] += r * r;
    c->cnt[tid] += 1;
  }
}

/* Solve H x = -g by Cholesky (H = L L^T).  Returns 0 on success, nonzero when
 * a pivot is <= 1e-12 * trace(H) (the system is treated as degenerate). */
static int cholesky_solve6(const double *H, const double *g, double *x) {
  double L[36];
  memset(L, 0, sizeof(L));
  double tr = 0;
  for (int a = 0; a < 6; ++a) tr += H[6 * a + a];
  if (!(tr > 0)) return 1;
  for (int j = 0; j < 6; ++j) {
    double s = H[6 * j + j];
    for (int m = 0; m < j; ++m) s -= L[6 * j + m] * L[6 * j + m];
    if (!(s > 1e-12 * tr)) return 1;
    double ljj = sqrt(s);
    L[6 * j + j] = ljj;
    for (int i = j + 1; i < 6; ++i) {
      double v = H[6 * i + j];
      for (int m = 0; m < j; ++m) v -= L[6 * i + m] * L[6 * j + m];
      L[6 * i + j] = v / ljj;
    }
  }
  double y[6];
  for (int i = 0; i < 6; ++i) { /* L y = -g */
    double v = -g[i];
    for (int m = 0; m < i; ++m) v -= L[6 * i + m] * y[m];
    y[i] = v / L[6 * i + i];
  }
  for (int i = 5; i >= 0; --i) { /* L^T x = y */
    double v = y[i];
    for (int m = i + 1; m < 6; ++m) v -= L[6 * m + i] * x[m];
    x[i] = v / L[6 * i + i];
  }
  return 0;
}

/* Rodrigues: exp of the skew matrix of w */
static void so3_exp(const double *w, double *R) {
  double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
  double th = sqrt(th2);
  double A, B; /* sin(th)/th, (1-cos(th))/th^2 */
  if (th < 1e-8) {
    A = 1.0 - th2 / 6.0;
    B = 0.5 - th2 / 24.0;
  } else {
    A = sin(th) / th;
    B = (1.0 - cos(th)) / th2;
  }
  double K[9] = {0, -w[2], w[1], w[2], 0, -w[0], -w[1], w[0], 0};
  double K2[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0;
      for (int m = 0; m < 3; ++m) s += K[3 * i + m] * K[3 * m + j];
      K2[3 * i + j] = s;
    }
  for (int i = 0; i < 9; ++i) R[i] = (i % 4 == 0 ? 1.0 : 0.0) + A * K[i] + B * K2[i];
}

/* One association pass at the transform (R, t): fills the per-thread sums. */
static void icp_accumulate(icp_ctx *c, int nt, double *H, double *g, double *r2, int64_t *cnt) {
  for (int tt = 0; tt < nt; ++tt) {
    memset(c->H[tt], 0, sizeof(double) * 36);
    memset(c->g[tt], 0, sizeof(double) * 6);
    c->r2[tt] = 0;
    c->cnt[tt] = 0;
  }
  parallel_for(c->n_src, nt, icp_range, c);
  memset(H, 0, sizeof(double) * 36);
  memset(g, 0, sizeof(double) * 6);
  *r2 = 0;
  *cnt = 0;
  for (int tt = 0; tt < nt; ++tt) { /* combine in thread order */
    for (int m = 0; m < 36; ++m) H[m] += c->H[tt][m];
    for (int m = 0; m < 6; ++m) g[m] += c->g[tt][m];
    *r2 += c->r2[tt];
    *cnt += c->cnt[tt];
  }
}

/*
 * T_init (NULL: identity), T_out: row-major 4x4, source -> target.
 * iters: number of correspondence/estimation rounds (fixed, no early stop).
 * After the last update one more association pass gives the final
 * point-to-plane RMSE over the inliers and their count.
 * status: 0, or ORACLE_ICP_DEGENERATE if any round had fewer than 6 inliers
 * or a failed Cholesky pivot (that round's update is skipped).
 * trace (optional): iters x 16 transforms after each round.
 * sums (optional): the 6x6 H and 6 g of every round, iters x 42.
 */
int oracle_icp(const float *src, int64_t n_src, const float *dst, const float *dst_normals,
               int64_t n_dst, const double *T_init, int iters, double max_corr_dist, double *T_out,
               double *rmse, int64_t *n_inliers, int *status, double *trace, double *sums,
               int use_kdtree, int n_threads) {
  if (iters < 0 || n_src < 0 || n_dst < 0 || n_dst > INT32_MAX) return 1;
  int nt = clamp_threads(n_threads);
  icp_ctx c;
  memset(&c, 0, sizeof(c));
  c.src = src;
  c.dst = dst;
  c.dst_n = dst_normals;
  c.n_src = n_src;
  c.n_dst = n_dst;
  c.dmax2 = max_corr_dist * max_corr_dist;
  kd_tree tree;
  memset(&tree, 0, sizeof(tree));
  if (use_kdtree) {
    if (kd_init(&tree, dst, n_dst)) {
      kd_free(&tree);
      return 2;
    }
    c.tree = &tree;
  }
  c.H = malloc(sizeof(double[36]) * nt);
  c.g = malloc(sizeof(double[6]) * nt);
  c.r2 = malloc(sizeof(double) * nt);
  c.cnt = malloc(sizeof(int64_t) * nt);
  double T[16];
  if (T_init) {
    memcpy(T, T_init, sizeof(T));
  } else {  /* identity */
    for (int j = 0; j < 16; ++j) T[j] = (j % 5) == 0 ? 1.0 : 0.0;
  }
  *status = 0;
  double H[36], g[6], r2;
  int64_t cnt;
  for (int it = 0; it < iters; ++it) {
    for (int a = 0; a < 3; ++a) {
      for (int b = 0; b < 3; ++b) c.R[3 * a + b] = T[4 * a + b];
      c.t[a] = T[4 * a + 3];
    }
    icp_accumulate(&c, nt, H, g, &r2, &cnt);
    if (sums) {
      memcpy(sums + 42 * it, H, sizeof(H));
      memcpy(sums + 42 * it + 36, g, sizeof(g));
    }
    double xi[6];
    if (cnt < 6 || cholesky_solve6(H, g, xi)) {
      *status = ORACLE_ICP_DEGENERATE;
    } else {
      /* T <- [exp(w^), tau; 0 1] * T  with xi = (w, tau) */
      double dR[9];
      so3_exp(xi, dR);
      double Tn[16];
      for (int a = 0; a < 3; ++a) {
        for (int b = 0; b < 4; ++b) {
          double s = 0;
          for (int m = 0; m < 3; ++m) s += dR[3 * a + m] * T[4 * m + b];
          Tn[4 * a + b] = s;
        }
        Tn[4 * a + 3] += xi[3 + a];
      }
      Tn[12] = Tn[13] = Tn[14] = 0;
      Tn[15] = 1;
      memcpy(T, Tn, sizeof(T));
    }
    if (trace) memcpy(trace + 16 * it, T, sizeof(T));
  }
  for (int a = 0; a < 3; ++a) {
    for (int b = 0; b < 3; ++b) c.R[3 * a + b] = T[4 * a + b];
    c.t[a] = T[4 * a + 3];
  }
  icp_accumulate(&c, nt, H, g, &r2, &cnt);
  *n_inliers = cnt;
  *rmse = cnt > 0 ? sqrt(r2 / (double)cnt) : NAN;
  memcpy(T_out, T, sizeof(T));
  free(c.H);
  free(c.g);
  free(c.r2);
  free(c.cnt);
  if (use_kdtree) kd_free(&tree);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* hybrid query: the k nearest points among those within distance r           */
/* (Sec. 3, KDTree "hybrid" queries): exhaustive search, (d2, idx) order,      */
/* missing entries padded with -1 / +inf                                        */
/* ------------------------------------------------------------------------- */
typedef struct {
  const float *ref, *qry;
  int64_t n_ref;
  int k;
  double r2;
  int32_t *out_idx;
  double *out_d2;
} hyb_ctx;

static void hyb_range(void *vctx, int64_t lo, int64_t hi, int tid) {
  (void)tid;
  hyb_ctx *c = (hyb_ctx *)vctx;
  for (int64_t q = lo; q < hi; ++q) {
    double *d = c->out_d2 + q * c->k;
    int32_t *ix = c->out_idx + q * c->k;
    int len = 0;
    for (int64_t i = 0; i < c->n_ref; ++i) {
      double dd = dist2(c->qry + 3 * q, c->ref + 3 * i);
      if (dd <= c->r2) topk_insert(d, ix, &len, c->k, dd, (int32_t)i);
    }
    pad_topk(d, ix, len, c->k);
  }
}

int oracle_knn_hybrid(const float *ref, int64_t n_ref, const float *qry, int64_t n_qry, int k,
                      double r, int32_t *out_idx, double *out_d2, int n_threads) {
  if (k <= 0 || r < 0 || n_ref < 0 || n_qry < 0) return 1;
  hyb_ctx c = {ref, qry, n_ref, k, r * r, out_idx, out_d2};
  parallel_for(n_qry, n_threads, hyb_range, &c);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* normals from radius neighbourhoods (Sec. 3; Sec. 4 uses a 1 cm radius):    */
/* every point within r (inclusive, the point itself included), then the same */
/* covariance / Jacobi / orientation / curvature as oracle_normals            */
/* ------------------------------------------------------------------------- */
typedef struct {
  const float *xyz;
  int64_t n;
  double r2;
  const double *vp;
  double *normals, *curv, *evals;
  int64_t *counts;
  const int64_t *sel; /* NULL: every point; else the points to evaluate */
} nrr_ctx;

static void nrr_range(void *vctx, int64_t lo, int64_t hi, int tid) {
  (void)tid;
  nrr_ctx *c = (nrr_ctx *)vctx;
  for (int64_t i = lo; i < hi; ++i) {
    const float *p = c->xyz + 3 * (c->sel ? c->sel[i] : i);
    double mu[3] = {0, 0, 0};
    int64_t m = 0;
    for (int64_t j = 0; j < c->n; ++j)
      if (dist2(p, c->xyz + 3 * j) <= c->r2) {
        for (int a = 0; a < 3; ++a) mu[a] += (double)c->xyz[3 * j + a];
        ++m;
      }
    if (c->counts) c->counts[i] = m;
    double *nout = c->normals + 3 * i;
    double ev[3] = {NAN, NAN, NAN};
    nout[0] = nout[1] = nout[2] = NAN;
    c->curv[i] = NAN;
    if (m >= 3) {
      for (int a = 0; a < 3; ++a) mu[a] /= (double)m;
      double C[6] = {0, 0, 0, 0, 0, 0};
      for (int64_t j = 0; j < c->n; ++j)
        if (dist2(p, c->xyz + 3 * j) <= c->r2) {
          const float *q = c->xyz + 3 * j;
          double e0 = q[0] - mu[0], e1 = q[1] - mu[1], e2 = q[2] - mu[2];
          C[0] += e0 * e0;
          C[1] += e0 * e1;
          C[2] += e0 * e2;
          C[3] += e1 * e1;
          C[4] += e1 * e2;
          C[5] += e2 * e2;
        }
      for (int t = 0; t < 6; ++t) C[t] /= (double)m;
      double vec[9];
      oracle_sym3_eigen(C, ev, vec);
      double tr = ev[0] + ev[1] + ev[2];
      if (tr > 0) {
        double nx = vec[0], ny = vec[3], nz = vec[6];
        double s = nx * (c->vp[0] - p[0]) + ny * (c->vp[1] - p[1]) + nz * (c->vp[2] - p[2]);
        if (s < 0) {
          nx = -nx;
          ny = -ny;
          nz = -nz;
        }
        nout[0] = nx;
        nout[1] = ny;
        nout[2] = nz;
        c->curv[i] = ev[0] / tr;
      }
    }
    if (c->evals)
      for (int a = 0; a < 3; ++a) c->evals[3 * i + a] = ev[a];
  }
}

/* sel (optional): evaluate only these points (outputs have n_sel rows); the
 * neighbourhoods are always searched in the whole cloud */
int oracle_normals_radius(const float *xyz, int64_t n, double r, const double *viewpoint,
                          double *normals, double *curvature, double *evals, int64_t *counts,
                          const int64_t *sel, int64_t n_sel, int n_threads) {
  if (r < 0 || n < 0 || (sel && n_sel < 0)) return 1;
  nrr_ctx c = {xyz, n, r * r, viewpoint, normals, curvature, evals, counts, sel};
  parallel_for(sel ? n_sel : n, n_threads, nrr_range, &c);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* voxel-grid downsampling (Sec. 3 GridAccumulator; Sec. 4 downsamples at     */
/* 1 cm before ICP): point i falls in voxel floor(x / v) per axis (float      */
/* division, as the float point type of the library computes it); every       */
/* occupied voxel yields the mean of its points.  Output in ascending         */
/* (ix, iy, iz) order.                                                         */
/* ------------------------------------------------------------------------- */
typedef struct {
  int64_t ix, iy, iz, idx;
} vox_rec;

static int cmp_vox(const void *a, const void *b) {
  const vox_rec *x = (const vox_rec *)a, *y = (const vox_rec *)b;
  if (x->ix != y->ix) return x->ix < y->ix ? -1 : 1;
  if (x->iy != y->iy) return x->iy < y->iy ? -1 : 1;
  if (x->iz != y->iz) return x->iz < y->iz ? -1 : 1;
  return x->idx < y->idx ? -1 : (x->idx > y->idx);
}

int oracle_voxel_downsample(const float *xyz, int64_t n, float voxel, double *out_xyz,
                            int64_t *out_counts, int64_t *out_n) {
  if (n < 0 || !(voxel > 0)) return 1;
  vox_rec *r = (vox_rec *)malloc(sizeof(vox_rec) * (size_t)(n > 0 ? n : 1));
  if (!r) return 2;
  for (int64_t i = 0; i < n; ++i) {
    r[i].ix = (int64_t)floorf(xyz[3 * i] / voxel);
    r[i].iy = (int64_t)floorf(xyz[3 * i + 1] / voxel);
    r[i].iz = (int64_t)floorf(xyz[3 * i + 2] / voxel);
    r[i].idx = i;
  }
  qsort(r, (size_t)n, sizeof(vox_rec), cmp_vox);
  int64_t m = 0;
  for (int64_t i = 0; i < n;) {
    int64_t j = i;
    double s[3] = {0, 0, 0};
    while (j < n && r[j].ix == r[i].ix && r[j].iy == r[i].iy && r[j].iz == r[i].iz) {
      for (int a = 0; a < 3; ++a) s[a] += (double)xyz[3 * r[j].idx + a];
      ++j;
    }
    for (int a = 0; a < 3; ++a) out_xyz[3 * m + a] = s[a] / (double)(j - i);
    out_counts[m] = j - i;
    ++m;
    i = j;
  }
  *out_n = m;
  free(r);
  return 0;
}
