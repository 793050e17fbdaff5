"""The C oracle built with AddressSanitizer and UndefinedBehaviorSanitizer
(host only) and driven through each entry point on small clouds, including
the edge cases (k above the point count, empty inputs, a query far outside,
duplicates): no out-of-bounds access, leak or undefined behaviour may be
reported."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

DRIVER = r"""
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
int oracle_knn(const float*, int64_t, const float*, int64_t, int, int32_t*, double*, int);
int oracle_knn_kdtree(const float*, int64_t, const float*, int64_t, int, int32_t*, double*, int);
int oracle_radius(const float*, int64_t, const float*, int64_t, double, int64_t*, int32_t*, double*, int);
int oracle_normals(const float*, int64_t, int, const double*, double*, double*, double*, int, int);
int oracle_icp(const float*, int64_t, const float*, const float*, int64_t, const double*, int, double,
               double*, double*, int64_t*, int*, double*, double*, int, int);
int oracle_knn_hybrid(const float*, int64_t, const float*, int64_t, int, double, int32_t*, double*, int);
int oracle_normals_radius(const float*, int64_t, double, const double*, double*, double*, double*,
                          int64_t*, const int64_t*, int64_t, int);
int oracle_voxel_downsample(const float*, int64_t, float, double*, int64_t*, int64_t*);

int main(void) {
  enum { N = 300 };
  float* P = malloc(sizeof(float) * 3 * N);
  unsigned s = 12345u;
  for (int i = 0; i < 3 * N; ++i) { s = s * 1664525u + 1013904223u; P[i] = (float)(s >> 8) / 16777216.0f; }
  for (int i = 0; i < 3; ++i) P[3 * 10 + i] = P[3 * 11 + i];  /* a duplicate */
  float far[3] = {50.0f, -40.0f, 30.0f};
  int32_t idx[N * 12]; double d2[N * 12];
  int rc = 0;
  for (int k = 1; k <= 12; k += 11) {
    rc |= oracle_knn(P, N, P, N, k, idx, d2, 2);
    rc |= oracle_knn_kdtree(P, N, P, N, k, idx, d2, 2);
    rc |= oracle_knn_kdtree(P, N, far, 1, k, idx, d2, 1);
  }
  rc |= oracle_knn(P, 5, P, 3, 8, idx, d2, 1);           /* k above the point count */
  rc |= oracle_knn_kdtree(P, 5, P, 3, 8, idx, d2, 1);
  rc |= oracle_knn(P, 0, P, 3, 4, idx, d2, 1);           /* empty reference */
  int64_t off[N + 1];
  rc |= oracle_radius(P, N, P, N, 0.2, off, NULL, NULL, 2);
  int64_t nnz = off[N];
  int32_t* ri = malloc(sizeof(int32_t) * (nnz + 1)); double* rd = malloc(sizeof(double) * (nnz + 1));
  rc |= oracle_radius(P, N, P, N, 0.2, off, ri, rd, 2);
  rc |= oracle_knn_hybrid(P, N, P, N, 12, 0.1, idx, d2, 2);
  double vp[3] = {0, 0, 10}, nrm[3 * N], cur[N], ev[3 * N];
  rc |= oracle_normals(P, N, 10, vp, nrm, cur, ev, 0, 2);
  rc |= oracle_normals(P, N, 10, vp, nrm, cur, ev, 1, 2);
  rc |= oracle_normals(P, 2, 10, vp, nrm, cur, ev, 0, 1);   /* fewer points than k */
  int64_t cnt[N];
  rc |= oracle_normals_radius(P, N, 0.15, vp, nrm, cur, ev, cnt, NULL, 0, 2);
  double vx[3 * N]; int64_t vc[N], vm = 0;
  rc |= oracle_voxel_downsample(P, N, 0.25f, vx, vc, &vm);
  float* nf = malloc(sizeof(float) * 3 * N);
  for (int i = 0; i < 3 * N; ++i) nf[i] = (float)nrm[i];
  double T[16], rmse, trace[16 * 6], sums[64]; int64_t ninl; int st;
  rc |= oracle_icp(P, N, P, nf, N, NULL, 5, 0.1, T, &rmse, &ninl, &st, NULL, NULL, 0, 2);
  rc |= oracle_icp(P, N, P, nf, N, NULL, 5, 0.1, T, &rmse, &ninl, &st, NULL, NULL, 1, 2);
  rc |= oracle_icp(far, 1, P, nf, N, NULL, 2, 0.1, T, &rmse, &ninl, &st, NULL, NULL, 0, 1);
  (void)trace; (void)sums;
  free(P); free(ri); free(rd); free(nf);
  printf("rc=%d\n", rc);
  return rc != 0;
}
"""


@pytest.mark.timeout(300)
def test_oracle_under_address_and_undefined_behaviour_sanitizers(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no host C compiler")
    drv = tmp_path / "driver.c"
    drv.write_text(DRIVER)
    exe = tmp_path / "oracle_asan"
    cmd = [gcc, "-O1", "-g", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off",
           "-fsanitize=address,undefined", "-fno-sanitize-recover=undefined", "-pthread",
           os.path.join(ROOT, "oracle", "cil_oracle.c"), str(drv), "-o", str(exe), "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0 and "sanitize" in (r.stderr or ""):
        pytest.skip("sanitizer runtime not available: " + r.stderr.strip().splitlines()[-1])
    assert r.returncode == 0, r.stderr
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1", UBSAN_OPTIONS="print_stacktrace=1")
    run = subprocess.run([str(exe)], capture_output=True, text=True, env=env, timeout=240)
    assert run.returncode == 0, run.stdout + run.stderr
    assert "rc=0" in run.stdout
