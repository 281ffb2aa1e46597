/*
 * A plain C99 caller of the library (include/cg.h), host buffers only: the
 * boundary used from C without Python or PyTorch.  It builds the 7-point
 * Laplacian on a 12^3 grid (diagonal 6, neighbours -1, boundary nodes
 * eliminated), a right-hand side b = A x* with x* of dyadic values (so b is
 * exact), and checks:
 *   - cg_create / cg_info / cg_partition_info / cg_solve / cg_destroy:
 *     the solve converges and x is within 1e-8 of x*;
 *   - an invalid call returns CG_EINVAL with a message;
 *   - the batch API: three requests (b, 2b, 0) solved in one object, each
 *     result as the single solve's (x*, 2x*, 0).
 * Prints "c caller ok" and exits 0 on success, prints the failure and exits
 * 1 otherwise.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include "cg.h"

#define N 12

static int fail(const char* what, int status, const char* msg) {
  printf("FAIL %s: status %d (%s)\n", what, status, msg ? msg : "");
  return 1;
}

static double max_err(const double* x, const double* ref, double scale, int64_t n) {
  double e = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    const double d = fabs(x[i] - scale * ref[i]);
    if (d > e) e = d;
  }
  return e;
}

int main(void) {
  const int64_t n = (int64_t)N * N * N;
  int32_t* rp = malloc(sizeof(int32_t) * (size_t)(n + 1));
  int32_t* ci = malloc(sizeof(int32_t) * (size_t)(7 * n));
  double* va = malloc(sizeof(double) * (size_t)(7 * n));
  double* xs = malloc(sizeof(double) * (size_t)n);
  double* b = malloc(sizeof(double) * (size_t)n);
  double* b2 = malloc(sizeof(double) * (size_t)n);
  double* b0 = malloc(sizeof(double) * (size_t)n);
  double* x = malloc(sizeof(double) * (size_t)n);
  double* xb[3];
  for (int k = 0; k < 3; ++k) xb[k] = malloc(sizeof(double) * (size_t)n);
  if (!rp || !ci || !va || !xs || !b || !b2 || !b0 || !x || !xb[0] || !xb[1] || !xb[2]) return fail("malloc", -1, 0);

  /* the operator, rows in lexicographic order, columns ascending */
  int64_t nnz = 0;
  rp[0] = 0;
  for (int k = 0; k < N; ++k)
    for (int j = 0; j < N; ++j)
      for (int i = 0; i < N; ++i) {
        const int64_t row = ((int64_t)k * N + j) * N + i;
        if (k > 0) { ci[nnz] = (int32_t)(row - N * N); va[nnz++] = -1.0; }
        if (j > 0) { ci[nnz] = (int32_t)(row - N); va[nnz++] = -1.0; }
        if (i > 0) { ci[nnz] = (int32_t)(row - 1); va[nnz++] = -1.0; }
        ci[nnz] = (int32_t)row; va[nnz++] = 6.0;
        if (i < N - 1) { ci[nnz] = (int32_t)(row + 1); va[nnz++] = -1.0; }
        if (j < N - 1) { ci[nnz] = (int32_t)(row + N); va[nnz++] = -1.0; }
        if (k < N - 1) { ci[nnz] = (int32_t)(row + N * N); va[nnz++] = -1.0; }
        rp[row + 1] = (int32_t)nnz;
      }
  for (int64_t r = 0; r < n; ++r) xs[r] = 1.0 + 0.125 * (double)(r % 7);
  for (int64_t r = 0; r < n; ++r) {
    double s = 0.0;
    for (int32_t e = rp[r]; e < rp[r + 1]; ++e) s += va[e] * xs[ci[e]];
    b[r] = s;
    b2[r] = 2.0 * s;
    b0[r] = 0.0;
  }

  /* one system through a handle */
  cg_csr csr = {rp, ci, va, 0, 0};
  cg_opts o;
  cg_opts_default(&o);
  cg_handle h = NULL;
  int st = cg_create(&h, &csr, n, nnz, &o);
  if (st != CG_OK) return fail("cg_create", st, cg_last_error(NULL));
  int64_t n_out = 0, nnz_out = 0;
  int32_t nblocks = 0, max_rows = 0, kernel = -1;
  st = cg_info(h, &n_out, &nnz_out, &nblocks);
  if (st != CG_OK || n_out != n || nnz_out != nnz || nblocks < 1) return fail("cg_info", st, cg_last_error(h));
  st = cg_partition_info(h, &max_rows, &kernel);
  if (st != CG_OK) return fail("cg_partition_info", st, cg_last_error(h));
  for (int64_t r = 0; r < n; ++r) x[r] = 0.0;
  int64_t iters = 0;
  double relres = 1.0;
  st = cg_solve(h, b, x, 1e-10, 10 * n, &iters, &relres);
  if (st != CG_OK || !(relres <= 1e-10) || iters <= 0) return fail("cg_solve", st, cg_last_error(h));
  if (!(max_err(x, xs, 1.0, n) <= 1e-8 * 1.875)) return fail("cg_solve accuracy", st, "x differs from x*");
  st = cg_solve(h, b, x, -1.0, 10, &iters, &relres);
  if (st != CG_EINVAL || cg_last_error(h)[0] == '\0') return fail("cg_solve with tol < 0", st, cg_last_error(h));
  st = cg_destroy(h);
  if (st != CG_OK) return fail("cg_destroy", st, 0);

  /* three systems through the batch API */
  cg_batch_opts bo;
  cg_batch_opts_default(&bo);
  bo.budget_bytes = (int64_t)256 << 20;
  cg_batch bt = NULL;
  st = cg_batch_create(&bt, &bo);
  if (st != CG_OK) return fail("cg_batch_create", st, cg_batch_last_error(NULL));
  const double* rhs[3] = {b, b2, b0};
  cg_request req[3];
  for (int k = 0; k < 3; ++k) {
    req[k].csr = csr;
    req[k].n = n;
    req[k].nnz = nnz;
    req[k].b = rhs[k];
    req[k].x = xb[k];
    req[k].tol = 1e-10;
    req[k].maxit = 10 * n;
    req[k].tag = (uint64_t)(100 + k);
  }
  uint64_t tickets[3];
  st = cg_batch_submit(bt, req, 3, tickets);
  if (st != CG_OK) return fail("cg_batch_submit", st, cg_batch_last_error(bt));
  const double scale[3] = {1.0, 2.0, 0.0};
  for (int k = 0; k < 3; ++k) {
    cg_result res;
    st = cg_batch_wait(bt, tickets[k], -1, &res);
    if (st != CG_OK || !res.done || res.status != CG_OK || res.tag != (uint64_t)(100 + k))
      return fail("cg_batch_wait", st != CG_OK ? st : res.status, cg_batch_last_error(bt));
    if (!(res.relres <= 1e-10)) return fail("batch relres", res.status, "above 1e-10");
    if (!(max_err(xb[k], xs, scale[k], n) <= 1e-8 * 1.875 * (scale[k] > 0.0 ? scale[k] : 1.0)))
      return fail("batch accuracy", res.status, "x differs from the scaled x*");
  }
  cg_batch_stats bs;
  st = cg_batch_get_stats(bt, &bs);
  if (st != CG_OK || bs.completed != 3) return fail("cg_batch_get_stats", st, cg_batch_last_error(bt));
  st = cg_batch_destroy(bt);
  if (st != CG_OK) return fail("cg_batch_destroy", st, 0);

  printf("c caller ok: n=%lld nnz=%lld iters=%lld relres=%.3e kernel=%d ctas=%d\n", (long long)n,
         (long long)nnz, (long long)iters, relres, (int)kernel, (int)nblocks);
  free(rp); free(ci); free(va); free(xs); free(b); free(b2); free(b0); free(x);
  for (int k = 0; k < 3; ++k) free(xb[k]);
  return 0;
}
