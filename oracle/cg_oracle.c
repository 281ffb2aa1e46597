/*
 * ORACLE — test infrastructure only.
 *
 * A plain, slow, sequential FP64 CPU statement of what the CG hot path
 * computes.  Only the test suite, the smoke check and the CPU-baseline leg of
 * the benchmark may call it; the product never does.  It shares no code,
 * header or table with the CUDA library: it is compiled on its own
 * (gcc -O2 -ffp-contract=off, so every a*b+c below is two roundings, exactly
 * as written) and called through ctypes.
 *
 * Every loop runs in index order; there is no blocking, fusion or reordering.
 *
 *   oracle_spmv   CSR product, Sec. 2.3 (the IA/JA/AA definition) and Sec. 5.2
 *   oracle_spmv_rows  the same product for a list of rows only (single outputs
 *                 of products too large to redo whole)
 *   oracle_dot    dot product, Sec. 5.2 ("Dot product" table)
 *   oracle_axpy   addition of vectors y <- a x + y, Sec. 5.2 (table labelled daxpy)
 *   oracle_ewmul  element-wise product, Sec. 5.2
 *   oracle_cg     classical (unpreconditioned) conjugate gradient, Sec. 5.3;
 *                 the paper prints no listing and cites Saad, "Iterative
 *                 Methods for Sparse Linear Systems" — the Hestenes-Stiefel form
 *                 is followed step by step.
 *   oracle_pcg_jacobi  preconditioned CG with M = diag(A) (z = dinv .* r by
 *                 the element-wise product), and oracle_jacobi_dinv.
 *   oracle_spmv_f32 / oracle_cg_mixed   the mixed-precision variant (FP32
 *                 matrix values and FP32-accumulated product; FP64 dots,
 *                 scalars, x and a true-residual replacement every k steps),
 *                 the mixed-precision refinement the paper cites in Sec. 5.3.
 *
 * Pins (what ties this file to the mathematics rather than to itself) are
 * the tests under tests/test_oracle_pins.py: the paper's 5x5 CSR example,
 * dense brute force, closed-form eigenpairs of the 7-point and Q1 operators,
 * finite termination, monotone A-norm error, the Chebyshev residual bound,
 * Lanczos extreme eigenvalues and manufactured solutions; for the mixed
 * iteration also the exact first step on integer data, the replacement
 * schedule (recursive = true residual to the bit after every replacement) and
 * FP32-rounding closeness to FP64 CG's early iterates.
 */
#include <stdint.h>
#include <math.h>
#include <string.h>
#include <stdlib.h>

/* y_i = sum_{k = IA(i)}^{IA(i+1)-1} AA(k) * x(JA(k)); base is 0 or 1 (Sec. 2.3:
 * "the i-th row starts at IA(i) and finishes at IA(i+1)-1"). */
void oracle_spmv(int64_t n, const int32_t* IA, const int32_t* JA, const double* AA,
                 int base, const double* x, double* y) {
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t k = (int64_t)IA[i] - base; k < (int64_t)IA[i + 1] - base; ++k)
            s = s + AA[k] * x[JA[k] - base];
        y[i] = s;
    }
}

/* The same product restricted to the listed rows: y_sel[t] = (A x)[rows[t]].
 * Used to check single outputs of products too large to redo whole. */
void oracle_spmv_rows(int64_t nrows, const int64_t* rows, const int32_t* IA, const int32_t* JA,
                      const double* AA, int base, const double* x, double* y_sel) {
    for (int64_t t = 0; t < nrows; ++t) {
        int64_t i = rows[t];
        double s = 0.0;
        for (int64_t k = (int64_t)IA[i] - base; k < (int64_t)IA[i + 1] - base; ++k)
            s = s + AA[k] * x[JA[k] - base];
        y_sel[t] = s;
    }
}

double oracle_dot(int64_t n, const double* x, const double* y) {
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s = s + x[i] * y[i];
    return s;
}

void oracle_axpy(int64_t n, double a, const double* x, double* y) {
    for (int64_t i = 0; i < n; ++i) y[i] = a * x[i] + y[i];
}

void oracle_ewmul(int64_t n, const double* x, const double* y, double* z) {
    for (int64_t i = 0; i < n; ++i) z[i] = x[i] * y[i];
}

/* Status codes (numerically the same meaning as the library's, kept separate). */
#define ORC_OK 0
#define ORC_NOTCONV 4
#define ORC_BREAKDOWN 5
#define ORC_NOMEM 2

/*
 * Classical CG (Hestenes-Stiefel) for SPD A, x in/out (initial guess in).
 *   r = b - A x;  p = r;  rho = r.r;  stop at once if sqrt(rho) <= tol*||b||
 *   for k = 1..maxit:
 *     q = A p;  gamma = p.q   (gamma <= 0 or not finite -> breakdown)
 *     alpha = rho / gamma;  x = x + alpha p;  r = r - alpha q
 *     rho_new = r.r;  if sqrt(rho_new) <= tol*||b||: stop with k iterations
 *     beta = rho_new / rho;  p = r + beta p;  rho = rho_new
 * The stopping rule compares the recursively updated residual with tol*||b||
 * (the paper does not state its rule).  If force_iters >= 0 the test is
 * ignored and exactly force_iters iterations run (for comparing iterates).
 * b = 0 gives x = 0, 0 iterations, residual 0.
 * Optional histories (NULL to skip) have room for hist_len entries:
 *   alpha_h[k-1], beta_h[k-1] (beta of step k), res_h[k] = ||r_k|| (res_h[0] = ||r_0||).
 * On return: iters, relres_rec = ||r_k||/||b||, relres_true = ||b - A x||/||b||.
 */
int oracle_cg(int64_t n, const int32_t* IA, const int32_t* JA, const double* AA, int base,
              const double* b, double* x, double tol, int64_t maxit, int64_t force_iters,
              int64_t* iters, double* relres_rec, double* relres_true,
              double* alpha_h, double* beta_h, double* res_h, int64_t hist_len) {
    double* r = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double* p = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double* q = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!r || !p || !q) { free(r); free(p); free(q); return ORC_NOMEM; }
    int status = ORC_OK;
    double bnorm = sqrt(oracle_dot(n, b, b));
    *iters = 0;
    if (bnorm == 0.0) {
        for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
        *relres_rec = 0.0; *relres_true = 0.0;
        free(r); free(p); free(q);
        return ORC_OK;
    }
    oracle_spmv(n, IA, JA, AA, base, x, q);
    for (int64_t i = 0; i < n; ++i) { r[i] = b[i] - q[i]; p[i] = r[i]; }
    double rho = oracle_dot(n, r, r);
    if (res_h && hist_len > 0) res_h[0] = sqrt(rho);
    int64_t k = 0;
    int done = (force_iters < 0) && (sqrt(rho) <= tol * bnorm);
    int64_t limit = force_iters >= 0 ? force_iters : maxit;
    while (!done && k < limit) {
        oracle_spmv(n, IA, JA, AA, base, p, q);
        double gamma = oracle_dot(n, p, q);
        if (!(gamma > 0.0) || !isfinite(gamma)) { status = ORC_BREAKDOWN; break; }
        double alpha = rho / gamma;
        for (int64_t i = 0; i < n; ++i) x[i] = x[i] + alpha * p[i];
        for (int64_t i = 0; i < n; ++i) r[i] = r[i] - alpha * q[i];
        double rho_new = oracle_dot(n, r, r);
        k = k + 1;
        if (alpha_h && k - 1 < hist_len) alpha_h[k - 1] = alpha;
        if (res_h && k < hist_len) res_h[k] = sqrt(rho_new);
        if (force_iters < 0 && sqrt(rho_new) <= tol * bnorm) { rho = rho_new; done = 1; break; }
        double beta = rho_new / rho;
        if (beta_h && k - 1 < hist_len) beta_h[k - 1] = beta;
        for (int64_t i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
        rho = rho_new;
    }
    *iters = k;
    *relres_rec = sqrt(rho) / bnorm;
    if (status == ORC_OK && force_iters < 0 && !done) status = ORC_NOTCONV;
    oracle_spmv(n, IA, JA, AA, base, x, q);
    double t = 0.0;
    for (int64_t i = 0; i < n; ++i) { double d = b[i] - q[i]; t = t + d * d; }
    *relres_true = sqrt(t) / bnorm;
    free(r); free(p); free(q);
    return status;
}

/* ------------------------------------------------------------------ mixed */

/* FP32 product: y_i = sum AA32(k) * x32(JA(k)) accumulated in FP32, in row order. */
void oracle_spmv_f32(int64_t n, const int32_t* IA, const int32_t* JA, const float* AA32,
                     int base, const float* x32, float* y32) {
    for (int64_t i = 0; i < n; ++i) {
        float s = 0.0f;
        for (int64_t k = (int64_t)IA[i] - base; k < (int64_t)IA[i + 1] - base; ++k)
            s = s + AA32[k] * x32[JA[k] - base];
        y32[i] = s;
    }
}

/*
 * Mixed-precision CG with residual replacement.
 *   The matrix is held twice: AA (FP64) and AA32 = (float)AA.
 *   Every step:  p32 = (float)p;  q = (double)(A32 p32)  [FP32 product, FP32 sums]
 *                gamma = p.q, alpha, x, r, rho_new, beta, p all in FP64 as in oracle_cg.
 *   Every `replace_every` steps (and before declaring convergence), r is
 *   replaced by the true FP64 residual b - A x (product with AA) and rho is
 *   recomputed from it; the direction update keeps the recurrence's own
 *   ratio, beta = rho_rec / rho with rho_rec the recursive r.r of this step,
 *   so p = r_true + beta p.  (With beta = rho_true / rho instead, a system
 *   whose recursive residual reaches tol long before the true one does gets
 *   beta >> 1 at that replacement and the iteration stalls along the old
 *   direction: the small Q1 systems never converge that way.)
 *   Convergence needs the true residual: sqrt(rho_true) <= tol*||b||.
 * If force_iters >= 0, exactly force_iters steps run: the replacements are
 * made as above (periodic, and whenever the recursive residual reaches
 * tol*||b||), but reaching the tolerance does not end the iteration, so the
 * iterate can be compared with a solver that stopped after that many steps.
 * Returns iterations and both residual measures as oracle_cg does.
 */
int oracle_cg_mixed(int64_t n, const int32_t* IA, const int32_t* JA, const double* AA,
                    const float* AA32, int base, const double* b, double* x, double tol,
                    int64_t maxit, int64_t replace_every, int64_t force_iters, int64_t* iters,
                    double* relres_rec, double* relres_true) {
    size_t m = (size_t)(n > 0 ? n : 1);
    double* r = (double*)malloc(sizeof(double) * m);
    double* p = (double*)malloc(sizeof(double) * m);
    double* q = (double*)malloc(sizeof(double) * m);
    float* p32 = (float*)malloc(sizeof(float) * m);
    float* q32 = (float*)malloc(sizeof(float) * m);
    if (!r || !p || !q || !p32 || !q32) { free(r); free(p); free(q); free(p32); free(q32); return ORC_NOMEM; }
    int status = ORC_OK;
    double bnorm = sqrt(oracle_dot(n, b, b));
    *iters = 0;
    if (bnorm == 0.0) {
        for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
        *relres_rec = 0.0; *relres_true = 0.0;
        free(r); free(p); free(q); free(p32); free(q32);
        return ORC_OK;
    }
    oracle_spmv(n, IA, JA, AA, base, x, q);
    for (int64_t i = 0; i < n; ++i) { r[i] = b[i] - q[i]; p[i] = r[i]; }
    double rho = oracle_dot(n, r, r);
    int64_t k = 0;
    int done = (force_iters < 0) && (sqrt(rho) <= tol * bnorm);
    int64_t limit = force_iters >= 0 ? force_iters : maxit;
    while (!done && k < limit) {
        for (int64_t i = 0; i < n; ++i) p32[i] = (float)p[i];
        oracle_spmv_f32(n, IA, JA, AA32, base, p32, q32);
        for (int64_t i = 0; i < n; ++i) q[i] = (double)q32[i];
        double gamma = oracle_dot(n, p, q);
        if (!(gamma > 0.0) || !isfinite(gamma)) { status = ORC_BREAKDOWN; break; }
        double alpha = rho / gamma;
        for (int64_t i = 0; i < n; ++i) x[i] = x[i] + alpha * p[i];
        for (int64_t i = 0; i < n; ++i) r[i] = r[i] - alpha * q[i];
        double rho_new = oracle_dot(n, r, r);
        double beta = rho_new / rho;
        k = k + 1;
        int replace = (replace_every > 0 && k % replace_every == 0) || sqrt(rho_new) <= tol * bnorm;
        if (replace) {
            oracle_spmv(n, IA, JA, AA, base, x, q);
            for (int64_t i = 0; i < n; ++i) r[i] = b[i] - q[i];
            rho_new = oracle_dot(n, r, r);
            if (force_iters < 0 && sqrt(rho_new) <= tol * bnorm) { rho = rho_new; done = 1; break; }
        }
        for (int64_t i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
        rho = rho_new;
    }
    *iters = k;
    *relres_rec = sqrt(rho) / bnorm;
    if (status == ORC_OK && force_iters < 0 && !done) status = ORC_NOTCONV;
    oracle_spmv(n, IA, JA, AA, base, x, q);
    double t = 0.0;
    for (int64_t i = 0; i < n; ++i) { double d = b[i] - q[i]; t = t + d * d; }
    *relres_true = sqrt(t) / bnorm;
    free(r); free(p); free(q); free(p32); free(q32);
    return status;
}

/* ---------------------------------------------------------------- Jacobi */

/* Inverse of the diagonal of A: dinv[i] = 1 / (sum of the stored entries of
 * row i in column i).  Returns 0, or ORC_BREAKDOWN if some diagonal is not
 * positive (then A is not SPD and no Jacobi preconditioner exists). */
int oracle_jacobi_dinv(int64_t n, const int32_t* IA, const int32_t* JA, const double* AA, int base,
                       double* dinv) {
    for (int64_t i = 0; i < n; ++i) {
        double d = 0.0;
        for (int64_t k = (int64_t)IA[i] - base; k < (int64_t)IA[i + 1] - base; ++k)
            if ((int64_t)JA[k] - base == i) d = d + AA[k];
        if (!(d > 0.0)) return ORC_BREAKDOWN;
        dinv[i] = 1.0 / d;
    }
    return ORC_OK;
}

/*
 * Jacobi-preconditioned CG: the preconditioned conjugate gradient iteration
 * with M = diag(A), the preconditioner applied as the element-wise product
 * z = dinv .* r (the paper's Sec. 5.2 element-wise product; it defers
 * preconditioning itself to domain decomposition):
 *   r = b - A x;  z = dinv .* r;  p = z;  rho = r.z
 *   for k = 1..maxit:
 *     q = A p;  gamma = p.q   (gamma <= 0 or not finite -> breakdown)
 *     alpha = rho / gamma;  x = x + alpha p;  r = r - alpha q
 *     if ||r|| <= tol*||b||: stop with k iterations   (the unpreconditioned test)
 *     z = dinv .* r;  rho_new = r.z;  beta = rho_new / rho;  p = z + beta p;  rho = rho_new
 * force_iters >= 0 runs exactly that many steps.  A diagonal that is not
 * positive gives ORC_BREAKDOWN with x untouched.
 */
int oracle_pcg_jacobi(int64_t n, const int32_t* IA, const int32_t* JA, const double* AA, int base,
                      const double* b, double* x, double tol, int64_t maxit, int64_t force_iters,
                      int64_t* iters, double* relres_rec, double* relres_true) {
    size_t m = (size_t)(n > 0 ? n : 1);
    double* r = (double*)malloc(sizeof(double) * m);
    double* z = (double*)malloc(sizeof(double) * m);
    double* p = (double*)malloc(sizeof(double) * m);
    double* q = (double*)malloc(sizeof(double) * m);
    double* dinv = (double*)malloc(sizeof(double) * m);
    if (!r || !z || !p || !q || !dinv) { free(r); free(z); free(p); free(q); free(dinv); return ORC_NOMEM; }
    *iters = 0;
    *relres_rec = 0.0;
    *relres_true = 0.0;
    if (oracle_jacobi_dinv(n, IA, JA, AA, base, dinv) != ORC_OK) {
        free(r); free(z); free(p); free(q); free(dinv);
        return ORC_BREAKDOWN;
    }
    int status = ORC_OK;
    double bnorm = sqrt(oracle_dot(n, b, b));
    if (bnorm == 0.0) {
        for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
        free(r); free(z); free(p); free(q); free(dinv);
        return ORC_OK;
    }
    oracle_spmv(n, IA, JA, AA, base, x, q);
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - q[i];
    oracle_ewmul(n, dinv, r, z);
    for (int64_t i = 0; i < n; ++i) p[i] = z[i];
    double rho = oracle_dot(n, r, z);
    double rr = oracle_dot(n, r, r);
    int64_t k = 0;
    int done = (force_iters < 0) && (sqrt(rr) <= tol * bnorm);
    int64_t limit = force_iters >= 0 ? force_iters : maxit;
    while (!done && k < limit) {
        oracle_spmv(n, IA, JA, AA, base, p, q);
        double gamma = oracle_dot(n, p, q);
        if (!(gamma > 0.0) || !isfinite(gamma)) { status = ORC_BREAKDOWN; break; }
        double alpha = rho / gamma;
        for (int64_t i = 0; i < n; ++i) x[i] = x[i] + alpha * p[i];
        for (int64_t i = 0; i < n; ++i) r[i] = r[i] - alpha * q[i];
        rr = oracle_dot(n, r, r);
        k = k + 1;
        if (force_iters < 0 && sqrt(rr) <= tol * bnorm) { done = 1; break; }
        oracle_ewmul(n, dinv, r, z);
        double rho_new = oracle_dot(n, r, z);
        double beta = rho_new / rho;
        for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
        rho = rho_new;
    }
    *iters = k;
    *relres_rec = sqrt(rr) / bnorm;
    if (status == ORC_OK && force_iters < 0 && !done) status = ORC_NOTCONV;
    oracle_spmv(n, IA, JA, AA, base, x, q);
    double t = 0.0;
    for (int64_t i = 0; i < n; ++i) { double d = b[i] - q[i]; t = t + d * d; }
    *relres_true = sqrt(t) / bnorm;
    free(r); free(z); free(p); free(q); free(dinv);
    return status;
}

/* Matrix statistics of the paper's Table 1 (Sec. 5.1): h (rows), nz, density
 * nz/h^2, bandwidth max|i-j| over stored entries, max_row, mean row length nz/h
 * and its standard deviation (population form).  out[7] in that order. */
void oracle_matrix_stats(int64_t n, const int32_t* IA, const int32_t* JA, int base, double* out) {
    int64_t nz = (int64_t)IA[n] - IA[0];
    int64_t bw = 0, maxrow = 0;
    double mean = n > 0 ? (double)nz / (double)n : 0.0, var = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t len = (int64_t)IA[i + 1] - IA[i];
        if (len > maxrow) maxrow = len;
        var = var + ((double)len - mean) * ((double)len - mean);
        for (int64_t k = (int64_t)IA[i] - base; k < (int64_t)IA[i + 1] - base; ++k) {
            int64_t d = (int64_t)(JA[k] - base) - i;
            if (d < 0) d = -d;
            if (d > bw) bw = d;
        }
    }
    out[0] = (double)n;
    out[1] = (double)nz;
    out[2] = n > 0 ? (double)nz / ((double)n * (double)n) : 0.0;
    out[3] = (double)bw;
    out[4] = (double)maxrow;
    out[5] = mean;
    out[6] = n > 0 ? sqrt(var / (double)n) : 0.0;
}
