/*
 * ORACLE, multi-core timing variant — test infrastructure only.
 *
 * The same classical conjugate gradient as oracle_cg in cg_oracle.c (Sec. 5.3,
 * Hestenes-Stiefel form; CSR product of Sec. 2.3), with every vector loop
 * spread over the host's cores with OpenMP.  It exists so that the CPU
 * baseline runs on all host cores and so that systems too large for the
 * single-threaded oracle (the 160^3 Q1 system) can still be solved on the
 * host.  It is pinned against the single-threaded oracle, never the other way
 * round: with one thread every result is the sequential oracle's to the bit;
 * with more, the products are still bit-identical, the iterates agree within
 * summation-order rounding and the stopping steps within max(2, 1 %).  Like
 * the sequential oracle, only the tests, the smoke check and the CPU legs of
 * the benchmark call it; it shares no code with the CUDA library.
 *
 * Arithmetic: each row of a product is summed in storage order exactly as
 * oracle_spmv does (same bits).  A dot product is split into T contiguous
 * blocks (T = the thread count), each summed in index order, and the T block
 * sums are added in block order: deterministic for a given T, and the only
 * difference from the sequential oracle.  Compiled with -ffp-contract=off
 * like the sequential oracle.
 */
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>

int oracle_omp_threads(void) { return omp_get_max_threads(); }

/* Threads of the calls that follow (T = 1 makes every result equal to the
 * sequential oracle's, bit for bit). */
void oracle_omp_set_threads(int t) {
    if (t > 0) omp_set_num_threads(t);
}

/* Block t of T over [0, n). */
static void block_range(int64_t n, int t, int T, int64_t* lo, int64_t* hi) {
    *lo = (n * t) / T;
    *hi = (n * (t + 1)) / T;
}

/* y = A x, rows in parallel, each row in storage order. */
void oracle_omp_spmv(int64_t n, const int32_t* IA, const int32_t* JA, const double* AA, int base,
                     const double* x, double* y) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t k = (int64_t)IA[i] - base; k < (int64_t)IA[i + 1] - base; ++k)
            s = s + AA[k] * x[JA[k] - base];
        y[i] = s;
    }
}

/* x.y: block sums in parallel, then added in block order.  part holds T doubles. */
static double omp_dot(int64_t n, const double* x, const double* y, double* part, int T) {
#pragma omp parallel num_threads(T)
    {
        int t = omp_get_thread_num();
        int64_t lo, hi;
        block_range(n, t, T, &lo, &hi);
        double s = 0.0;
        for (int64_t i = lo; i < hi; ++i) s = s + x[i] * y[i];
        part[t] = s;
    }
    double s = 0.0;
    for (int t = 0; t < T; ++t) s = s + part[t];
    return s;
}

double oracle_omp_dot(int64_t n, const double* x, const double* y) {
    int T = omp_get_max_threads();
    double* part = (double*)malloc(sizeof(double) * (size_t)T);
    if (!part) return NAN;
    double s = omp_dot(n, x, y, part, T);
    free(part);
    return s;
}

#define ORC_OK 0
#define ORC_NOTCONV 4
#define ORC_BREAKDOWN 5
#define ORC_NOMEM 2

/*
 * Classical CG, the steps and outputs of oracle_cg (x in/out, force_iters >= 0
 * runs exactly that many steps, b = 0 gives x = 0):
 *   r = b - A x;  p = r;  rho = r.r
 *   repeat: q = A p; gamma = p.q (breakdown if <= 0 or not finite);
 *           alpha = rho/gamma; x += alpha p; r -= alpha q; rho' = r.r;
 *           stop if sqrt(rho') <= tol ||b||; beta = rho'/rho; p = r + beta p.
 */
int oracle_omp_cg(int64_t n, const int32_t* IA, const int32_t* JA, const double* AA, int base,
                  const double* b, double* x, double tol, int64_t maxit, int64_t force_iters,
                  int64_t* iters, double* relres_rec, double* relres_true) {
    size_t m = (size_t)(n > 0 ? n : 1);
    int T = omp_get_max_threads();
    double* r = (double*)malloc(sizeof(double) * m);
    double* p = (double*)malloc(sizeof(double) * m);
    double* q = (double*)malloc(sizeof(double) * m);
    double* part = (double*)malloc(sizeof(double) * (size_t)T);
    if (!r || !p || !q || !part) { free(r); free(p); free(q); free(part); return ORC_NOMEM; }
    int status = ORC_OK;
    double bnorm = sqrt(omp_dot(n, b, b, part, T));
    *iters = 0;
    if (bnorm == 0.0) {
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
        *relres_rec = 0.0; *relres_true = 0.0;
        free(r); free(p); free(q); free(part);
        return ORC_OK;
    }
    oracle_omp_spmv(n, IA, JA, AA, base, x, q);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) { r[i] = b[i] - q[i]; p[i] = r[i]; }
    double rho = omp_dot(n, r, r, part, T);
    int64_t k = 0;
    int done = (force_iters < 0) && (sqrt(rho) <= tol * bnorm);
    int64_t limit = force_iters >= 0 ? force_iters : maxit;
    while (!done && k < limit) {
        oracle_omp_spmv(n, IA, JA, AA, base, p, q);
        double gamma = omp_dot(n, p, q, part, T);
        if (!(gamma > 0.0) || !isfinite(gamma)) { status = ORC_BREAKDOWN; break; }
        double alpha = rho / gamma;
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) x[i] = x[i] + alpha * p[i];
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) r[i] = r[i] - alpha * q[i];
        double rho_new = omp_dot(n, r, r, part, T);
        k = k + 1;
        if (force_iters < 0 && sqrt(rho_new) <= tol * bnorm) { rho = rho_new; done = 1; break; }
        double beta = rho_new / rho;
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
        rho = rho_new;
    }
    *iters = k;
    *relres_rec = sqrt(rho) / bnorm;
    if (status == ORC_OK && force_iters < 0 && !done) status = ORC_NOTCONV;
    oracle_omp_spmv(n, IA, JA, AA, base, x, q);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) q[i] = b[i] - q[i];
    *relres_true = sqrt(omp_dot(n, q, q, part, T)) / bnorm;
    free(r); free(p); free(q); free(part);
    return status;
}

/*
 * Mixed-precision CG with residual replacement, the steps and outputs of
 * oracle_cg_mixed in cg_oracle.c (FP32 values AA32 and FP32-accumulated
 * product, each row in storage order; FP64 dots, scalars, x, r and p; r
 * replaced by the FP64 true residual every replace_every steps and whenever
 * the recursive residual reaches tol*||b||, the direction keeping the
 * recurrence's beta; convergence on the true residual; force_iters >= 0 runs
 * exactly that many steps) with every vector loop spread over the host's
 * cores.  The FP32 and FP64 products are the sequential oracle's to the bit;
 * the dots are summed in T blocks added in block order.
 */
int oracle_omp_cg_mixed(int64_t n, const int32_t* IA, const int32_t* JA, const double* AA, const float* AA32,
                        int base, const double* b, double* x, double tol, int64_t maxit, int64_t replace_every,
                        int64_t force_iters, int64_t* iters, double* relres_rec, double* relres_true) {
    size_t m = (size_t)(n > 0 ? n : 1);
    int T = omp_get_max_threads();
    double* r = (double*)malloc(sizeof(double) * m);
    double* p = (double*)malloc(sizeof(double) * m);
    double* q = (double*)malloc(sizeof(double) * m);
    float* p32 = (float*)malloc(sizeof(float) * m);
    double* part = (double*)malloc(sizeof(double) * (size_t)T);
    if (!r || !p || !q || !p32 || !part) { free(r); free(p); free(q); free(p32); free(part); return ORC_NOMEM; }
    int status = ORC_OK;
    double bnorm = sqrt(omp_dot(n, b, b, part, T));
    *iters = 0;
    if (bnorm == 0.0) {
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
        *relres_rec = 0.0; *relres_true = 0.0;
        free(r); free(p); free(q); free(p32); free(part);
        return ORC_OK;
    }
    oracle_omp_spmv(n, IA, JA, AA, base, x, q);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) { r[i] = b[i] - q[i]; p[i] = r[i]; }
    double rho = omp_dot(n, r, r, part, T);
    int64_t k = 0;
    int done = (force_iters < 0) && (sqrt(rho) <= tol * bnorm);
    int64_t limit = force_iters >= 0 ? force_iters : maxit;
    while (!done && k < limit) {
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) p32[i] = (float)p[i];
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            float s = 0.0f;
            for (int64_t kk = (int64_t)IA[i] - base; kk < (int64_t)IA[i + 1] - base; ++kk)
                s = s + AA32[kk] * p32[JA[kk] - base];
            q[i] = (double)s;
        }
        double gamma = omp_dot(n, p, q, part, T);
        if (!(gamma > 0.0) || !isfinite(gamma)) { status = ORC_BREAKDOWN; break; }
        double alpha = rho / gamma;
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) x[i] = x[i] + alpha * p[i];
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) r[i] = r[i] - alpha * q[i];
        double rho_new = omp_dot(n, r, r, part, T);
        double beta = rho_new / rho;
        k = k + 1;
        int replace = (replace_every > 0 && k % replace_every == 0) || sqrt(rho_new) <= tol * bnorm;
        if (replace) {
            oracle_omp_spmv(n, IA, JA, AA, base, x, q);
#pragma omp parallel for schedule(static)
            for (int64_t i = 0; i < n; ++i) r[i] = b[i] - q[i];
            rho_new = omp_dot(n, r, r, part, T);
            if (force_iters < 0 && sqrt(rho_new) <= tol * bnorm) { rho = rho_new; done = 1; break; }
        }
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
        rho = rho_new;
    }
    *iters = k;
    *relres_rec = sqrt(rho) / bnorm;
    if (status == ORC_OK && force_iters < 0 && !done) status = ORC_NOTCONV;
    oracle_omp_spmv(n, IA, JA, AA, base, x, q);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) q[i] = b[i] - q[i];
    *relres_true = sqrt(omp_dot(n, q, q, part, T)) / bnorm;
    free(r); free(p); free(q); free(p32); free(part);
    return status;
}
