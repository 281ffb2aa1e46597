/*
 * cg.h — C ABI of the GB300 conjugate-gradient library (libcg.so).
 *
 * Solves sparse symmetric positive definite systems A x = b stored in CSR
 * with the classical, unpreconditioned conjugate gradient method, and
 * exposes the operations that method is built from: the CSR matrix-vector
 * product, the dot product, the addition of vectors and the element-wise
 * product.  These are the operations and the solver benchmarked in
 * "Fast and Green Computing with Graphics Processing Units for solving
 * Sparse Linear Systems" (CSR format: Sec. 2.3; vector operations, dot
 * product and SpMV: Sec. 5.2; CG: Sec. 5.3).
 *
 * Conventions for every entry point:
 *   - Returns a cg_status code; nothing aborts and no C++ exception crosses
 *     the ABI.  cg_last_error() gives a message for the last failure.
 *   - "device" pointers are CUDA global-memory pointers of the handle's
 *     device (e.g. torch.Tensor.data_ptr() of a CUDA tensor).  They are
 *     borrowed: the library never frees or retains them after the call.
 *   - Work is queued on the handle's stream (cg_opts.stream); functions that
 *     produce a host-visible result (cg_solve) synchronise that stream.
 *   - Sizes are int64_t; the CSR arrays use int32_t indices, so n and nnz
 *     must each stay below 2^31 - 16.
 */
#ifndef CG_GB300_H
#define CG_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
typedef enum {
  CG_OK = 0,
  CG_EINVAL = 1,      /* bad argument, or malformed CSR rejected by cg_create */
  CG_ENOMEM = 2,      /* device or pinned-host allocation failed */
  CG_ECUDA = 3,       /* a CUDA runtime call failed; the message names it */
  CG_ENOTCONV = 4,    /* cg_solve: maxit steps done, tolerance not reached */
  CG_EBREAKDOWN = 5,  /* cg_solve: p.Ap <= 0 or not finite (A not SPD, or overflow) */
  CG_ETIMEOUT = 6,    /* a device-side wait exceeded its limit (the solve was abandoned) */
  CG_EBUSY = 7        /* admission refused (no free slot / over the memory budget) */
} cg_status;

/* Opaque solver handle: a CSR matrix resident on one GPU plus the work
 * vectors, partition tables and stream used to operate on it. */
typedef struct cg_ctx* cg_handle;

/* A CSR matrix as the paper defines it (Sec. 2.3): AA = values, JA = column
 * indices (both nnz long, row by row), IA = row starts (n+1 long); row i
 * holds AA[IA[i]-base .. IA[i+1]-base-1].  index_base is 0 or 1 (the paper's
 * arrays are 1-based).  on_device = 1 if the three arrays are device
 * pointers, 0 if host pointers.  Columns need not be sorted; duplicates are
 * kept and summed like any other entry. */
typedef struct {
  const int32_t* row_ptr; /* IA, n+1 entries */
  const int32_t* col_idx; /* JA, nnz entries */
  const double* val;      /* AA, nnz entries */
  int32_t index_base;     /* 0 or 1 */
  int32_t on_device;      /* 1: device pointers; 0: host pointers */
} cg_csr;

/* Precision of the solve. */
typedef enum {
  CG_PREC_FP64 = 0,  /* everything in FP64 (the paper's arithmetic, Sec. 5: double precision) */
  CG_PREC_MIXED = 1  /* FP32 values and FP32-accumulated product; FP64 sums, scalars, x, r;
                        r replaced by the FP64 true residual every replace_every steps */
} cg_precision;

typedef struct {
  void* stream;           /* cudaStream_t for all work of the handle; NULL = legacy default stream */
  int32_t device;         /* CUDA device ordinal; -1 = the current device */
  int32_t precision;      /* cg_precision */
  int32_t replace_every;  /* CG_PREC_MIXED: residual-replacement period in steps (default 50) */
  int32_t validate;       /* 1 (default): check the CSR in cg_create (O(n + nnz) on the host) */
  int32_t wait_limit_ms;  /* bound on any device-side wait inside a kernel (default 2000) */
  int32_t reserved[7];    /* zero */
} cg_opts;

/* Fill *o with the defaults above. */
void cg_opts_default(cg_opts* o);

/*
 * Create a handle for the n x n matrix `csr` with nnz stored entries.
 * The library copies the matrix into device memory it owns (converted to
 * 0-based indices); the caller's arrays may be freed when this returns.
 * With validate = 1 it rejects (CG_EINVAL): index_base not 0/1, row_ptr[0]
 * != base, decreasing row_ptr, row_ptr[n] != nnz + base, a column outside
 * [base, n + base).  n = 0 is allowed (every call is then a no-op).
 * opts may be NULL (defaults).  On failure *out is NULL.
 */
int cg_create(cg_handle* out, const cg_csr* csr, int64_t n, int64_t nnz, const cg_opts* opts);

/* Release everything the handle owns.  NULL is accepted. */
int cg_destroy(cg_handle h);

/* Message of the last failure on h (or of the last failed cg_create on this
 * thread when h is NULL).  Valid until the next call on h / this thread. */
const char* cg_last_error(cg_handle h);

/* Matrix size of the handle (n, nnz) and the CTA count of its partition. */
int cg_info(cg_handle h, int64_t* n, int64_t* nnz, int32_t* nblocks);

/*
 * y = A x (Sec. 2.3 / 5.2): y_i = sum_{k=IA(i)}^{IA(i+1)-1} AA(k) x(JA(k)),
 * FP64 with FMA, each row summed in storage order.  x, y: device pointers to
 * n doubles; x and y must not overlap.  Asynchronous on the handle's stream.
 */
int cg_spmv(cg_handle h, const double* x, double* y);

/*
 * *result = sum_i x_i y_i over n elements (Sec. 5.2 "dot product").
 * x, y: device pointers to n doubles; result: device pointer to one double.
 * Deterministic for a given n: same inputs give the same bits.  Uses the
 * handle's device scratch, so calls on one handle must not overlap in time.
 * n may differ from the matrix size.  Asynchronous.
 */
int cg_dot(cg_handle h, int64_t n, const double* x, const double* y, double* result);

/* y <- a x + y over n elements (Sec. 5.2 "addition of vectors"), FMA.
 * Device pointers; x and y must not overlap.  Asynchronous. */
int cg_axpy(cg_handle h, int64_t n, double a, const double* x, double* y);

/* z_i = x_i * y_i over n elements (Sec. 5.2 "element wise product").
 * Device pointers; z may alias x or y exactly.  Asynchronous. */
int cg_ewmul(cg_handle h, int64_t n, const double* x, const double* y, double* z);

/*
 * Solve A x = b by classical CG (Sec. 5.3; Hestenes-Stiefel form):
 *   r = b - A x0, p = r; each step q = A p, alpha = r.r / p.q,
 *   x += alpha p, r -= alpha q, beta = r'.r' / r.r, p = r' + beta p;
 *   stop when ||r|| <= tol ||b|| (recursive residual; in CG_PREC_MIXED the
 *   replaced, true residual).
 * b (n doubles) and x (n doubles; in: initial guess, out: solution) may be
 * device or host pointers (each detected separately; host memory is copied
 * in and out inside the call).  One persistent cooperative kernel runs the
 * whole iteration; alpha, beta and the stopping test are computed on the
 * device.  Synchronous: returns after x and the outputs are written.
 * Outputs: *iters = steps taken (each step is one product with p);
 *          *relres = ||b - A x|| / ||b|| recomputed in FP64 at exit.
 * Returns CG_OK (converged), CG_ENOTCONV (maxit reached; x is the last
 * iterate), CG_EBREAKDOWN (x is the last iterate before the failing step),
 * CG_ETIMEOUT, CG_EINVAL (tol < 0 or NaN, maxit < 0, NULL outputs).
 * b = 0 gives x = 0, *iters = 0, *relres = 0.
 */
int cg_solve(cg_handle h, const double* b, double* x, double tol, int64_t maxit, int64_t* iters,
             double* relres);

/*
 * *result = sum_i x_i y_i over n elements, like cg_dot, but without a handle
 * and without allocating anything.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate GPU memory at the moment they
 * need a dot product, for example code running under a fixed memory budget
 * that forbids allocation after start-up, code called from inside another
 * allocator or memory pool that must not be re-entered, or latency-critical
 * loops that cannot afford cudaMalloc's implicit device synchronisation.
 * (cg_create, which cg_dot needs, allocates device memory.)
 *
 * x, y: device pointers to n doubles; result: device pointer to one double;
 * stream: cudaStream_t (NULL = legacy default stream).  Asynchronous.
 * The scratch (per-CTA partial sums and an arrival counter) is one fixed
 * array of about 128 KB compiled into the library, so n is limited to
 * 33,554,432 elements (CG_EINVAL beyond, with a message).  Every GPU that
 * loads the library holds that array until the process exits.
 * The first call on each device looks up the array's device address (a CUDA
 * runtime call made with that device current); make that first call before
 * any stream capture.  All calls share the one array: calls that overlap on
 * the GPU (different streams, or different host threads) race and give wrong
 * results; serialise them.  Each call clears the counter it needs before its
 * kernel runs.  Deterministic for a given n.
 */
int cg_dot_noalloc(int64_t n, const double* x, const double* y, double* result, void* stream);

/*
 * Self-test of the library's bounded device-side waits (no paper
 * counterpart): launches a one-CTA kernel that waits at a grid barrier no
 * other CTA will reach.  The wait must give up after limit_ms and the kernel
 * must report CG_ETIMEOUT, leaving the CUDA context usable.  *kernel_status
 * receives the status the kernel wrote.  Runs on the current device and the
 * legacy default stream; synchronous.
 */
int cg_selftest_wait_timeout(int32_t limit_ms, int32_t* kernel_status);

#ifdef __cplusplus
}
#endif

#endif /* CG_GB300_H */
