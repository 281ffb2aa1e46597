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
 *     device, or of the current device for the calls without a handle
 *     (e.g. torch.Tensor.data_ptr() of a CUDA tensor).  They are borrowed:
 *     the library never frees or retains them after the call.
 *   - Work of a handle is queued on the handle's stream (cg_opts.stream);
 *     the vector calls without a handle take their stream as an argument.
 *     Functions that produce a host-visible result (cg_solve, cg_dot_host)
 *     synchronise their stream.
 *   - Sizes are int64_t; the CSR arrays use int32_t indices, so n and nnz
 *     must each stay below 2^31 - 16.
 *   - Threads: a handle holds the work vectors of one solve, so calls on
 *     one handle must not overlap (use one handle per thread); the calls
 *     without a handle and the batch API may be used from any thread.
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

/* Preconditioner of cg_solve (the paper's CG has none; it defers
 * preconditioning to domain decomposition). */
typedef enum {
  CG_PRECOND_NONE = 0,   /* classical CG (default) */
  CG_PRECOND_JACOBI = 1  /* M = diag(A): z = diag(A)^-1 r by the element-wise product;
                            the stopping test stays ||r|| <= tol ||b|| */
} cg_preconditioner;

typedef struct {
  void* stream;           /* cudaStream_t for all work of the handle; NULL = legacy default stream */
  int32_t device;         /* CUDA device ordinal; -1 = the current device */
  int32_t precision;      /* cg_precision */
  int32_t replace_every;  /* CG_PREC_MIXED: residual-replacement period in steps (default 50) */
  int32_t validate;       /* 1 (default): check the CSR in cg_create (O(n + nnz) on the host) */
  int32_t wait_limit_ms;  /* bound on any device-side wait inside a kernel (default 2000) */
  int32_t preconditioner; /* cg_preconditioner (default CG_PRECOND_NONE) */
  int32_t ctas;           /* CTAs of the persistent kernels (at most one per SM); 0 (default):
                             one per SM */
  int32_t reserved[5];    /* zero */
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
 * With preconditioner = CG_PRECOND_JACOBI the inverse diagonal is computed
 * on the device (each row's entries in its own column summed); a diagonal
 * that is not positive (A cannot be SPD) is refused with CG_EINVAL.
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

/* The kernel cg_solve runs on a handle (cg_partition_info). */
enum {
  CG_SOLVE_KERNEL_LARGE_SHARE = 0, /* whole grid; residual in global memory, x updated with p, each
                                      step ending with a wait for the CTAs that own the columns of
                                      the CTA's rows only */
  CG_SOLVE_KERNEL_SMALL_SHARE = 1, /* whole grid, every CTA range at most 2560 rows: the range's
                                      residual in shared memory, x updated behind the r.r barrier */
  CG_SOLVE_KERNEL_CLUSTER = 2      /* plain FP64, at most 16384 rows whose CSR fits the CTAs' shared
                                      memory, CTA count left automatic: one cluster of 16 CTAs holding
                                      the system in shared memory */
};

/*
 * The partition of the kernel cg_solve runs: *max_rows = the most rows in
 * one CTA's range; *kernel = one of CG_SOLVE_KERNEL_*.  The two whole-grid
 * kernels give the same bits; the cluster kernel sums over 16 CTAs instead of
 * the grid's, so its bits differ within rounding.  Either pointer may be
 * NULL.  Host only: no GPU work.
 */
int cg_partition_info(cg_handle h, int32_t* max_rows, int32_t* kernel);

/*
 * y = A x (Sec. 2.3 / 5.2): y_i = sum_{k=IA(i)}^{IA(i+1)-1} AA(k) x(JA(k)),
 * FP64 with FMA, each row summed in storage order.  x, y: device pointers to
 * n doubles; x and y must not overlap.  Asynchronous on the handle's stream.
 */
int cg_spmv(cg_handle h, const double* x, double* y);

/* ------------------------------------------------------------------------
 * The vector operations of Sec. 5.2 ("Vectors operations" and "Dot product"
 * tables) as stand-alone calls: no handle.  x, y, z and result are device
 * pointers of the CURRENT CUDA device (cudaSetDevice before the call if
 * several are in use) and `stream` a cudaStream_t of that device (NULL = the
 * legacy default stream).  Work is queued on `stream`; the calls return at
 * once except cg_dot_host.
 * ---------------------------------------------------------------------- */

/*
 * *result = sum_i x_i y_i over n elements (Sec. 5.2 "dot product"); result:
 * device pointer to one double.  When x and y are 16-byte aligned and n is at
 * least 32768 the sum streams through a bulk-copy ring (one CTA per SM);
 * otherwise a grid-stride kernel runs.  Deterministic: the same n and
 * alignment of x and y give the same bits.
 * Scratch: the first call on a (device, stream) pair allocates about 8 KB of
 * device memory (cudaMalloc, so make that first call outside any stream
 * capture), which later calls on the same pair reuse and cg_blas_release()
 * frees.  Calls on one stream run in order, so they may share it; calls on
 * different streams get different scratch (cudaStreamPerThread counts as a
 * different stream in every host thread).  If a device-side wait of the
 * kernel gives up (only a fault of the copy engine could cause it), *result
 * is NaN; cg_dot_host reports it as CG_ETIMEOUT.
 */
int cg_dot(int64_t n, const double* x, const double* y, double* result, void* stream);

/*
 * cg_dot with the sum written to *result in host memory: the same kernel (the
 * same bits) into the scratch's device scalar, then a copy to the host and a
 * synchronisation of `stream`.  Synchronous; for tests and callers without a
 * device buffer.
 */
int cg_dot_host(int64_t n, const double* x, const double* y, double* result, void* stream);

/* y <- a x + y over n elements (Sec. 5.2 "addition of vectors"), one FMA per
 * element.  x and y must not overlap.  16-byte accesses when both are
 * 16-byte aligned.  No scratch. */
int cg_axpy(int64_t n, double a, const double* x, double* y, void* stream);

/* z_i = x_i * y_i over n elements (Sec. 5.2 "element wise product"); z may
 * alias x or y exactly.  No scratch. */
int cg_ewmul(int64_t n, const double* x, const double* y, double* z, void* stream);

/* Free the dot product's scratch of every (device, stream) pair.  No call of
 * cg_dot / cg_dot_host may be queued or running on any of them.  Later calls
 * allocate again. */
int cg_blas_release(void);

/*
 * FP64 fused multiply-add throughput of `device` (-1 = the current device)
 * in GFLOP/s (2 flops per FMA): a kernel of 2, 4 and 8 CTAs of 256 threads
 * per SM, each thread running eight independent FMA chains, timed with CUDA
 * events over about 40 ms per launch (the best of three timed launches after
 * two warm-up launches, for each CTA count).  The ceiling of the ALU roofline that the CG solves of systems
 * resident in L2 are held against; no counterpart in the paper, which
 * reports times only.  Synchronous; allocates and frees a small buffer.
 */
int cg_probe_fp64_peak(int32_t device, double* gflops);

/*
 * The cost of the solves' group-wide synchronisations, measured on the
 * device (no counterpart in the paper; it explains the time of a step that
 * the FP64 pipe does not).  A cooperative launch of one CTA per SM, the
 * solve kernels' block, runs `iters` group barriers (*barrier_us: the
 * barrier a solve step ends with) and then `iters` group sums
 * (*sum_us: a CTA value published, the barrier, the group's values summed
 * exactly in fixed point, as for alpha and beta), each between CTA barriers
 * as in a step; the results are microseconds per barrier and per sum (CUDA
 * events, one warm-up launch first).  device < 0: the current device.
 * iters in [1, 10^6] (2*10^4 takes about 0.1 s).  Returns CG_ETIMEOUT if a
 * wait gave up (2 s), CG_EINVAL for bad arguments.
 */
int cg_probe_group_sync(int32_t device, int32_t iters, double* barrier_us, double* sum_us);

/*
 * Solve A x = b by classical CG (Sec. 5.3; Hestenes-Stiefel form):
 *   r = b - A x0, p = r; each step q = A p, alpha = r.r / p.q,
 *   x += alpha p, r -= alpha q, beta = r'.r' / r.r, p = r' + beta p;
 *   stop when ||r|| <= tol ||b|| (recursive residual; in CG_PREC_MIXED the
 *   replaced, true residual).  With CG_PRECOND_JACOBI: z = diag(A)^-1 r,
 *   r.z in place of r.r in alpha and beta, p = z' + beta p; same test.
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
 * *result = sum_i x_i y_i over n elements, like cg_dot, but without
 * allocating anything.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate GPU memory at the moment they
 * need a dot product, for example code running under a fixed memory budget
 * that forbids allocation after start-up, code called from inside another
 * allocator or memory pool that must not be re-entered, or latency-critical
 * loops that cannot afford cudaMalloc's implicit device synchronisation.
 * (cg_dot allocates its scratch on the first call for each stream.)
 *
 * x, y: device pointers to n doubles and result a device pointer to one
 * double, all of the CURRENT CUDA device, and stream a cudaStream_t of that
 * device (NULL = legacy default stream): the call finds the array's address
 * on the current device, so memory or a stream of another device would be
 * paired with the wrong array.  Asynchronous.
 * The scratch (per-CTA partial sums and an arrival counter) is one fixed
 * array of about 128 KB compiled into the library, so n is limited to
 * 33,554,432 elements (CG_EINVAL beyond, with a message).  Every GPU that
 * loads the library holds that array until the process exits.
 * The first call on each device looks up the array's device address (a CUDA
 * runtime call made with that device current); make that first call before
 * any stream capture.  The cached address belongs to the device's current
 * context: after cudaDeviceReset the array must not be used again in that
 * process.  All calls share the one array: calls that overlap on
 * the GPU (different streams, or different host threads) race and give wrong
 * results; serialise them.  Each call clears the counter it needs before its
 * kernel runs.  Deterministic for a given n.
 */
int cg_dot_noalloc(int64_t n, const double* x, const double* y, double* result, void* stream);

/*
 * Self-test of the library's bounded device-side waits (no paper
 * counterpart): launches a one-CTA kernel whose thread 0 waits at the solves'
 * group barrier for a group of two CTAs that no other CTA joins.  The wait
 * must give up after limit_ms, raise the solve's abort flag and report
 * CG_ETIMEOUT, leaving the CUDA context usable.  *kernel_status receives the
 * status the kernel wrote; the call returns CG_ECUDA if the wait gave up
 * without raising the abort flag.  Runs on the current device and the legacy
 * default stream; synchronous.
 */
int cg_selftest_wait_timeout(int32_t limit_ms, int32_t* kernel_status);

/* ------------------------------------------------------------------------
 * Batched and served solves: many independent systems on one GPU.
 *
 * The paper solves one system at a time (Sec. 5.3); these entry points
 * extend the same classical CG to many independent SPD systems sharing one
 * GPU.  A batch object owns a device memory budget, a table of resident
 * systems and a worker thread.  cg_batch_submit() queues requests and
 * returns at once; the worker admits queued requests in arrival order as
 * memory and slots free up (copying each matrix and right-hand side into the
 * budget), and advances every resident system with one persistent
 * cooperative kernel launch per round (replayed from a captured CUDA graph):
 * each CTA takes systems from a queue; a large system is solved by a group
 * of CTAs with its own group barrier, most by one CTA.  With chunk_iters > 0
 * each round advances every system at most chunk_iters steps, so requests
 * that arrive meanwhile join at the next round (continuous batching); with
 * chunk_iters = 0 a round runs every resident system to its end (one launch
 * for a batch that fits the budget).  A finished system's solution is
 * copied to the request's x and its memory released before the next round.
 *
 * The arithmetic of every system is that of cg_solve with the batch's
 * precision (x0 = 0; the same stopping test and outputs; the product's step
 * shapes, and so the split of a row's sum, follow the batch object's table,
 * see cg_batch_opts.autotune and step_shape).  How many CTAs
 * solve a system (its "group") is chosen from the system alone (its rows,
 * entries and row lengths), never from the rest of the batch, so a system
 * gives the same bits alone and in any mix on the same batch object.  The
 * choice is the smallest group whose estimated solo solve time meets
 * group_target_ms under a cost model (per-CTA streaming rate and per-step overheads) that
 * cg_batch_opts.autotune measures on the GPU at creation; a group has at most half the
 * CTAs of the persistent grid and at least 1024 rows per CTA, and when no group meets the
 * target the largest one is taken.
 * ---------------------------------------------------------------------- */

typedef struct cg_batch_ctx* cg_batch;

typedef struct {
  int32_t device;          /* CUDA device ordinal; -1 = the current device */
  int32_t precision;       /* cg_precision of every system of the batch */
  int64_t budget_bytes;    /* device memory for resident systems (matrices, vectors,
                              partition tables); 0 = half of the free memory at creation */
  int32_t max_systems;     /* resident systems at most (default 1024) */
  int32_t chunk_iters;     /* steps per system per round; 0 = until the system ends */
  int32_t replace_every;   /* CG_PREC_MIXED residual-replacement period (default 50) */
  int32_t wait_limit_ms;   /* bound on any device-side wait (default 2000) */
  int32_t max_pending;     /* queued requests not yet admitted (default 65536) */
  int32_t use_graph;       /* 1 (default): replay each round from a captured CUDA graph */
  int32_t group_override;  /* > 0: every system uses this many CTAs (tests); 0 = automatic */
  int32_t validate;        /* 1 (default): check each request's CSR on the host */
  int32_t preconditioner;  /* cg_preconditioner of every system (a non-positive diagonal
                              ends that request with CG_EINVAL) */
  int32_t autotune;        /* 1: at creation, measure on this GPU which step shape (one lane,
                              two lanes or a warp per row) the product runs fastest with for
                              each bucket of row lengths, then the group-size cost model, with
                              synthetic systems (about a second of rounds); 0 (default):
                              built-in shapes and constants */
  int32_t group_target_ms; /* solo solve time the automatic group size aims at (default 50:
                              smaller favours latency, larger favours throughput).  Keep it
                              well below wait_limit_ms when chunk_iters is 0: the first
                              ranks of a group may wait at their first barrier for about
                              one task (up to one solo solve) to end */
  int32_t step_shape;      /* 0 (default): the built-in step shapes, or the measured ones with
                              autotune; 1: the built-in shapes (one lane per row up to 32
                              entries, two lanes up to 64) even with autotune; 2: two lanes per
                              row up to 64 entries; 3: a warp per row.  Rows of more than 64
                              entries always take a warp each. */
  int32_t reserved[2];     /* zero */
} cg_batch_opts;

/* One system to solve: A x = b from x0 = 0. */
typedef struct {
  cg_csr csr;              /* the matrix (host or device arrays) */
  int64_t n, nnz;
  const double* b;         /* n doubles, host or device */
  double* x;               /* n doubles, host or device: receives the solution */
  double tol;              /* relative residual target (as cg_solve) */
  int64_t maxit;           /* step limit (as cg_solve) */
  uint64_t tag;            /* caller's value, returned in the result */
} cg_request;

typedef struct {
  uint64_t ticket;
  uint64_t tag;
  int32_t done;            /* 1 once the request has ended (status and x final) */
  int32_t status;          /* as cg_solve: CG_OK, CG_ENOTCONV, CG_EBREAKDOWN, CG_ETIMEOUT,
                              or CG_EINVAL / CG_ENOMEM / CG_ECUDA if it could not be admitted */
  int64_t iters;           /* steps taken */
  double relres;           /* ||b - A x|| / ||b|| recomputed in FP64 at exit */
  double submit_ms;        /* host times in ms since the batch object was created: */
  double admit_ms;         /*   queued, resident on the device, */
  double done_ms;          /*   solution written to x */
  int32_t group;           /* CTAs that solved the system */
  int32_t rounds;          /* rounds (kernel launches) the system took part in */
} cg_result;

typedef struct {
  int64_t rounds;          /* persistent kernel launches so far */
  int64_t submitted, admitted, completed;
  int64_t pending;         /* queued, not yet admitted */
  int64_t resident;        /* on the device now */
  int64_t bytes_in_use, bytes_peak, budget_bytes;
  int32_t graph;           /* 1 if rounds are replayed from a CUDA graph */
  int32_t nblocks;         /* CTAs of the persistent kernel */
  double round_ms_total;   /* device time of all rounds (CUDA events around each) */
  double last_round_ms;    /* device time of the last round */
  /* cost model of the automatic group size (measured if autotuned): a step of
   * a system on G CTAs takes bytes_per_step / (G * cta_bytes_per_s) + overhead */
  double cta_bytes_per_s;          /* one CTA's streaming rate with every SM busy, G = 1 */
  double group_cta_bytes_per_s;    /* the same inside a group of several CTAs */
  double step_overhead_s;          /* per step, G = 1 */
  double group_step_overhead_s;    /* per step, G > 1 */
  int32_t autotuned;               /* 1 if the model was measured */
  /* step shapes of the product (measured with autotune, else built in): the
   * kind of step rows of (0,8], (8,16], (16,24], (24,32], (32,48], (48,64]
   * entries go to: 0 = one lane per row (up to 32 rows per warp step), 1 = two
   * lanes per row (up to 16 rows), 2 = one warp per row.  Rows of more than
   * 64 entries always take a warp each. */
  int32_t shape_tuned;             /* 1 if the step shapes were measured */
  int32_t step_kind[6];
  int32_t pad;
  /* rounds whose product loaded the row pointers with the evict-first L2
   * policy: those whose systems' vectors and row pointers together take
   * more than 4/7 of the L2 (the row pointers then give way to the vectors
   * that every step reads again) */
  int64_t rounds_stream_rows;
} cg_batch_stats;

/* Fill *o with the defaults above. */
void cg_batch_opts_default(cg_batch_opts* o);

/* Create a batch object: reserves budget_bytes of device memory, the system
 * table and the worker thread.  opts may be NULL.  On failure *out is NULL
 * and cg_batch_last_error(NULL) gives the reason. */
int cg_batch_create(cg_batch* out, const cg_batch_opts* opts);

/* Stop the worker (after the round in flight), drop queued requests and
 * release everything.  Pointers of unfinished requests are never touched
 * again.  No other call on b may run concurrently with this one or follow
 * it.  NULL is accepted.  The other cg_batch_* calls may be made from any
 * number of host threads at once. */
int cg_batch_destroy(cg_batch b);

/*
 * Queue `count` requests; tickets[i] receives the ticket of reqs[i].
 * Non-blocking: the matrices are copied when the worker admits a request,
 * so every array a request names (csr arrays, b, x) must stay valid and
 * unchanged until its result is done.  Device arrays must already hold
 * their values (synchronise the stream that wrote them before submitting):
 * the worker copies them on a stream of its own.  Returns CG_EINVAL (bad request: NULL
 * pointer, n or nnz out of range, tol < 0, maxit < 0; nothing is queued),
 * CG_ENOMEM (a request needs more memory than the whole budget; nothing is
 * queued) or CG_EBUSY (the pending queue is full; nothing is queued).
 * A CSR that fails validation is reported in that request's result
 * (status CG_EINVAL) when the worker reaches it.
 */
int cg_batch_submit(cg_batch b, const cg_request* reqs, int32_t count, uint64_t* tickets);

/* Result of a ticket so far: res->done = 0 while it is queued or running.
 * Once a done result has been returned, the ticket is forgotten (a later
 * poll gives CG_EINVAL). */
int cg_batch_poll(cg_batch b, uint64_t ticket, cg_result* res);

/* As cg_batch_poll, but waits up to timeout_ms (< 0: without limit) for the
 * request to end; res->done tells whether it did. */
int cg_batch_wait(cg_batch b, uint64_t ticket, int32_t timeout_ms, cg_result* res);

/* Counters of the batch object (a consistent snapshot). */
int cg_batch_get_stats(cg_batch b, cg_batch_stats* st);

/* Group size (CTAs) the batch object would give an n-row system with the
 * row pointers row_ptr (host, n+1 entries, base 0 or 1): the automatic
 * choice from the system alone. */
int cg_batch_group_for(cg_batch b, const int32_t* row_ptr, int64_t n, int32_t* group);

/* Message of the last failure on b (or of the last failed cg_batch_create on
 * this thread when b is NULL). */
const char* cg_batch_last_error(cg_batch b);

#ifdef __cplusplus
}
#endif

#endif /* CG_GB300_H */
