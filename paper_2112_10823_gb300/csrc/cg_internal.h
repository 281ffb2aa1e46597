// Internal structures shared by the host side of the C-ABI and the kernels.
// Not part of the public interface (that is include/cg.h).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace cgk {

// The persistent kernels run one CTA per SM: kConsumerWarps consumer warps
// that compute, plus one producer warp that streams the CSR matrix into a
// shared-memory ring with 1-D TMA bulk copies (warp specialisation).
constexpr int kConsumerWarps = 15;  // with the producer: four warps per SM sub-partition
constexpr int kConsumers = kConsumerWarps * 32;  // 480 computing threads
constexpr int kBlock = kConsumers + 32;          // + the producer warp
constexpr int kCtasPerSm = 1;
constexpr int kWarps = kConsumerWarps;           // warps taking part in CTA reductions

// Matrix stream of a CTA: its CSR values and column indices, one pass after
// another, flow through a ring of kSlots pieces of kPiece entries.  Each slot
// has a "full" mbarrier (TMA completion) and an "empty" mbarrier on which
// every consumer warp arrives once it no longer needs the piece.
constexpr int kPieceLog = 11;
constexpr int kPiece = 1 << kPieceLog;  // 2048 entries: 16 KB of FP64 values + 8 KB of indices
constexpr int kSlots = 8;
constexpr int kRing = kPiece * kSlots;  // 16384 entries
constexpr int kRingMask = kRing - 1;
// Entries mirrored behind the end of the ring: the head of the piece in
// slot 0 is copied there as well, so a row segment of up to kMirror entries
// starting anywhere in the ring reads contiguously, without wrapping.
constexpr int kMirror = 32;
// A step is what a consumer warp computes at once: up to 32 rows of <= 32
// entries (one lane per row), up to 16 rows of 33..64 entries (two lanes per
// row), both at most kStepNnz entries (so they span at most two pieces), or
// one longer row, whose entries the warp walks piece by piece (lanes stride
// them), releasing each piece as soon as it is done with it, so a row may be
// longer than the ring.  Steps of a CTA go to its consumer warps round-robin.
constexpr int kStepNnz = 1024;
constexpr int kLaneMax = 32;  // longest row computed by a single lane
// Largest CTA share (rows) of the small-share solve kernels, which keep the
// share's r in shared memory (20 KB behind the ring layout; the FP64 layout
// then takes 218 KB of the 227 KB a CTA may have).
constexpr int kLocalRows = 2560;

// Padding (in entries) behind val/col allocations so that rounding a copy's
// end up to 16 bytes never reads past the allocation.
constexpr int kPadEntries = 8;

enum StepMode : int32_t {
  kLanePerRow = 0,   // lane l computes row r0 + l (rows of <= kLaneMax entries)
  kPairPerRow = 1,   // lanes 2t, 2t+1 split row r0 + t (rows of <= 2 kLaneMax entries)
  kLongRow = 2,      // the whole row r0 (entries [e0, e1)); lanes stride it
};
// Bits 8..15 of a step's mode word: the longest per-lane segment of the step
// (precomputed so that the lanes need no warp reduction to bound their loops).
constexpr int kWmaxShift = 8;

// Device view of a CSR matrix with its step partition.
struct DevCsr {
  const int32_t* row_ptr;     // [n+1], 0-based
  const int32_t* col_idx;     // [nnz + kPadEntries]
  const double* val;          // [nnz + kPadEntries]
  const float* val32;         // [nnz + kPadEntries] FP32 copy (mixed precision) or nullptr
  const int4* step;           // [nsteps + 2] {r0, r1, e0, e1} (two trailing sentinels)
  const int32_t* step_mode;   // [nsteps + 2] StepMode | flags
  const int32_t* block_step;  // [nblocks + 1] first step of each CTA
  const int32_t* block_row;   // [nblocks + 1] first row of each CTA (vector phases)
  int32_t n;
  int32_t nsteps;
  int32_t nblocks;            // CTAs the partition was balanced for
  int32_t max_rows;           // most rows in one CTA's range (host side; 0 if unknown)
  int64_t nnz;
};

// Whether a solve of A in one launch (chunk_iters <= 0) runs the small-share
// kernel: every CTA's range fits kLocalRows.
inline bool small_share(const DevCsr& A, int64_t chunk_iters) {
  return A.max_rows > 0 && A.max_rows <= kLocalRows && chunk_iters <= 0;
}

// Control block of one solve, in device memory, cleared before its first
// launch.  A solve may run over several launches (batched solves advance
// each system a bounded number of steps per launch): the fields below
// `phase` carry its state from one launch to the next.
enum SolvePhase : int32_t { kPhaseNew = 0, kPhaseRunning = 1, kPhaseDone = 2 };
struct SolveCtrl {
  unsigned long long barrier;   // monotonic arrival counter of the group barrier
  int32_t abort;                // set by any CTA that gives up (timeout)
  int32_t status;               // CG_* code
  int64_t iters;                // steps done
  double rho;                   // r.z of the current iterate (r.r without preconditioner)
  double bnorm2;                // b.b
  double relres_rec;            // ||r||/||b|| of the recursive residual
  double relres_true;           // ||b - A x|| / ||b||
  int32_t timeout_site;         // which wait gave up (diagnostics)
  int32_t phase;                // SolvePhase
  unsigned long long rounds;    // group-barrier rounds completed so far
  int32_t slot;                 // partial-sum slot the next group sum uses
  int32_t pad;
};

struct SolveParams {
  DevCsr A;
  const double* b;
  double* x;
  double* r;
  double* p;
  double* q;
  float* p32;                   // FP32 shadow of p (mixed precision) or nullptr
  double* partials;             // [2][nblocks][2] per-CTA partial sums, two slots
  SolveCtrl* ctrl;
  double tol;
  int64_t maxit;
  int64_t replace_every;        // mixed precision: true-residual period
  unsigned long long wait_limit_ns;  // bound on every device-side wait
  int32_t group;                // CTAs that solve this system together (its partition's CTA count)
  int32_t stream_rows;          // single-system kernels: row pointers evict-first (stream_row_ptrs)
  int64_t chunk_iters;          // steps per launch (<= 0: until the solve ends)
  const double* dinv;           // Jacobi preconditioner 1/diag(A), or nullptr (plain CG)
  // Single-system solves: one epoch flag per CTA (zeroed before the launch).
  // In the large-share kernel a CTA publishes the step number in its flag
  // after its p update and waits only for the CTAs whose rows its own rows'
  // columns reach, instead of a barrier of the whole group.  nullptr (and
  // the other kernels): the group barrier.
  unsigned long long* flags;
};

// Batched solves: one persistent launch over many systems.  Every CTA takes
// tasks from a queue; a task is one CTA's share (rank) of one system.
struct BatchTask {
  int32_t sys;                  // index into the system table
  int32_t rank;                 // 0 .. group-1
};
struct BatchQueue {
  int32_t ntasks;
  int32_t stream_rows;          // row pointers evict-first in this launch (stream_row_ptrs)
  BatchTask task[1];            // ntasks entries (allocated to capacity)
};
struct BatchParams {
  const SolveParams* sys;       // system table (one entry per slot)
  const BatchQueue* queue;      // tasks of this launch, longest time per CTA first
  int32_t* next;                // next task to take (zeroed before each launch)
};

// Bytes that a step of the CG iteration on n rows reads again in the next
// step: p, q and r, the row pointers, the FP32 copy of p (mixed precision)
// and 1/diag(A) (Jacobi).  x and the matrix stream through with the
// evict-first policy.
inline int64_t step_reused_bytes(int64_t n, bool mixed, bool jacobi) {
  return n * (28 + (mixed ? 4 : 0) + (jacobi ? 8 : 0));
}

// Whether the product loads the row pointers with the evict-first policy:
// when the bytes that the running steps read again take more than 4/7 of
// the L2.  Below that, row pointers and vectors both stay in the L2 from
// step to step; above it the row pointers, read once per product, are the
// better ones to give up.  On GB300 with the Q1 systems: 128^3 was 5.7 %
// (mixed 3.5 %) and 136^3 0.5 % slower with them streamed; 136^3 mixed,
// 144^3 and larger 0.3 to 1.8 % faster, and a batch of 256 systems of 8^3
// to 48^3 4.5 % (mixed 8.9 %).
inline bool stream_row_ptrs(int64_t reused_bytes, int64_t l2_bytes) {
  return l2_bytes > 0 && 7 * reused_bytes > 4 * l2_bytes;
}

// Status codes (same values as include/cg.h).
enum : int32_t {
  kOK = 0, kEINVAL = 1, kENOMEM = 2, kECUDA = 3, kENOTCONV = 4,
  kEBREAKDOWN = 5, kETIMEOUT = 6, kEBUSY = 7,
};

// Launchers (defined in the .cu files; return the CUDA error of the launch).
// dinv[i] = 1 / (sum of row i's stored entries in column i); err set to the
// first row (+1) whose diagonal is not positive.
cudaError_t launch_jacobi_dinv(const int32_t* row_ptr, const int32_t* col_idx, const double* val, int64_t n,
                               double* dinv, int32_t* err, cudaStream_t s);
cudaError_t launch_spmv(const DevCsr& A, const double* x, double* y, int32_t* err, cudaStream_t s);
cudaError_t launch_dot(int64_t n, const double* x, const double* y, double* out,
                       double* partials, unsigned int* counter, int grid, cudaStream_t s);
cudaError_t launch_axpy(int64_t n, double a, const double* x, double* y, cudaStream_t s);
cudaError_t launch_ewmul(int64_t n, const double* x, const double* y, double* z, cudaStream_t s);
cudaError_t launch_solve(const SolveParams& P, bool mixed, cudaStream_t s);
int solve_blocks_per_sm(bool mixed, bool jacobi);   // occupancy of the persistent kernel
// The batched solve (cooperative launch of `nblocks` CTAs, one per SM).
cudaError_t launch_batch(const BatchParams& B, bool mixed, bool jacobi, int nblocks, cudaStream_t s);
int batch_blocks_per_sm(bool mixed, bool jacobi);
int dot_grid(int64_t n, int num_sms);
// Streamed dot product (x and y 16-byte aligned, n >= dot_stream_min_n()):
// `grid` = dot_stream_grid(n, SMs) CTAs; err[0] is raised by a wait that gave
// up, and the last CTA moves it to err[1] (the result is then NaN) and clears
// it.
cudaError_t launch_dot_stream(int64_t n, const double* x, const double* y, double* out, double* partials,
                              unsigned int* counter, int32_t* err, int grid, unsigned long long limit_ns,
                              cudaStream_t s);
int dot_stream_grid(int64_t n, int num_sms);
int64_t dot_stream_min_n();
// FP64 FMA throughput probe: `grid` CTAs of 256 threads, each thread 8
// independent chains of 4 x iters FMAs.
constexpr int kFp64ProbeThreads = 256;
constexpr int kFp64ProbeFmasPerIter = 32;
cudaError_t launch_fp64_probe(int64_t iters, int grid, double* sink, cudaStream_t s);
cudaError_t launch_wait_timeout_selftest(SolveCtrl* ctrl, unsigned long long limit_ns, cudaStream_t s);

// Small systems on one thread-block cluster (cluster_solve.cu): kClusterCtas
// CTAs of kClusterThreads threads, each holding R consecutive rows (R a power
// of two, at most kClusterMaxRows) and up to E entries in shared memory.
constexpr int kClusterCtas = 16;  // a non-portable cluster size (opted in)
constexpr int kClusterThreads = 512;
constexpr int kClusterMaxRows = 1024;
size_t cluster_smem_bytes(int R, int E);
// Clusters of this layout that can be resident at once (0: none, or an error).
int cluster_max_active(int R, int E);
cudaError_t launch_cluster_solve(const int32_t* row_ptr, const int32_t* col_idx, const double* val,
                                 const double* b, double* x, SolveCtrl* ctrl, double tol, int64_t maxit, int32_t n,
                                 int32_t R, int32_t E, cudaStream_t s);
// timeout_site the self-test's wait records
constexpr int32_t kSelftestSite = 99;
// timeout_site of a single-system solve's wait for its neighbours' p
constexpr int32_t kNeighborSite = 98;
// timeout_site of the synchronisation probe's barrier
constexpr int32_t kProbeSite = 97;
// The solves' group-wide synchronisations timed alone (cg_probe_group_sync):
// a cooperative launch of `nblocks` CTAs (one per SM) running `iters` group
// barriers (mode 0) or group sums (mode 1); ctrl zeroed before the launch,
// partials 2 * nblocks doubles, out nblocks doubles.
cudaError_t launch_sync_probe(SolveCtrl* ctrl, double* partials, int iters, int mode, int nblocks,
                              unsigned long long limit_ns, double* out, cudaStream_t s);
// Shared-memory bytes of a persistent solve CTA (FP32 ring values if mixed;
// `local`: the small-share kernels, with r of the share).
size_t solve_smem_bytes(bool mixed, bool local = false);
// Opt a kernel in to `bytes` of dynamic shared memory with the smallest
// carveout that holds them (once per kernel and device).
cudaError_t ensure_smem_attr(const void* kernel, size_t bytes);

}  // namespace cgk
