// Internal structures shared by the host side of the C-ABI and the kernels.
// Not part of the public interface (that is include/cg.h).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace cgk {

// The persistent kernels run two 256-thread CTAs per SM: two independent
// instruction streams whose memory-latency phases overlap each other's FP64
// phases.
constexpr int kBlock = 256;
constexpr int kCtasPerSm = 2;
constexpr int kWarps = kBlock / 32;

// Matrix stream of a CTA: its CSR values and column indices flow through a
// shared-memory ring of kSlots pieces of kPiece entries, each piece one pair
// of 1-D TMA bulk copies completing on the slot's mbarrier.
constexpr int kPieceLog = 11;
constexpr int kPiece = 1 << kPieceLog;  // 2048 entries
constexpr int kSlots = 4;
constexpr int kRing = kPiece * kSlots;  // 8192 entries: 64 KB of FP64 values + 32 KB of indices
constexpr int kRingMask = kRing - 1;
// A compute chunk is a run of consecutive rows computed together: at most
// kChunkNnz entries (half the ring, so the next pieces stream in meanwhile)
// and at most kBlock rows (one thread per row) or kBlock/2 rows (two threads
// per row).  A row longer than kChunkNnz is a chunk of its own, streamed from
// global memory by the whole CTA.
constexpr int kChunkNnz = kRing / 2;
// Padding (in entries) behind val/col allocations so that rounding a copy's
// end up to 16 bytes never reads past the allocation.
constexpr int kPadEntries = 8;

enum ChunkMode : int32_t {
  kThreadPerRow = 0,  // rows of <= 16 entries: thread t computes row r0 + t
  kPairPerRow = 1,    // rows of <= 64 entries: threads 2t, 2t+1 split row r0 + t
  kWarpPerRow = 2,    // longer rows: warp w computes rows r0 + w, r0 + w + 8, ...
  kBlockPerRow = 3,   // one row longer than kChunkNnz, streamed from global memory
};

// Device view of a CSR matrix with its chunk partition.
struct DevCsr {
  const int32_t* row_ptr;     // [n+1], 0-based
  const int32_t* col_idx;     // [nnz + kPadEntries]
  const double* val;          // [nnz + kPadEntries]
  const float* val32;         // [nnz + kPadEntries] FP32 copy (mixed precision) or nullptr
  const int32_t* chunk_row;   // [nchunks+1] first row of each chunk
  const int32_t* chunk_mode;  // [nchunks]
  const int32_t* block_chunk; // [nblocks+1] first chunk of each persistent CTA
  int32_t n;
  int32_t nchunks;
  int32_t nblocks;            // CTAs the chunk partition was balanced for
  int64_t nnz;
};

// Control block of one solve, in device memory, cleared before each launch.
struct SolveCtrl {
  unsigned long long barrier;   // monotonic arrival counter of the grid barrier
  int32_t abort;                // set by any CTA that gives up (timeout)
  int32_t status;               // CG_* code
  int64_t iters;
  double rho;                   // r.r of the last iterate (recursive residual)
  double bnorm2;                // b.b
  double relres_rec;            // sqrt(rho)/||b||
  double relres_true;           // ||b - A x|| / ||b||
  int32_t timeout_site;         // which wait gave up (diagnostics)
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
};

// Status codes (same values as include/cg.h).
enum : int32_t {
  kOK = 0, kEINVAL = 1, kENOMEM = 2, kECUDA = 3, kENOTCONV = 4,
  kEBREAKDOWN = 5, kETIMEOUT = 6, kEBUSY = 7,
};

// Launchers (defined in the .cu files; return the CUDA error of the launch).
cudaError_t launch_spmv(const DevCsr& A, const double* x, double* y, int32_t* err, cudaStream_t s);
cudaError_t launch_dot(int64_t n, const double* x, const double* y, double* out,
                       double* partials, unsigned int* counter, int grid, cudaStream_t s);
cudaError_t launch_axpy(int64_t n, double a, const double* x, double* y, cudaStream_t s);
cudaError_t launch_ewmul(int64_t n, const double* x, const double* y, double* z, cudaStream_t s);
cudaError_t launch_solve(const SolveParams& P, bool mixed, cudaStream_t s);
int solve_blocks_per_sm(bool mixed);   // occupancy of the persistent kernel
int dot_grid(int64_t n, int num_sms);
cudaError_t launch_wait_timeout_selftest(SolveCtrl* ctrl, unsigned long long limit_ns, cudaStream_t s);
// Shared-memory bytes of the streamed product (ring + scratch).
size_t spmv_smem_bytes();

}  // namespace cgk
