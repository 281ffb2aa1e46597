// Host side of the C ABI declared in include/cg.h: argument checks, CSR
// validation and upload, the row partition of the persistent kernels, device
// memory ownership, and the launch + read-back of each call.
#include <cmath>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <utility>
#include <vector>

#include "../../include/cg.h"
#include "cg_internal.h"
#include "host_util.h"

using cgh::Partition;
using cgh::build_partition;

namespace cgk {
cudaError_t launch_f64_to_f32(int64_t n, const double* src, float* dst, cudaStream_t s);
cudaError_t launch_dot_noalloc(int64_t n, const double* x, const double* y, double* out, cudaStream_t s);
int64_t dot_noalloc_max_n();
}

namespace cgh {

// Row partition of the persistent kernels.  Rows are split into `nblocks`
// contiguous CTA ranges of about equal cost (stored entries + kRowCost per
// row, the per-row vector work), and each CTA range into steps (see
// cg_internal.h): up to 32 rows of <= 32 entries (one lane per row), up to 16
// rows of <= 64 entries (two lanes per row), never more than kStepNnz entries,
// or one longer row.  Two sentinel steps follow the last one (the kernels
// read descriptors ahead).
constexpr int64_t kRowCost = 6;

int64_t cost_split(const std::vector<int32_t>& rp, int64_t lo_row, int64_t hi_row, int64_t part, int64_t parts) {
  // first row i in [lo_row, hi_row] with cost(lo_row, i) >= cost(lo_row, hi_row) * part / parts
  const int64_t c0 = static_cast<int64_t>(rp[lo_row]) + kRowCost * lo_row;
  const int64_t c1 = static_cast<int64_t>(rp[hi_row]) + kRowCost * hi_row;
  const int64_t goal = c0 + ((c1 - c0) * part) / parts;
  int64_t lo = lo_row, hi = hi_row;
  while (lo < hi) {
    const int64_t mid = (lo + hi) / 2;
    if (static_cast<int64_t>(rp[mid]) + kRowCost * mid >= goal) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

StepShape::StepShape() {
  for (int L = 0; L <= kShapeMaxLen; ++L)
    mode[L] = static_cast<int8_t>(L <= cgk::kLaneMax ? cgk::kLanePerRow : cgk::kPairPerRow);
}

bool StepShape::valid() const {
  for (int L = 0; L <= kShapeMaxLen; ++L) {
    const int m = mode[L];
    if (m != cgk::kLanePerRow && m != cgk::kPairPerRow && m != cgk::kLongRow) return false;
    if (m == cgk::kLanePerRow && L > cgk::kLaneMax) return false;
  }
  return true;
}

void warp_steps(const std::vector<int32_t>& rp, int64_t row, int64_t end, const StepShape& shape, Partition& P) {
  auto kind = [&](int64_t len) -> int { return len > kShapeMaxLen ? cgk::kLongRow : shape.mode[len]; };
  while (row < end) {
    const int64_t len0 = rp[row + 1] - rp[row];
    if (kind(len0) == cgk::kLongRow) {  // a warp per row: one step, walked piece by piece
      P.step.push_back(make_int4(static_cast<int>(row), static_cast<int>(row + 1), rp[row], rp[row + 1]));
      P.step_mode.push_back(cgk::kLongRow);
      ++row;
      continue;
    }
    const int64_t start = row;
    int64_t cnt = 0, maxlen = 0;
    int m = cgk::kLanePerRow;  // the widest kind so far (one lane < two lanes)
    while (row < end) {
      const int64_t len = rp[row + 1] - rp[row];
      const int k = kind(len);
      if (k == cgk::kLongRow || cnt + len > cgk::kStepNnz) break;
      const int nm = std::max(m, k);
      const int64_t cap = nm == cgk::kLanePerRow ? 32 : 16;
      if (row - start + 1 > cap) break;
      cnt += len;
      maxlen = std::max(maxlen, len);
      m = nm;
      ++row;
    }
    P.step.push_back(make_int4(static_cast<int>(start), static_cast<int>(row), rp[start], rp[row]));
    const int64_t wmax = m == cgk::kLanePerRow ? maxlen : (maxlen + 1) / 2;  // longest segment of one lane
    P.step_mode.push_back(m | static_cast<int32_t>(wmax << cgk::kWmaxShift));
  }
}

void build_partition(const std::vector<int32_t>& rp, int64_t n, int nblocks, Partition& P, const StepShape& shape) {
  P.step.clear();
  P.step_mode.clear();
  P.block_step.assign(static_cast<size_t>(nblocks) + 1, 0);
  P.block_row.assign(static_cast<size_t>(nblocks) + 1, 0);
  for (int b = 0; b <= nblocks; ++b) P.block_row[b] = static_cast<int32_t>(cost_split(rp, 0, n, b, nblocks));
  P.block_row[nblocks] = static_cast<int32_t>(n);
  for (int b = 0; b < nblocks; ++b) {
    P.block_step[b] = static_cast<int32_t>(P.step.size());
    warp_steps(rp, P.block_row[b], P.block_row[b + 1], shape, P);
  }
  P.block_step[nblocks] = static_cast<int32_t>(P.step.size());
  for (int t = 0; t < 2; ++t) {  // sentinels
    P.step.push_back(make_int4(static_cast<int>(n), static_cast<int>(n), rp[n], rp[n]));
    P.step_mode.push_back(cgk::kLanePerRow);
  }
}

}  // namespace cgh

struct cg_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int precision = CG_PREC_FP64;
  int preconditioner = CG_PRECOND_NONE;
  int replace_every = 50;
  unsigned long long wait_limit_ns = 2000000000ull;
  int64_t n = 0, nnz = 0;
  int num_sms = 0;
  int nblocks = 0;
  int nsteps = 0;
  int max_rows = 0;  // most rows in one CTA's range
  int cluster_R = 0;  // > 0: cg_solve runs the cluster kernel, R rows and E entries per CTA
  int cluster_E = 0;
  // device memory owned by the handle
  int32_t* d_row_ptr = nullptr;
  int32_t* d_col = nullptr;
  double* d_val = nullptr;
  float* d_val32 = nullptr;
  int4* d_step = nullptr;
  int32_t* d_step_mode = nullptr;
  int32_t* d_block_step = nullptr;
  int32_t* d_block_row = nullptr;
  double* d_r = nullptr;
  double* d_p = nullptr;
  double* d_q = nullptr;
  float* d_p32 = nullptr;
  double* d_dinv = nullptr;   // Jacobi: 1 / diag(A)
  double* d_xbuf = nullptr;   // staging of host x
  double* d_bbuf = nullptr;   // staging of host b
  double* d_partials = nullptr;
  cgk::SolveCtrl* d_ctrl = nullptr;  // followed by the CTAs' epoch flags (one allocation, one memset per solve)
  unsigned long long* d_flags = nullptr;
  int32_t* d_err = nullptr;
  cgk::SolveCtrl* h_ctrl = nullptr;  // pinned
  std::vector<void*> allocs;
  std::string err;
};

namespace {

thread_local std::string g_create_err;

int fail(cg_ctx* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  else g_create_err = msg;
  return code;
}

int cuda_fail(cg_ctx* h, cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  return fail(h, e == cudaErrorMemoryAllocation ? CG_ENOMEM : CG_ECUDA, m);
}

// The control block of a solve followed by one epoch flag per CTA.
constexpr size_t ctrl_flags_offset() { return (sizeof(cgk::SolveCtrl) + 15) & ~size_t(15); }
size_t ctrl_block_bytes(int nblocks) {
  return ctrl_flags_offset() + sizeof(unsigned long long) * static_cast<size_t>(nblocks > 0 ? nblocks : 1);
}

template <typename T>
cudaError_t dalloc(cg_ctx* h, T** p, size_t count) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, count ? count * sizeof(T) : 16);
  if (e == cudaSuccess) {
    h->allocs.push_back(q);
    *p = static_cast<T*>(q);
  }
  return e;
}

void release(cg_ctx* h) {
  if (!h) return;
  int cur = -1;
  cudaGetDevice(&cur);
  cudaSetDevice(h->device);
  for (void* p : h->allocs) cudaFree(p);
  h->allocs.clear();
  if (h->h_ctrl) cudaFreeHost(h->h_ctrl);
  h->h_ctrl = nullptr;
  if (cur >= 0) cudaSetDevice(cur);
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();  // clear the sticky-free error of an unknown pointer
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

cgk::DevCsr dev_view(const cg_ctx* h) {
  cgk::DevCsr A;
  A.row_ptr = h->d_row_ptr;
  A.col_idx = h->d_col;
  A.val = h->d_val;
  A.val32 = h->d_val32;
  A.step = h->d_step;
  A.step_mode = h->d_step_mode;
  A.block_step = h->d_block_step;
  A.block_row = h->d_block_row;
  A.n = static_cast<int32_t>(h->n);
  A.nsteps = h->nsteps;
  A.nblocks = h->nblocks;
  A.max_rows = h->max_rows;
  A.nnz = h->nnz;
  return A;
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

}  // namespace

// ---- BLAS-1 without a handle (Sec. 5.2): scratch per (device, stream)

namespace {

// Scratch of the dot product for one (device, stream) pair, allocated by the
// first call on that pair: kBlasPartials CTA sums, then the arrival counter
// and the two error words, then the device scalar of cg_dot_host.  Calls on
// one stream run one after another, so they can share it; calls on
// different streams use different scratch.
constexpr int kBlasPartials = 1024;
constexpr size_t kBlasScratchBytes = sizeof(double) * (kBlasPartials + 4);
struct BlasScratch {
  double* partials;
  unsigned int* counter;
  int32_t* err;  // [0] raised by the kernel, [1] outcome of the last call
  double* result;
};
// Key: (device, stream, host thread).  The thread is part of the key only for
// cudaStreamPerThread, whose one handle value names a different stream in
// every host thread.
std::mutex g_blas_mu;
std::map<std::tuple<int, uintptr_t, size_t>, double*> g_blas;

int sm_count(int dev) {
  static std::mutex mu;
  static int cache[64] = {0};
  if (dev < 0 || dev >= 64) return 0;
  std::lock_guard<std::mutex> lock(mu);
  if (!cache[dev] && cudaDeviceGetAttribute(&cache[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    cache[dev] = 0;
  }
  return cache[dev];
}

int64_t l2_bytes(int dev) {
  static std::mutex mu;
  static int cache[64] = {0};
  if (dev < 0 || dev >= 64) return 0;
  std::lock_guard<std::mutex> lock(mu);
  if (!cache[dev] && cudaDeviceGetAttribute(&cache[dev], cudaDevAttrL2CacheSize, dev) != cudaSuccess) {
    cudaGetLastError();
    cache[dev] = 0;
  }
  return cache[dev];
}

cudaError_t blas_scratch(cudaStream_t s, int* dev_out, BlasScratch* out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_blas_mu);
  const size_t thread_part = s == cudaStreamPerThread ? std::hash<std::thread::id>{}(std::this_thread::get_id()) : 0;
  auto key = std::make_tuple(dev, reinterpret_cast<uintptr_t>(s), thread_part);
  auto it = g_blas.find(key);
  double* base = nullptr;
  if (it == g_blas.end()) {
    e = cudaMalloc(&base, kBlasScratchBytes);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(base, 0, kBlasScratchBytes, s);
    if (e != cudaSuccess) {
      cudaFree(base);
      return e;
    }
    g_blas.emplace(key, base);
  } else {
    base = it->second;
  }
  out->partials = base;
  out->counter = reinterpret_cast<unsigned int*>(base + kBlasPartials);
  out->err = reinterpret_cast<int32_t*>(base + kBlasPartials + 1);
  out->result = base + kBlasPartials + 2;
  *dev_out = dev;
  return cudaSuccess;
}

inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// The dot product into `result` (device; NULL: the scratch's scalar);
// *streamed tells which kernel ran.
int dot_launch(const char* who, int64_t n, const double* x, const double* y, double* result, cudaStream_t s,
               BlasScratch* sc, bool* streamed) {
  int dev = 0;
  cudaError_t e = blas_scratch(s, &dev, sc);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, (std::string(who) + ": scratch").c_str());
  const int sms = sm_count(dev);
  if (sms <= 0 || 4 * sms > kBlasPartials)
    return fail(nullptr, CG_ECUDA, std::string(who) + ": unsupported SM count");
  if (!result) result = sc->result;
  *streamed = n >= cgk::dot_stream_min_n() && aligned16(x) && aligned16(y);
  if (*streamed)
    e = cgk::launch_dot_stream(n, x, y, result, sc->partials, sc->counter, sc->err, cgk::dot_stream_grid(n, sms),
                               2000000000ull, s);
  else
    e = cgk::launch_dot(n, x, y, result, sc->partials, sc->counter, cgk::dot_grid(n, sms), s);
  return e == cudaSuccess ? CG_OK : cuda_fail(nullptr, e, (std::string(who) + ": launch").c_str());
}

}  // namespace

extern "C" {

void cg_opts_default(cg_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->stream = nullptr;
  o->device = -1;
  o->precision = CG_PREC_FP64;
  o->replace_every = 50;
  o->validate = 1;
  o->wait_limit_ms = 2000;
  o->preconditioner = CG_PRECOND_NONE;
  o->ctas = 0;
}

const char* cg_last_error(cg_handle h) { return h ? h->err.c_str() : g_create_err.c_str(); }

int cg_create(cg_handle* out, const cg_csr* csr, int64_t n, int64_t nnz, const cg_opts* opts) {
  if (!out) return fail(nullptr, CG_EINVAL, "cg_create: out is NULL");
  *out = nullptr;
  if (!csr) return fail(nullptr, CG_EINVAL, "cg_create: csr is NULL");
  cg_opts o;
  cg_opts_default(&o);
  if (opts) o = *opts;
  const int base = csr->index_base;
  if (base != 0 && base != 1) return fail(nullptr, CG_EINVAL, "cg_create: index_base must be 0 or 1");
  const int64_t kMaxIdx = 2147483647LL - 16;
  if (n < 0 || nnz < 0 || n > kMaxIdx || nnz > kMaxIdx)
    return fail(nullptr, CG_EINVAL, "cg_create: n and nnz must be in [0, 2^31 - 16)");
  if (o.precision != CG_PREC_FP64 && o.precision != CG_PREC_MIXED)
    return fail(nullptr, CG_EINVAL, "cg_create: unknown precision");
  if (o.replace_every < 0) return fail(nullptr, CG_EINVAL, "cg_create: replace_every must be >= 0");
  if (o.preconditioner != CG_PRECOND_NONE && o.preconditioner != CG_PRECOND_JACOBI)
    return fail(nullptr, CG_EINVAL, "cg_create: unknown preconditioner");
  if (o.ctas < 0) return fail(nullptr, CG_EINVAL, "cg_create: ctas must be >= 0");
  if (!csr->row_ptr || (nnz > 0 && (!csr->col_idx || !csr->val)))
    return fail(nullptr, CG_EINVAL, "cg_create: NULL CSR array");

  // Host copies of row_ptr and col_idx (needed for validation and partitioning).
  std::vector<int32_t> rp(static_cast<size_t>(n) + 1), ci;
  const bool need_cols_on_host = o.validate || base != 0 || !csr->on_device;
  if (!csr->on_device) {
    std::memcpy(rp.data(), csr->row_ptr, sizeof(int32_t) * (n + 1));
    ci.assign(csr->col_idx, csr->col_idx + nnz);
  }

  // Host inputs are validated before any CUDA call (see the block below).
  auto validate_csr = [&](std::string& bad) {
    bad.clear();
    if (rp[0] != base) bad = "row_ptr[0] != index_base";
    for (int64_t i = 0; bad.empty() && i < n; ++i)
      if (rp[i + 1] < rp[i]) bad = "row_ptr decreases at row " + std::to_string(i);
    if (bad.empty() && static_cast<int64_t>(rp[n]) - base != nnz) bad = "row_ptr[n] != nnz + index_base";
    for (int64_t k = 0; bad.empty() && k < nnz; ++k)
      if (ci[k] < base || static_cast<int64_t>(ci[k]) - base >= n)
        bad = "column index out of range at entry " + std::to_string(k);
    return bad.empty();
  };
  if (!csr->on_device && o.validate) {
    std::string bad;
    if (!validate_csr(bad)) return fail(nullptr, CG_EINVAL, "cg_create: invalid CSR: " + bad);
  }

  cg_ctx* h = new (std::nothrow) cg_ctx();
  if (!h) return fail(nullptr, CG_ENOMEM, "cg_create: host allocation failed");
  if (o.device >= 0) h->device = o.device;
  else if (cudaGetDevice(&h->device) != cudaSuccess) h->device = 0;
  DeviceGuard guard(h->device);
  h->stream = static_cast<cudaStream_t>(o.stream);
  h->precision = o.precision;
  h->preconditioner = o.preconditioner;
  h->replace_every = o.replace_every;
  h->wait_limit_ns = static_cast<unsigned long long>(o.wait_limit_ms > 0 ? o.wait_limit_ms : 2000) * 1000000ull;
  h->n = n;
  h->nnz = nnz;
  cudaError_t e;
#define CG_TRY(call, what)                       \
  do {                                           \
    e = (call);                                  \
    if (e != cudaSuccess) {                      \
      int rc__ = cuda_fail(nullptr, e, what);    \
      release(h);                                \
      delete h;                                  \
      return rc__;                               \
    }                                            \
  } while (0)

  if (csr->on_device) {
    CG_TRY(cudaMemcpy(rp.data(), csr->row_ptr, sizeof(int32_t) * (n + 1), cudaMemcpyDeviceToHost),
           "cg_create: copy of row_ptr");
    if (need_cols_on_host && nnz > 0) {
      ci.resize(static_cast<size_t>(nnz));
      CG_TRY(cudaMemcpy(ci.data(), csr->col_idx, sizeof(int32_t) * nnz, cudaMemcpyDeviceToHost),
             "cg_create: copy of col_idx");
    }
  }
  // Validation of the CSR structure (Sec. 2.3 definition) for device inputs.
  if (csr->on_device && o.validate) {
    std::string bad;
    if (!validate_csr(bad)) {
      delete h;
      return fail(nullptr, CG_EINVAL, "cg_create: invalid CSR: " + bad);
    }
  }
  if (base) {
    for (auto& v : rp) v -= 1;
    for (auto& v : ci) v -= 1;
  }

  int sms = 0;
  CG_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device), "cg_create: SM count");
  h->num_sms = sms;
  const int per_sm = cgk::solve_blocks_per_sm(o.precision == CG_PREC_MIXED, o.preconditioner == CG_PRECOND_JACOBI);
  if (per_sm <= 0) {
    int rc = fail(nullptr, CG_ECUDA, "cg_create: the solve kernel cannot be resident (occupancy 0)");
    release(h);
    delete h;
    return rc;
  }
  h->nblocks = sms * per_sm;
  // every SM unless the caller asks for fewer: measured on GB300, fewer CTAs
  // do not shorten the solve of small systems (a 16^3 7-point system takes
  // 0.90 ms on 152 CTAs, 0.93 ms on 16 and 1.85 ms on one)
  if (o.ctas > 0) h->nblocks = std::min(h->nblocks, o.ctas);
  if (h->nblocks > 1024) {  // the group-wide fixed-point sum takes at most 1024 CTA values
    int rc = fail(nullptr, CG_ECUDA, "cg_create: more persistent CTAs than the grid-wide sum supports");
    release(h);
    delete h;
    return rc;
  }

  Partition part;
  build_partition(rp, n, h->nblocks, part);
  h->nsteps = static_cast<int>(part.step.size()) - 2;
  for (int b = 0; b < h->nblocks; ++b)
    h->max_rows = std::max(h->max_rows, part.block_row[b + 1] - part.block_row[b]);
  // Small plain FP64 systems (the CTA count left automatic): one cluster of
  // CTAs holding the system in shared memory, if its layout fits and such a
  // cluster can be resident.
  if (h->precision == CG_PREC_FP64 && h->preconditioner == CG_PRECOND_NONE && o.ctas <= 0 && n > 0 &&
      n <= static_cast<int64_t>(cgk::kClusterCtas) * cgk::kClusterMaxRows) {
    int R = 1;  // rows per CTA: a power of two, so the owner of a column is a shift
    while (static_cast<int64_t>(R) * cgk::kClusterCtas < n) R <<= 1;
    int E = 0;
    for (int c = 0; c < cgk::kClusterCtas; ++c) {
      const int64_t r0 = std::min<int64_t>(static_cast<int64_t>(c) * R, n);
      const int64_t r1 = std::min<int64_t>(r0 + R, n);
      E = std::max(E, rp[r1] - rp[r0]);
    }
    E = std::max(E, 1);
    if (cgk::cluster_max_active(R, E) > 0) {  // 0 if the layout is too large or no cluster fits
      h->cluster_R = R;
      h->cluster_E = E;
    }
  }

  const size_t pad = cgk::kPadEntries;
  CG_TRY(dalloc(h, &h->d_row_ptr, n + 1), "cg_create: cudaMalloc");
  CG_TRY(dalloc(h, &h->d_col, nnz + pad), "cg_create: cudaMalloc");
  CG_TRY(dalloc(h, &h->d_val, nnz + pad), "cg_create: cudaMalloc");
  CG_TRY(dalloc(h, &h->d_step, part.step.size()), "cg_create: cudaMalloc");
  CG_TRY(dalloc(h, &h->d_step_mode, part.step_mode.size()), "cg_create: cudaMalloc");
  CG_TRY(dalloc(h, &h->d_block_step, part.block_step.size()), "cg_create: cudaMalloc");
  CG_TRY(dalloc(h, &h->d_block_row, part.block_row.size()), "cg_create: cudaMalloc");
  CG_TRY(dalloc(h, &h->d_r, n), "cg_create: cudaMalloc");
  CG_TRY(dalloc(h, &h->d_p, n), "cg_create: cudaMalloc");
  CG_TRY(dalloc(h, &h->d_q, n), "cg_create: cudaMalloc");
  CG_TRY(dalloc(h, &h->d_xbuf, n), "cg_create: cudaMalloc");
  CG_TRY(dalloc(h, &h->d_bbuf, n), "cg_create: cudaMalloc");
  CG_TRY(dalloc(h, &h->d_partials, static_cast<size_t>(6) * h->nblocks), "cg_create: cudaMalloc");
  {
    unsigned char* blk = nullptr;
    CG_TRY(dalloc(h, &blk, ctrl_block_bytes(h->nblocks)), "cg_create: cudaMalloc");
    h->d_ctrl = reinterpret_cast<cgk::SolveCtrl*>(blk);
    h->d_flags = reinterpret_cast<unsigned long long*>(blk + ctrl_flags_offset());
  }
  CG_TRY(dalloc(h, &h->d_err, 4), "cg_create: cudaMalloc");
  if (o.precision == CG_PREC_MIXED) {
    CG_TRY(dalloc(h, &h->d_val32, nnz + pad), "cg_create: cudaMalloc");
    CG_TRY(dalloc(h, &h->d_p32, n), "cg_create: cudaMalloc");
  }
  if (o.preconditioner == CG_PRECOND_JACOBI) CG_TRY(dalloc(h, &h->d_dinv, n), "cg_create: cudaMalloc");
  CG_TRY(cudaMallocHost(&h->h_ctrl, sizeof(cgk::SolveCtrl)), "cg_create: cudaMallocHost");

  CG_TRY(cudaMemcpy(h->d_row_ptr, rp.data(), sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice), "cg_create: upload");
  CG_TRY(cudaMemset(h->d_col, 0, sizeof(int32_t) * (nnz + pad)), "cg_create: memset");
  CG_TRY(cudaMemset(h->d_val, 0, sizeof(double) * (nnz + pad)), "cg_create: memset");
  if (nnz > 0) {
    if (!ci.empty())
      CG_TRY(cudaMemcpy(h->d_col, ci.data(), sizeof(int32_t) * nnz, cudaMemcpyHostToDevice), "cg_create: upload");
    else
      CG_TRY(cudaMemcpy(h->d_col, csr->col_idx, sizeof(int32_t) * nnz, cudaMemcpyDeviceToDevice),
             "cg_create: upload");
    CG_TRY(cudaMemcpy(h->d_val, csr->val, sizeof(double) * nnz,
                      csr->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice),
           "cg_create: upload");
  }
  CG_TRY(cudaMemcpy(h->d_step, part.step.data(), sizeof(int4) * part.step.size(), cudaMemcpyHostToDevice),
         "cg_create: upload");
  CG_TRY(cudaMemcpy(h->d_step_mode, part.step_mode.data(), sizeof(int32_t) * part.step_mode.size(),
                    cudaMemcpyHostToDevice),
         "cg_create: upload");
  CG_TRY(cudaMemcpy(h->d_block_step, part.block_step.data(), sizeof(int32_t) * part.block_step.size(),
                    cudaMemcpyHostToDevice),
         "cg_create: upload");
  CG_TRY(cudaMemcpy(h->d_block_row, part.block_row.data(), sizeof(int32_t) * part.block_row.size(),
                    cudaMemcpyHostToDevice),
         "cg_create: upload");
  CG_TRY(cudaMemset(h->d_err, 0, 16), "cg_create: memset");
  if (o.precision == CG_PREC_MIXED) {
    CG_TRY(cudaMemset(h->d_val32, 0, sizeof(float) * (nnz + pad)), "cg_create: memset");
    if (nnz > 0) CG_TRY(cgk::launch_f64_to_f32(nnz, h->d_val, h->d_val32, nullptr), "cg_create: FP32 copy");
  }
  if (o.preconditioner == CG_PRECOND_JACOBI) {
    CG_TRY(cgk::launch_jacobi_dinv(h->d_row_ptr, h->d_col, h->d_val, n, h->d_dinv, h->d_err, nullptr),
           "cg_create: Jacobi diagonal");
    int32_t bad_row = 0;
    CG_TRY(cudaMemcpy(&bad_row, h->d_err, sizeof(int32_t), cudaMemcpyDeviceToHost), "cg_create: read-back");
    if (bad_row != 0) {
      release(h);
      delete h;
      return fail(nullptr, CG_EINVAL, "cg_create: Jacobi preconditioner: diagonal of row " +
                                          std::to_string(bad_row - 1) + " is not positive (A is not SPD)");
    }
    CG_TRY(cudaMemset(h->d_err, 0, 16), "cg_create: memset");
  }
  CG_TRY(cudaDeviceSynchronize(), "cg_create: synchronize");
#undef CG_TRY
  *out = h;
  return CG_OK;
}

int cg_destroy(cg_handle h) {
  if (!h) return CG_OK;
  release(h);
  delete h;
  return CG_OK;
}

int cg_info(cg_handle h, int64_t* n, int64_t* nnz, int32_t* nblocks) {
  if (!h) return fail(nullptr, CG_EINVAL, "cg_info: NULL handle");
  if (n) *n = h->n;
  if (nnz) *nnz = h->nnz;
  if (nblocks) *nblocks = h->nblocks;
  return CG_OK;
}

int cg_partition_info(cg_handle h, int32_t* max_rows, int32_t* kernel) {
  if (!h) return fail(nullptr, CG_EINVAL, "cg_partition_info: NULL handle");
  if (max_rows) *max_rows = h->cluster_R > 0 ? h->cluster_R : h->max_rows;
  if (kernel)
    *kernel = h->cluster_R > 0                      ? CG_SOLVE_KERNEL_CLUSTER
              : cgk::small_share(dev_view(h), 0) ? CG_SOLVE_KERNEL_SMALL_SHARE
                                                  : CG_SOLVE_KERNEL_LARGE_SHARE;
  return CG_OK;
}

int cg_spmv(cg_handle h, const double* x, double* y) {
  if (!h) return fail(nullptr, CG_EINVAL, "cg_spmv: NULL handle");
  if (h->n == 0) return CG_OK;
  if (!x || !y) return fail(h, CG_EINVAL, "cg_spmv: NULL vector");
  DeviceGuard g(h->device);
  cudaError_t e = cgk::launch_spmv(dev_view(h), x, y, h->d_err, h->stream);
  return e == cudaSuccess ? CG_OK : cuda_fail(h, e, "cg_spmv: launch");
}

int cg_dot(int64_t n, const double* x, const double* y, double* result, void* stream) {
  if (n < 0 || !result || (n > 0 && (!x || !y))) return fail(nullptr, CG_EINVAL, "cg_dot: bad arguments");
  BlasScratch sc;
  bool streamed = false;
  return dot_launch("cg_dot", n, x, y, result, static_cast<cudaStream_t>(stream), &sc, &streamed);
}

int cg_dot_host(int64_t n, const double* x, const double* y, double* result, void* stream) {
  if (n < 0 || !result || (n > 0 && (!x || !y))) return fail(nullptr, CG_EINVAL, "cg_dot_host: bad arguments");
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  BlasScratch sc;
  bool streamed = false;
  const int rc = dot_launch("cg_dot_host", n, x, y, nullptr, s, &sc, &streamed);
  if (rc != CG_OK) return rc;
  double v = 0.0;
  int32_t bad = 0;
  cudaError_t e = cudaMemcpyAsync(&v, sc.result, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && streamed) e = cudaMemcpyAsync(&bad, sc.err + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "cg_dot_host");
  if (bad) return fail(nullptr, CG_ETIMEOUT, "cg_dot_host: a device-side wait of the dot kernel gave up");
  *result = v;
  return CG_OK;
}

int cg_axpy(int64_t n, double a, const double* x, double* y, void* stream) {
  if (n < 0 || (n > 0 && (!x || !y))) return fail(nullptr, CG_EINVAL, "cg_axpy: bad arguments");
  if (n == 0) return CG_OK;
  cudaError_t e = cgk::launch_axpy(n, a, x, y, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? CG_OK : cuda_fail(nullptr, e, "cg_axpy: launch");
}

int cg_ewmul(int64_t n, const double* x, const double* y, double* z, void* stream) {
  if (n < 0 || (n > 0 && (!x || !y || !z))) return fail(nullptr, CG_EINVAL, "cg_ewmul: bad arguments");
  if (n == 0) return CG_OK;
  cudaError_t e = cgk::launch_ewmul(n, x, y, z, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? CG_OK : cuda_fail(nullptr, e, "cg_ewmul: launch");
}

int cg_probe_fp64_peak(int32_t device, double* gflops) {
  if (!gflops) return fail(nullptr, CG_EINVAL, "cg_probe_fp64_peak: NULL output");
  *gflops = 0.0;
  int dev = device;
  if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) return fail(nullptr, CG_ECUDA, "cg_probe_fp64_peak: no device");
  DeviceGuard g(dev);
  const int sms = sm_count(dev);
  if (sms <= 0) return fail(nullptr, CG_ECUDA, "cg_probe_fp64_peak: SM count");
  double* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc(&sink, sizeof(double) * static_cast<size_t>(sms) * 8);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  double best = 0.0;
  // two, four and eight CTAs of 256 threads per SM; for each, two launches
  // warm up and size the next three to about 40 ms, the best of which counts
  for (int per_sm = 2; e == cudaSuccess && per_sm <= 8; per_sm *= 2) {
    const int grid = sms * per_sm;
    const double per_iter = static_cast<double>(grid) * cgk::kFp64ProbeThreads * cgk::kFp64ProbeFmasPerIter;
    int64_t iters = 500;
    for (int rep = 0; e == cudaSuccess && rep < 5; ++rep) {
      e = cudaEventRecord(e0, nullptr);
      if (e == cudaSuccess) e = cgk::launch_fp64_probe(iters, grid, sink, nullptr);
      if (e == cudaSuccess) e = cudaEventRecord(e1, nullptr);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess || ms <= 0.f) break;
      if (rep >= 2) best = std::max(best, 2.0 * per_iter * static_cast<double>(iters) / (ms * 1e-3) / 1e9);
      if (rep == 1) iters = std::max<int64_t>(iters, static_cast<int64_t>(iters * (40.0 / ms)));
    }
  }
  if (e1) cudaEventDestroy(e1);
  if (e0) cudaEventDestroy(e0);
  if (sink) cudaFree(sink);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "cg_probe_fp64_peak");
  *gflops = best;
  return CG_OK;
}

int cg_probe_group_sync(int32_t device, int32_t iters, double* barrier_us, double* sum_us) {
  if (!barrier_us || !sum_us || iters < 1 || iters > 1000000)
    return fail(nullptr, CG_EINVAL, "cg_probe_group_sync: iters in [1, 10^6] and two outputs");
  *barrier_us = 0.0;
  *sum_us = 0.0;
  int dev = device;
  if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) return fail(nullptr, CG_ECUDA, "cg_probe_group_sync: no device");
  DeviceGuard g(dev);
  const int sms = sm_count(dev);
  if (sms <= 0) return fail(nullptr, CG_ECUDA, "cg_probe_group_sync: SM count");
  const int nb = sms * cgk::kCtasPerSm;
  char* buf = nullptr;
  cgk::SolveCtrl* ctrl = nullptr;
  double* partials = nullptr;
  double* out = nullptr;
  const size_t ctrl_bytes = (sizeof(cgk::SolveCtrl) + 255) & ~size_t(255);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc(&buf, ctrl_bytes + sizeof(double) * 3 * static_cast<size_t>(nb));
  if (e == cudaSuccess) {
    ctrl = reinterpret_cast<cgk::SolveCtrl*>(buf);
    partials = reinterpret_cast<double*>(buf + ctrl_bytes);
    out = partials + 2 * static_cast<size_t>(nb);
    e = cudaEventCreate(&e0);
  }
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  bool timed_out = false;
  double per_iter[2] = {0.0, 0.0};
  for (int mode = 0; e == cudaSuccess && mode < 2 && !timed_out; ++mode) {
    // a short launch first (clocks, first-touch), then the timed one
    for (int rep = 0; e == cudaSuccess && rep < 2; ++rep) {
      const int n_it = rep == 0 ? std::max(1, iters / 10) : iters;
      e = cudaMemset(ctrl, 0, sizeof(cgk::SolveCtrl));
      if (e == cudaSuccess) e = cudaEventRecord(e0, nullptr);
      if (e == cudaSuccess) e = cgk::launch_sync_probe(ctrl, partials, n_it, mode, nb, 2000000000ull, out, nullptr);
      if (e == cudaSuccess) e = cudaEventRecord(e1, nullptr);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      int32_t abort_flag = 0;
      if (e == cudaSuccess)
        e = cudaMemcpy(&abort_flag, &ctrl->abort, sizeof(int32_t), cudaMemcpyDeviceToHost);
      if (e == cudaSuccess && abort_flag) timed_out = true;
      if (e == cudaSuccess && rep == 1) per_iter[mode] = 1000.0 * static_cast<double>(ms) / n_it;
      if (timed_out) break;
    }
  }
  if (e1) cudaEventDestroy(e1);
  if (e0) cudaEventDestroy(e0);
  if (buf) cudaFree(buf);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "cg_probe_group_sync");
  if (timed_out) return fail(nullptr, CG_ETIMEOUT, "cg_probe_group_sync: a group barrier wait gave up");
  *barrier_us = per_iter[0];
  *sum_us = per_iter[1];
  return CG_OK;
}

int cg_blas_release(void) {
  std::lock_guard<std::mutex> lock(g_blas_mu);
  int cur = -1;
  cudaGetDevice(&cur);
  for (auto& kv : g_blas) {
    cudaSetDevice(std::get<0>(kv.first));
    cudaFree(kv.second);
  }
  g_blas.clear();
  if (cur >= 0) cudaSetDevice(cur);
  return CG_OK;
}

int cg_solve(cg_handle h, const double* b, double* x, double tol, int64_t maxit, int64_t* iters, double* relres) {
  if (!h) return fail(nullptr, CG_EINVAL, "cg_solve: NULL handle");
  if (!iters || !relres) return fail(h, CG_EINVAL, "cg_solve: NULL output");
  if (!(tol >= 0.0)) return fail(h, CG_EINVAL, "cg_solve: tol must be >= 0");
  if (maxit < 0) return fail(h, CG_EINVAL, "cg_solve: maxit must be >= 0");
  *iters = 0;
  *relres = 0.0;
  if (h->n == 0) return CG_OK;
  if (!b || !x) return fail(h, CG_EINVAL, "cg_solve: NULL vector");
  DeviceGuard g(h->device);
  const size_t bytes = sizeof(double) * static_cast<size_t>(h->n);
  const bool b_dev = is_device_ptr(b), x_dev = is_device_ptr(x);
  const double* db = b;
  double* dx = x;
  cudaError_t e;
  if (!b_dev) {
    e = cudaMemcpyAsync(h->d_bbuf, b, bytes, cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "cg_solve: copy of b");
    db = h->d_bbuf;
  }
  if (!x_dev) {
    e = cudaMemcpyAsync(h->d_xbuf, x, bytes, cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "cg_solve: copy of x");
    dx = h->d_xbuf;
  }
  e = cudaMemsetAsync(h->d_ctrl, 0, ctrl_block_bytes(h->nblocks), h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "cg_solve: memset");
  cgk::SolveParams P;
  P.A = dev_view(h);
  P.b = db;
  P.x = dx;
  P.r = h->d_r;
  P.p = h->d_p;
  P.q = h->d_q;
  P.p32 = h->d_p32;
  P.partials = h->d_partials;
  P.ctrl = h->d_ctrl;
  P.tol = tol;
  P.maxit = maxit;
  P.replace_every = h->replace_every;
  P.wait_limit_ns = h->wait_limit_ns;
  P.group = h->nblocks;
  P.stream_rows = cgk::stream_row_ptrs(
      cgk::step_reused_bytes(h->n, h->precision == CG_PREC_MIXED, h->d_dinv != nullptr), l2_bytes(h->device));
  P.chunk_iters = 0;
  P.dinv = h->d_dinv;
  P.flags = h->nblocks > 1 ? h->d_flags : nullptr;
  if (h->cluster_R > 0)
    e = cgk::launch_cluster_solve(h->d_row_ptr, h->d_col, h->d_val, db, dx, h->d_ctrl, tol, maxit,
                                  static_cast<int32_t>(h->n), h->cluster_R, h->cluster_E, h->stream);
  else
    e = cgk::launch_solve(P, h->precision == CG_PREC_MIXED, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "cg_solve: launch");
  e = cudaMemcpyAsync(h->h_ctrl, h->d_ctrl, sizeof(cgk::SolveCtrl), cudaMemcpyDeviceToHost, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "cg_solve: read-back");
  if (!x_dev) {
    e = cudaMemcpyAsync(x, h->d_xbuf, bytes, cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "cg_solve: copy of x");
  }
  e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "cg_solve: synchronize");
  *iters = h->h_ctrl->iters;
  *relres = h->h_ctrl->relres_true;
  const int st = h->h_ctrl->status;
  if (st == CG_ETIMEOUT)
    return fail(h, CG_ETIMEOUT, "cg_solve: a device-side wait gave up (site " +
                                    std::to_string(h->h_ctrl->timeout_site) + ")");
  if (st == CG_EBREAKDOWN) return fail(h, CG_EBREAKDOWN, "cg_solve: breakdown (p.Ap <= 0 or not finite)");
  if (st == CG_ENOTCONV) return fail(h, CG_ENOTCONV, "cg_solve: maxit reached before the tolerance");
  return st;
}

int cg_dot_noalloc(int64_t n, const double* x, const double* y, double* result, void* stream) {
  const int64_t max_n = cgk::dot_noalloc_max_n();
  if (n < 0 || !result || (n > 0 && (!x || !y))) return fail(nullptr, CG_EINVAL, "cg_dot_noalloc: bad arguments");
  if (n > max_n)
    return fail(nullptr, CG_EINVAL,
                "cg_dot_noalloc: n = " + std::to_string(n) + " exceeds the fixed scratch capacity of " +
                    std::to_string(max_n) + " elements; use cg_dot");
  cudaError_t e = cgk::launch_dot_noalloc(n, x, y, result, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? CG_OK : cuda_fail(nullptr, e, "cg_dot_noalloc");
}

int cg_selftest_wait_timeout(int32_t limit_ms, int32_t* kernel_status) {
  if (!kernel_status || limit_ms <= 0 || limit_ms > 10000)
    return fail(nullptr, CG_EINVAL, "cg_selftest_wait_timeout: limit_ms in (0, 10000] and a status pointer");
  cgk::SolveCtrl* d = nullptr;
  cudaError_t e = cudaMalloc(&d, sizeof(cgk::SolveCtrl));
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "cg_selftest_wait_timeout: cudaMalloc");
  cgk::SolveCtrl hc;
  e = cudaMemset(d, 0, sizeof(cgk::SolveCtrl));
  if (e == cudaSuccess)
    e = cgk::launch_wait_timeout_selftest(d, static_cast<unsigned long long>(limit_ms) * 1000000ull, nullptr);
  if (e == cudaSuccess) e = cudaMemcpy(&hc, d, sizeof(hc), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "cg_selftest_wait_timeout");
  *kernel_status = hc.status;
  if (hc.status == CG_ETIMEOUT && (hc.abort != 1 || hc.timeout_site != cgk::kSelftestSite))
    return fail(nullptr, CG_ECUDA, "cg_selftest_wait_timeout: the wait gave up without raising the abort flag");
  return CG_OK;
}

}  // extern "C"
