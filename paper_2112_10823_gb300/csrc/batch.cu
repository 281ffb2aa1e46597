// Host runtime of the batched and served solves (cg_batch_* in cg.h).
//
// A batch object holds one device allocation (the memory budget) managed by
// a first-fit arena, a table of resident systems (SolveParams + SolveCtrl per
// slot), and a worker thread.  The worker repeats rounds: it launches the
// persistent batch kernel over the resident systems, admits queued requests
// while that round runs (host preparation, copies on a second stream), then
// reads back every system's control block, copies out and releases finished
// systems.  A round is one CUDA graph replay: task queue upload, counter
// reset, the cooperative kernel, control-block read-back.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/cg.h"
#include "cg_internal.h"
#include "host_util.h"

namespace cgk {
cudaError_t launch_f64_to_f32(int64_t n, const double* src, float* dst, cudaStream_t s);
}

namespace {

thread_local std::string g_batch_create_err;
constexpr size_t kAlign = 256;

size_t align_up(size_t v) { return (v + kAlign - 1) & ~(kAlign - 1); }

// First-fit allocator over [0, cap) in kAlign granules; free blocks are
// coalesced with their neighbours on release.
class Arena {
 public:
  void init(size_t cap) {
    cap_ = cap & ~(kAlign - 1);
    free_.clear();
    if (cap_) free_[0] = cap_;
  }
  bool alloc(size_t bytes, size_t& off) {
    bytes = align_up(bytes ? bytes : 1);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      off = it->first;
      const size_t rest = it->second - bytes;
      free_.erase(it);
      if (rest) free_[off + bytes] = rest;
      in_use += bytes;
      peak = std::max(peak, in_use);
      return true;
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = align_up(bytes ? bytes : 1);
    in_use -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t cap() const { return cap_; }
  size_t in_use = 0, peak = 0;

 private:
  size_t cap_ = 0;
  std::map<size_t, size_t> free_;
};

// Cost model behind the automatic group size.  A system's solve on G CTAs
// is estimated as steps * (bytes_per_step / (G * rate_G) + overhead_G); the
// group is the smallest G whose estimate meets target_s, at most half the
// grid and at least 1024 rows per CTA (the largest such G when no G meets
// the target: with a 5 ms target, 100 requests/s of 16^3..96^3 systems were
// served with a p50 latency of 12.8 ms at 1024 rows per CTA, 13.3 ms at
// 2048 and 17.0 ms at 4096).  The step count of
// a 3-D finite-element system grows like n^(1/3) (CG's step count follows
// sqrt(condition number), which grows like h^-1).  The rates and overheads
// are built-in guesses unless measured on the GPU (calibrate() below).
struct GroupModel {
  double cta_rate = 40e9;        // bytes/s one CTA streams while every SM is busy (G = 1)
  double group_rate = 40e9;      // the same for a CTA inside a group (G > 1)
  double overhead_1 = 3e-6;      // s per step of a one-CTA group (CTA barriers, sums)
  double overhead_g = 8e-6;      // s per step of a multi-CTA group (group barriers)
  double steps_per_cbrt_n = 6.2; // estimated steps / n^(1/3)
  double target_s = 50e-3;       // solo solve time a group should meet
};

double est_steps(const GroupModel& m, int64_t n) { return m.steps_per_cbrt_n * std::cbrt(static_cast<double>(n)); }

double bytes_per_step(int64_t n, int64_t nnz, bool mixed) {
  return static_cast<double>(mixed ? 8 : 12) * static_cast<double>(nnz) + (mixed ? 100.0 : 92.0) * n;
}

int auto_group(const GroupModel& m, int64_t n, int64_t nnz, bool mixed, int nblocks) {
  const int gmax = std::max<int64_t>(1, std::min<int64_t>({static_cast<int64_t>(nblocks / 2),
                                                           static_cast<int64_t>(1024),
                                                           n / 1024}));
  const double steps = est_steps(m, n), bs = bytes_per_step(n, nnz, mixed);
  for (int g = 1; g <= gmax; ++g) {
    const double t = g == 1 ? steps * (bs / m.cta_rate + m.overhead_1)
                            : steps * (bs / (g * m.group_rate) + m.overhead_g);
    if (t <= m.target_s) return g;
  }
  return gmax;
}

double now_ms(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Upper bound of a system's device footprint (before its partition is known:
// at most one step per row).
size_t footprint_bound(int64_t n, int64_t nnz, bool mixed, bool jacobi, int nblocks) {
  const size_t pad = cgk::kPadEntries;
  size_t b = 0;
  b += align_up(4 * (n + 1));
  b += align_up(4 * (nnz + pad)) + align_up(8 * (nnz + pad));
  if (mixed) b += align_up(4 * (nnz + pad)) + align_up(4 * n);
  b += align_up(sizeof(int4) * (n + 2)) + align_up(4 * (n + 2));
  b += 2 * align_up(4 * (static_cast<size_t>(nblocks) + 1));
  b += (jacobi ? 6 : 5) * align_up(8 * n);
  b += align_up(sizeof(double) * 6 * nblocks);
  return b;
}

enum JobState { kQueued, kResident, kFinished };

struct Job {
  uint64_t ticket = 0;
  cg_request req{};
  cg_result res{};
  JobState state = kQueued;
  int slot = -1;
  size_t off = 0, bytes = 0;   // arena block
  int group = 1;
  double* d_x = nullptr;
  double bytes_step = 0.0;
  double steps_est = 0.0;
};

}  // namespace

// Pinned host memory for the small per-system arrays of an admission pass
// (row pointers, step partition, rebased columns), so that every upload is
// an asynchronous copy from pinned memory; chunks are kept and reused, and
// reset() starts a new pass once the previous pass's copies have completed.
struct PinnedPool {
  struct Chunk {
    char* p;
    size_t size, used;
  };
  std::vector<Chunk> chunks;
  ~PinnedPool() {
    for (auto& c : chunks) cudaFreeHost(c.p);
  }
  void reset() {
    for (auto& c : chunks) c.used = 0;
  }
  // bytes of pinned memory (16-byte aligned), or nullptr if none can be had
  void* take(size_t bytes) {
    bytes = (bytes + 15) & ~size_t(15);
    for (auto& c : chunks)
      if (c.size - c.used >= bytes) {
        void* q = c.p + c.used;
        c.used += bytes;
        return q;
      }
    const size_t size = std::max(bytes, size_t(8) << 20);
    char* q = nullptr;
    if (cudaMallocHost(&q, size) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    chunks.push_back({q, size, bytes});
    return q;
  }
};

struct cg_batch_ctx {
  int device = 0;
  bool mixed = false;
  bool jacobi = false;
  int max_systems = 1024;
  int chunk_iters = 0;
  int replace_every = 50;
  unsigned long long wait_ns = 2000000000ull;
  int max_pending = 65536;
  int group_override = 0;
  int calib_group = 0;        // group of the calibration requests (while calibrating)
  bool autotuned = false;
  cgh::StepShape shape;       // step kind per row length of every admitted system
  bool shape_tuned = false;
  bool shape_fixed = false;   // set by cg_batch_opts.step_shape (not tuned)
  bool validate = true;
  int nblocks = 0;
  int task_cap = 0;
  int64_t l2_bytes = 0;       // the device's L2 (row-pointer policy of a round)
  GroupModel model;
  std::chrono::steady_clock::time_point t0;

  cudaStream_t compute = nullptr, copy = nullptr;
  char* d_arena = nullptr;
  Arena arena;
  cgk::SolveParams* d_sys = nullptr;
  cgk::SolveCtrl* d_ctrl = nullptr;
  cgk::BatchQueue* d_queue = nullptr;
  int32_t* d_next = nullptr;
  int32_t* d_admit_err = nullptr;      // per slot, Jacobi: first row without a positive diagonal (+1)
  int32_t* h_admit_err = nullptr;      // pinned, per slot
  PinnedPool staging;                  // host arrays of the admission pass in flight
  cgk::SolveParams* h_sys = nullptr;   // pinned
  cgk::SolveCtrl* h_ctrl = nullptr;    // pinned
  cgk::BatchQueue* h_queue = nullptr;  // pinned
  size_t queue_bytes = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  bool use_graph = true;

  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::thread worker;
  bool stop = false;
  uint64_t next_ticket = 1;
  std::deque<uint64_t> queued;
  std::unordered_map<uint64_t, std::unique_ptr<Job>> jobs;
  std::vector<int> free_slots;
  std::vector<Job*> resident;
  int64_t rounds = 0, submitted = 0, admitted = 0, completed = 0;
  int64_t rounds_stream_rows = 0;  // rounds whose product loaded the row pointers evict-first
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;  // around each round, on the compute stream
  double round_ms_total = 0.0, last_round_ms = 0.0;
  std::string err;
};

namespace {

int bfail(cg_batch_ctx* b, int code, const std::string& msg) {
  if (b) {
    std::lock_guard<std::mutex> lk(b->mu);
    b->err = msg;
  } else {
    g_batch_create_err = msg;
  }
  return code;
}

std::string cuda_msg(cudaError_t e, const char* what) {
  return std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
}

// The launch sequence of one round, on b->compute (captured once into the
// graph when possible).
cudaError_t enqueue_round(cg_batch_ctx* b) {
  cudaError_t e = cudaMemcpyAsync(b->d_queue, b->h_queue, b->queue_bytes, cudaMemcpyHostToDevice, b->compute);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_next, 0, sizeof(int32_t), b->compute);
  if (e == cudaSuccess) {
    cgk::BatchParams P{b->d_sys, b->d_queue, b->d_next};
    e = cgk::launch_batch(P, b->mixed, b->jacobi, b->nblocks, b->compute);
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->h_ctrl, b->d_ctrl, sizeof(cgk::SolveCtrl) * b->max_systems, cudaMemcpyDeviceToHost,
                        b->compute);
  return e;
}

void try_capture(cg_batch_ctx* b) {
  if (!b->use_graph) return;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(b->compute, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaError_t e1 = enqueue_round(b);
    e = cudaStreamEndCapture(b->compute, &g);
    if (e1 != cudaSuccess) e = e1;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph_exec, g, 0);
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (g) cudaGraphDestroy(g);
    b->graph_exec = nullptr;
    b->use_graph = false;
    return;
  }
  b->graph = g;
}

// Host copies of a request's CSR structure (0-based) and its validation.
bool load_structure(const cg_request& r, bool validate, std::vector<int32_t>& rp, std::vector<int32_t>& ci,
                    std::string& bad) {
  const int64_t n = r.n, nnz = r.nnz;
  const int base = r.csr.index_base;
  rp.resize(static_cast<size_t>(n) + 1);
  ci.clear();
  if (r.csr.on_device) {
    if (cudaMemcpy(rp.data(), r.csr.row_ptr, 4 * (n + 1), cudaMemcpyDeviceToHost) != cudaSuccess) {
      cudaGetLastError();
      bad = "copy of row_ptr failed";
      return false;
    }
    if (validate && nnz > 0) {
      ci.resize(static_cast<size_t>(nnz));
      if (cudaMemcpy(ci.data(), r.csr.col_idx, 4 * nnz, cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        bad = "copy of col_idx failed";
        return false;
      }
    }
  } else {
    std::memcpy(rp.data(), r.csr.row_ptr, 4 * (n + 1));
    if (validate) ci.assign(r.csr.col_idx, r.csr.col_idx + nnz);
  }
  if (validate) {
    if (rp[0] != base) bad = "row_ptr[0] != index_base";
    for (int64_t i = 0; bad.empty() && i < n; ++i)
      if (rp[i + 1] < rp[i]) bad = "row_ptr decreases at row " + std::to_string(i);
    if (bad.empty() && static_cast<int64_t>(rp[n]) - base != nnz) bad = "row_ptr[n] != nnz + index_base";
    for (int64_t k = 0; bad.empty() && k < nnz; ++k)
      if (ci[k] < base || static_cast<int64_t>(ci[k]) - base >= n)
        bad = "column index out of range at entry " + std::to_string(k);
    if (!bad.empty()) return false;
  }
  if (base)
    for (auto& v : rp) v -= 1;
  return true;
}

// A job's device layout inside its arena block.
struct Layout {
  size_t rp, col, val, val32, step, mode, bstep, brow, b, x, r, p, q, p32, dinv, part, total;
};

Layout layout_of(int64_t n, int64_t nnz, size_t nsteps2, int group, bool mixed, bool jacobi) {
  const size_t pad = cgk::kPadEntries;
  Layout L{};
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o += align_up(bytes);
    return at;
  };
  L.rp = take(4 * (n + 1));
  L.col = take(4 * (nnz + pad));
  L.val = take(8 * (nnz + pad));
  L.val32 = mixed ? take(4 * (nnz + pad)) : 0;
  L.step = take(sizeof(int4) * nsteps2);
  L.mode = take(4 * nsteps2);
  L.bstep = take(4 * (static_cast<size_t>(group) + 1));
  L.brow = take(4 * (static_cast<size_t>(group) + 1));
  L.b = take(8 * n);
  L.x = take(8 * n);
  L.r = take(8 * n);
  L.p = take(8 * n);
  L.q = take(8 * n);
  L.p32 = mixed ? take(4 * n) : 0;
  L.dinv = jacobi ? take(8 * n) : 0;
  L.part = take(sizeof(double) * 6 * group);
  L.total = o;
  return L;
}

void finish_without_device(cg_batch_ctx* b, Job* j, int status) {
  j->res.done = 1;
  j->res.status = status;
  j->res.done_ms = now_ms(b->t0);
  j->state = kFinished;
  ++b->completed;
}

// Prepare and upload the queue head while memory and slots allow.  Called by
// the worker without the lock held (the lock guards the queue only).  The
// copies of every system of the pass go onto the copy stream back to back
// (the host prepares the next system while the previous one's copies run);
// the small host arrays are staged in pinned memory that stays untouched
// until the one synchronisation at the end of the pass, after which each
// system is checked and made resident.
void admit(cg_batch_ctx* b) {
  struct Staged {
    Job* j;
    cudaError_t e;
  };
  std::vector<Staged> staged;
  b->staging.reset();  // the previous pass ended with a synchronisation
  cudaStream_t s = b->copy;
  // host -> device from pinned staging (a copy the host may overwrite only
  // after the pass's synchronisation); without pinned memory, from src, and
  // the stream is drained before src can go away
  auto upload = [&](void* dst, const void* src, size_t bytes) -> cudaError_t {
    if (bytes == 0) return cudaSuccess;
    void* q = b->staging.take(bytes);
    if (q == nullptr) {
      cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s);
      return e == cudaSuccess ? cudaStreamSynchronize(s) : e;
    }
    std::memcpy(q, src, bytes);
    return cudaMemcpyAsync(dst, q, bytes, cudaMemcpyHostToDevice, s);
  };
  for (;;) {
    Job* j = nullptr;
    {
      std::lock_guard<std::mutex> lk(b->mu);
      if (b->stop || b->queued.empty()) break;
      if (b->free_slots.empty()) break;
      j = b->jobs[b->queued.front()].get();
    }
    const cg_request& r = j->req;
    std::vector<int32_t> rp, ci;
    std::string bad;
    if (!load_structure(r, b->validate, rp, ci, bad)) {
      std::lock_guard<std::mutex> lk(b->mu);
      b->queued.pop_front();
      finish_without_device(b, j, CG_EINVAL);
      b->err = "request " + std::to_string(j->ticket) + ": invalid CSR: " + bad;
      b->cv_done.notify_all();
      continue;
    }
    const int64_t n = r.n, nnz = r.nnz;
    const int group = b->calib_group > 0      ? std::min(b->calib_group, b->nblocks)
                      : b->group_override > 0 ? std::min(b->group_override, b->nblocks)
                                              : auto_group(b->model, n, nnz, b->mixed, b->nblocks);
    cgh::StepShape shape;
    {
      std::lock_guard<std::mutex> lk(b->mu);
      shape = b->shape;
    }
    cgh::Partition part;
    cgh::build_partition(rp, n, group, part, shape);
    const Layout L = layout_of(n, nnz, part.step.size(), group, b->mixed, b->jacobi);
    size_t off = 0;
    int slot = -1;
    {
      std::lock_guard<std::mutex> lk(b->mu);
      if (!b->arena.alloc(L.total, off)) break;  // wait for memory (arrival order is kept)
      slot = b->free_slots.back();
      b->free_slots.pop_back();
      b->queued.pop_front();
    }
    j->slot = slot;
    j->off = off;
    j->bytes = L.total;
    j->group = group;
    j->bytes_step = bytes_per_step(n, nnz, b->mixed);
    j->steps_est = est_steps(b->model, n);
    char* base = b->d_arena + off;
    auto at = [&](size_t o) { return base + o; };
    const size_t pad = cgk::kPadEntries;
    cudaError_t e = cudaSuccess;
    auto step = [&](cudaError_t x) {
      if (e == cudaSuccess) e = x;
    };
    step(upload(at(L.rp), rp.data(), 4 * (n + 1)));
    step(cudaMemsetAsync(at(L.col), 0, 4 * (nnz + pad), s));
    step(cudaMemsetAsync(at(L.val), 0, 8 * (nnz + pad), s));
    if (nnz > 0) {
      // the request's own arrays stay valid until its result is final
      const cudaMemcpyKind k = r.csr.on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
      if (r.csr.index_base == 0) {
        step(cudaMemcpyAsync(at(L.col), r.csr.col_idx, 4 * nnz, k, s));
      } else {
        if (ci.empty()) {  // not validated: the columns are not on the host yet
          if (r.csr.on_device) {
            ci.resize(static_cast<size_t>(nnz));
            step(cudaMemcpy(ci.data(), r.csr.col_idx, 4 * nnz, cudaMemcpyDeviceToHost));
          } else {
            ci.assign(r.csr.col_idx, r.csr.col_idx + nnz);
          }
        }
        for (auto& v : ci) v -= 1;
        step(upload(at(L.col), ci.data(), 4 * nnz));
      }
      step(cudaMemcpyAsync(at(L.val), r.csr.val, 8 * nnz, k, s));
      if (b->mixed) {
        step(cudaMemsetAsync(at(L.val32), 0, 4 * (nnz + pad), s));
        step(cgk::launch_f64_to_f32(nnz, reinterpret_cast<double*>(at(L.val)), reinterpret_cast<float*>(at(L.val32)),
                                    s));
      }
    }
    step(upload(at(L.step), part.step.data(), sizeof(int4) * part.step.size()));
    step(upload(at(L.mode), part.step_mode.data(), 4 * part.step_mode.size()));
    step(upload(at(L.bstep), part.block_step.data(), 4 * part.block_step.size()));
    step(upload(at(L.brow), part.block_row.data(), 4 * part.block_row.size()));
    step(cudaMemcpyAsync(at(L.b), r.b, 8 * n, is_device_ptr(r.b) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                         s));
    step(cudaMemsetAsync(at(L.x), 0, 8 * n, s));
    if (b->jacobi) {
      step(cudaMemsetAsync(b->d_admit_err + slot, 0, sizeof(int32_t), s));
      step(cgk::launch_jacobi_dinv(reinterpret_cast<int32_t*>(at(L.rp)), reinterpret_cast<int32_t*>(at(L.col)),
                                   reinterpret_cast<double*>(at(L.val)), n, reinterpret_cast<double*>(at(L.dinv)),
                                   b->d_admit_err + slot, s));
      step(cudaMemcpyAsync(b->h_admit_err + slot, b->d_admit_err + slot, sizeof(int32_t), cudaMemcpyDeviceToHost,
                           s));
    }
    step(cudaMemsetAsync(b->d_ctrl + slot, 0, sizeof(cgk::SolveCtrl), s));
    cgk::SolveParams& P = b->h_sys[slot];  // pinned; read by the copy below when it runs
    std::memset(&P, 0, sizeof(P));
    P.A.row_ptr = reinterpret_cast<int32_t*>(at(L.rp));
    P.A.col_idx = reinterpret_cast<int32_t*>(at(L.col));
    P.A.val = reinterpret_cast<double*>(at(L.val));
    P.A.val32 = b->mixed ? reinterpret_cast<float*>(at(L.val32)) : nullptr;
    P.A.step = reinterpret_cast<int4*>(at(L.step));
    P.A.step_mode = reinterpret_cast<int32_t*>(at(L.mode));
    P.A.block_step = reinterpret_cast<int32_t*>(at(L.bstep));
    P.A.block_row = reinterpret_cast<int32_t*>(at(L.brow));
    P.A.n = static_cast<int32_t>(n);
    P.A.nsteps = static_cast<int32_t>(part.step.size()) - 2;
    P.A.nblocks = group;
    for (int g = 0; g < group; ++g)
      P.A.max_rows = std::max(P.A.max_rows, part.block_row[g + 1] - part.block_row[g]);
    P.A.nnz = nnz;
    P.b = reinterpret_cast<double*>(at(L.b));
    P.x = reinterpret_cast<double*>(at(L.x));
    P.r = reinterpret_cast<double*>(at(L.r));
    P.p = reinterpret_cast<double*>(at(L.p));
    P.q = reinterpret_cast<double*>(at(L.q));
    P.p32 = b->mixed ? reinterpret_cast<float*>(at(L.p32)) : nullptr;
    P.partials = reinterpret_cast<double*>(at(L.part));
    P.ctrl = b->d_ctrl + slot;
    P.tol = r.tol;
    P.maxit = r.maxit;
    P.replace_every = b->replace_every;
    P.wait_limit_ns = b->wait_ns;
    P.group = group;
    P.chunk_iters = b->chunk_iters;
    P.dinv = b->jacobi ? reinterpret_cast<double*>(at(L.dinv)) : nullptr;
    step(cudaMemcpyAsync(b->d_sys + slot, &P, sizeof(P), cudaMemcpyHostToDevice, s));
    j->d_x = reinterpret_cast<double*>(at(L.x));
    staged.push_back({j, e});
  }
  if (staged.empty()) return;
  const cudaError_t es = cudaStreamSynchronize(s);
  std::vector<Job*> uploaded;
  for (const Staged& st : staged) {
    Job* j = st.j;
    const cudaError_t e = st.e != cudaSuccess ? st.e : es;
    const int slot = j->slot;
    if (e == cudaSuccess && b->jacobi && b->h_admit_err[slot] != 0) {
      std::lock_guard<std::mutex> lk(b->mu);
      b->arena.release(j->off, j->bytes);
      b->free_slots.push_back(slot);
      j->slot = -1;
      finish_without_device(b, j, CG_EINVAL);
      b->err = "request " + std::to_string(j->ticket) + ": Jacobi preconditioner: diagonal of row " +
               std::to_string(b->h_admit_err[slot] - 1) + " is not positive";
      b->cv_done.notify_all();
      continue;
    }
    if (e != cudaSuccess) {
      cudaGetLastError();
      std::lock_guard<std::mutex> lk(b->mu);
      b->arena.release(j->off, j->bytes);
      b->free_slots.push_back(slot);
      j->slot = -1;
      finish_without_device(b, j, CG_ECUDA);
      b->err = cuda_msg(e, "admission copies");
      b->cv_done.notify_all();
      continue;
    }
    uploaded.push_back(j);
  }
  if (!uploaded.empty()) {
    std::lock_guard<std::mutex> lk(b->mu);
    const double t = now_ms(b->t0);
    for (Job* j : uploaded) {
      j->state = kResident;
      j->res.admit_ms = t;
      j->res.group = j->group;
      b->resident.push_back(j);
      ++b->admitted;
    }
  }
}

// Build the task queue of a round: the tasks of every resident system (the
// ranks of a group next to each other), the longest estimated remaining
// time per CTA first.  CTAs take the next entry as they free up, so this is
// list scheduling in the longest-processing-time order: the round ends close
// to the total work over the grid, with the short tasks filling the tail.
// Returns the systems of the round.
//
// A group's ranks are taken as CTAs free up; its first ranks wait at their
// first group barrier meanwhile.  This cannot deadlock: take the first group
// in queue order with an entry not yet taken; every entry before it has been
// taken, no entry after it has, so every busy CTA outside that group runs a
// task that can finish (a one-CTA task or a group whose ranks are all
// running), and each group has at most as many ranks as the grid has CTAs.
// Such a wait lasts at most as long as the tasks ahead of the group in the
// queue, which the order makes no shorter than the group's own.
std::vector<Job*> build_queue(cg_batch_ctx* b, const std::vector<Job*>& res) {
  const GroupModel& m = b->model;
  auto remaining = [&](const Job* j) {
    const double left = std::max(1.0, j->steps_est - static_cast<double>(j->res.iters));
    const double steps = b->chunk_iters > 0 ? std::min(left, static_cast<double>(b->chunk_iters)) : left;
    const double per_step = j->group > 1 ? j->bytes_step / (j->group * m.group_rate) + m.overhead_g
                                         : j->bytes_step / m.cta_rate + m.overhead_1;
    return steps * per_step;
  };
  std::vector<std::pair<double, Job*>> order;
  order.reserve(res.size());
  int singles = 0;
  for (Job* j : res) {
    order.emplace_back(remaining(j), j);
    singles += j->group > 1 ? 0 : 1;
  }
  std::sort(order.begin(), order.end(), [](const std::pair<double, Job*>& a, const std::pair<double, Job*>& c) {
    return a.first != c.first ? a.first > c.first : a.second->ticket < c.second->ticket;
  });
  std::vector<Job*> in_round;
  int nt = 0;
  int room = b->task_cap - singles;
  for (const auto& e : order) {
    Job* j = e.second;
    if (j->group > 1) {
      if (j->group > room) continue;  // the queue is full: next round
      room -= j->group;
      for (int rk = 0; rk < j->group; ++rk) b->h_queue->task[nt++] = cgk::BatchTask{j->slot, rk};
    } else {
      b->h_queue->task[nt++] = cgk::BatchTask{j->slot, 0};
    }
    in_round.push_back(j);
  }
  b->h_queue->ntasks = nt;
  // the systems of a round run side by side: their vectors share the L2
  int64_t reused = 0;
  for (const Job* j : in_round) reused += cgk::step_reused_bytes(j->req.n, b->mixed, b->jacobi);
  b->h_queue->stream_rows = cgk::stream_row_ptrs(reused, b->l2_bytes) ? 1 : 0;
  return in_round;
}

// Copy out and release the finished systems of a round.
void retire(cg_batch_ctx* b, const std::vector<Job*>& in_round) {
  std::vector<Job*> fin;
  for (Job* j : in_round) {
    const cgk::SolveCtrl& c = b->h_ctrl[j->slot];
    j->res.rounds += 1;
    j->res.iters = c.iters;
    if (c.phase == cgk::kPhaseDone || c.status == cgk::kETIMEOUT) fin.push_back(j);
  }
  if (fin.empty()) return;
  cudaError_t e = cudaSuccess;
  for (Job* j : fin) {
    const size_t bytes = 8 * static_cast<size_t>(j->req.n);
    const cudaMemcpyKind k = is_device_ptr(j->req.x) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    cudaError_t e1 = cudaMemcpyAsync(j->req.x, j->d_x, bytes, k, b->copy);
    if (e == cudaSuccess) e = e1;
  }
  cudaError_t e2 = cudaStreamSynchronize(b->copy);
  if (e == cudaSuccess) e = e2;
  std::lock_guard<std::mutex> lk(b->mu);
  const double t = now_ms(b->t0);
  for (Job* j : fin) {
    const cgk::SolveCtrl& c = b->h_ctrl[j->slot];
    j->res.status = e == cudaSuccess ? c.status : CG_ECUDA;
    j->res.iters = c.iters;
    j->res.relres = c.relres_true;
    j->res.done = 1;
    j->res.done_ms = t;
    j->state = kFinished;
    b->arena.release(j->off, j->bytes);
    b->free_slots.push_back(j->slot);
    j->slot = -1;
    ++b->completed;
    b->resident.erase(std::find(b->resident.begin(), b->resident.end(), j));
  }
  if (e != cudaSuccess) b->err = cuda_msg(e, "copy of a solution");
  b->cv_done.notify_all();
}

void worker_main(cg_batch_ctx* b) {
  cudaSetDevice(b->device);
  for (;;) {
    std::vector<Job*> res;
    {
      std::unique_lock<std::mutex> lk(b->mu);
      b->cv_work.wait(lk, [&] { return b->stop || !b->queued.empty() || !b->resident.empty(); });
      if (b->stop) break;
      res = b->resident;
    }
    std::vector<Job*> in_round;
    bool launched = false;
    if (!res.empty()) {
      in_round = build_queue(b, res);
      cudaError_t e = cudaEventRecord(b->ev0, b->compute);
      if (e == cudaSuccess) e = b->use_graph ? cudaGraphLaunch(b->graph_exec, b->compute) : enqueue_round(b);
      if (e == cudaSuccess) e = cudaEventRecord(b->ev1, b->compute);
      if (e != cudaSuccess) {
        cudaGetLastError();
        std::lock_guard<std::mutex> lk(b->mu);
        b->err = cuda_msg(e, "round launch");
        for (Job* j : in_round) {
          b->arena.release(j->off, j->bytes);
          b->free_slots.push_back(j->slot);
          j->slot = -1;
          finish_without_device(b, j, CG_ECUDA);
          b->resident.erase(std::find(b->resident.begin(), b->resident.end(), j));
        }
        b->cv_done.notify_all();
        in_round.clear();
      } else {
        launched = true;
      }
    }
    admit(b);  // overlaps the round in flight
    if (launched) {
      cudaError_t e = cudaStreamSynchronize(b->compute);
      float ms = 0.0f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, b->ev0, b->ev1);
      {
        std::lock_guard<std::mutex> lk(b->mu);
        ++b->rounds;
        if (b->h_queue->stream_rows) ++b->rounds_stream_rows;
        b->last_round_ms = ms;
        b->round_ms_total += ms;
      }
      if (e != cudaSuccess) {
        std::lock_guard<std::mutex> lk(b->mu);
        b->err = cuda_msg(e, "round");
        for (Job* j : in_round) {
          j->slot = -1;
          finish_without_device(b, j, CG_ECUDA);
          b->resident.erase(std::find(b->resident.begin(), b->resident.end(), j));
        }
        b->cv_done.notify_all();
        b->stop = true;  // the context is unusable
        break;
      }
      retire(b, in_round);
    }
  }
}

void release_all(cg_batch_ctx* b) {
  if (b->graph_exec) cudaGraphExecDestroy(b->graph_exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->d_arena) cudaFree(b->d_arena);
  if (b->d_sys) cudaFree(b->d_sys);
  if (b->d_ctrl) cudaFree(b->d_ctrl);
  if (b->d_queue) cudaFree(b->d_queue);
  if (b->d_next) cudaFree(b->d_next);
  if (b->d_admit_err) cudaFree(b->d_admit_err);
  if (b->h_admit_err) cudaFreeHost(b->h_admit_err);
  if (b->h_sys) cudaFreeHost(b->h_sys);
  if (b->h_ctrl) cudaFreeHost(b->h_ctrl);
  if (b->h_queue) cudaFreeHost(b->h_queue);
  if (b->ev0) cudaEventDestroy(b->ev0);
  if (b->ev1) cudaEventDestroy(b->ev1);
  if (b->compute) cudaStreamDestroy(b->compute);
  if (b->copy) cudaStreamDestroy(b->copy);
}

bool request_ok(const cg_request& r, std::string& why) {
  const int64_t kMaxIdx = 2147483647LL - 16;
  if (r.n < 0 || r.nnz < 0 || r.n > kMaxIdx || r.nnz > kMaxIdx) why = "n and nnz must be in [0, 2^31 - 16)";
  else if (r.csr.index_base != 0 && r.csr.index_base != 1) why = "index_base must be 0 or 1";
  else if (r.n > 0 && (!r.csr.row_ptr || !r.b || !r.x)) why = "NULL row_ptr, b or x";
  else if (r.nnz > 0 && (!r.csr.col_idx || !r.csr.val)) why = "NULL col_idx or val";
  else if (!(r.tol >= 0.0)) why = "tol must be >= 0";
  else if (r.maxit < 0) why = "maxit must be >= 0";
  return why.empty();
}

// 27-point stencil on an m^3 grid, boundary eliminated: diagonal 27, each
// of the (up to) 26 neighbours -1 (strictly diagonally dominant, hence SPD).
// A timing workload of the calibration only.
void stencil27(int m, std::vector<int32_t>& rp, std::vector<int32_t>& ci, std::vector<double>& va) {
  const int64_t n = static_cast<int64_t>(m) * m * m;
  rp.assign(static_cast<size_t>(n) + 1, 0);
  ci.clear();
  va.clear();
  for (int z = 0; z < m; ++z)
    for (int y = 0; y < m; ++y)
      for (int x = 0; x < m; ++x) {
        const int64_t i = (static_cast<int64_t>(z) * m + y) * m + x;
        for (int dz = -1; dz <= 1; ++dz)
          for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
              const int zz = z + dz, yy = y + dy, xx = x + dx;
              if (zz < 0 || yy < 0 || xx < 0 || zz >= m || yy >= m || xx >= m) continue;
              const int64_t j = (static_cast<int64_t>(zz) * m + yy) * m + xx;
              ci.push_back(static_cast<int32_t>(j));
              va.push_back(j == i ? 27.0 : -1.0);
            }
        rp[static_cast<size_t>(i) + 1] = static_cast<int32_t>(ci.size());
      }
}

// Device time per step when `copies` copies of one system are solved
// together, each by `group` CTAs, for exactly `steps` steps (tol 0).  < 0 if
// they do not fit the budget at once or a request failed.
double time_per_step(cg_batch_ctx* b, const std::vector<int32_t>& rp, const std::vector<int32_t>& ci,
                     const std::vector<double>& va, int copies, int group, int steps) {
  const int64_t n = static_cast<int64_t>(rp.size()) - 1, nnz = static_cast<int64_t>(ci.size());
  if (copies <= 0 || static_cast<size_t>(copies) * footprint_bound(n, nnz, b->mixed, b->jacobi, b->nblocks) >
                         b->arena.cap() ||
      copies > b->max_systems)
    return -1.0;
  std::vector<double> bv(static_cast<size_t>(n), 1.0);
  std::vector<std::vector<double>> xs(static_cast<size_t>(copies), std::vector<double>(static_cast<size_t>(n)));
  std::vector<cg_request> reqs(static_cast<size_t>(copies));
  for (int i = 0; i < copies; ++i) {
    cg_request& r = reqs[static_cast<size_t>(i)];
    std::memset(&r, 0, sizeof(r));
    r.csr.row_ptr = rp.data();
    r.csr.col_idx = ci.data();
    r.csr.val = va.data();
    r.n = n;
    r.nnz = nnz;
    r.b = bv.data();
    r.x = xs[static_cast<size_t>(i)].data();
    r.tol = 0.0;
    r.maxit = steps;
  }
  {
    std::lock_guard<std::mutex> lk(b->mu);
    b->calib_group = group;
  }
  cg_batch_stats s0, s1;
  cg_batch_get_stats(b, &s0);
  std::vector<uint64_t> tickets(static_cast<size_t>(copies));
  bool ok = cg_batch_submit(b, reqs.data(), copies, tickets.data()) == CG_OK;
  for (size_t i = 0; ok && i < tickets.size(); ++i) {
    cg_result r;
    if (cg_batch_wait(b, tickets[i], 60000, &r) != CG_OK || !r.done || (r.status != CG_OK && r.status != CG_ENOTCONV))
      ok = false;
  }
  cg_batch_get_stats(b, &s1);
  {
    std::lock_guard<std::mutex> lk(b->mu);
    b->calib_group = 0;
  }
  if (!ok) return -1.0;
  return (s1.round_ms_total - s0.round_ms_total) * 1e-3 / steps;
}

// Banded system of n rows with rows of L entries inside (L odd): columns
// i - (L-1)/2 .. i + (L-1)/2, diagonal L + 1, the others -1 (strictly
// diagonally dominant, hence SPD).  A timing workload of the calibration only.
void banded(int64_t n, int L, std::vector<int32_t>& rp, std::vector<int32_t>& ci, std::vector<double>& va) {
  const int64_t h = (L - 1) / 2;
  rp.assign(static_cast<size_t>(n) + 1, 0);
  ci.clear();
  va.clear();
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t j = std::max<int64_t>(0, i - h); j <= std::min<int64_t>(n - 1, i + h); ++j) {
      ci.push_back(static_cast<int32_t>(j));
      va.push_back(j == i ? static_cast<double>(L + 1) : -1.0);
    }
    rp[static_cast<size_t>(i) + 1] = static_cast<int32_t>(ci.size());
  }
}

// Row-length buckets of the step-shape table: rows of (kShapeLo[k], kShapeHi[k]]
// entries share one step kind, measured on a banded system whose rows have
// kShapeRep[k] entries.
constexpr int kShapeBuckets = 6;
constexpr int kShapeHi[kShapeBuckets] = {8, 16, 24, 32, 48, 64};
constexpr int kShapeRep[kShapeBuckets] = {7, 15, 23, 31, 47, 63};

// The autotuner of the step shapes: for each bucket of row lengths, time one
// copy per CTA of a banded system with such rows (one CTA each, every SM busy,
// a fixed number of steps) with each step kind the rows allow (one lane or
// two lanes per row up to 32 entries, two lanes or a warp per row above), and
// keep the kind of the shortest time; the built-in kind stays unless another
// is at least 2 % faster.  The table then applies to every system the batch
// object admits, so a system's partition still depends on the system alone.
void calibrate_shape(cg_batch_ctx* b) {
  constexpr int kSteps = 40;
  cgh::StepShape best;  // the built-in table
  bool measured_all = true;
  for (int k = 0; k < kShapeBuckets; ++k) {
    const int L = kShapeRep[k];
    std::vector<int32_t> rp, ci;
    std::vector<double> va;
    banded(static_cast<int64_t>(131072) / L, L, rp, ci, va);
    const int lo = k == 0 ? 0 : kShapeHi[k - 1] + 1;
    const int cand[2] = {L <= cgk::kLaneMax ? cgk::kLanePerRow : cgk::kPairPerRow,
                         L <= cgk::kLaneMax ? cgk::kPairPerRow : cgk::kLongRow};
    double t[2] = {-1.0, -1.0};
    for (int c = 0; c < 2; ++c) {
      cgh::StepShape trial = best;
      for (int len = lo; len <= kShapeHi[k]; ++len) trial.mode[len] = static_cast<int8_t>(cand[c]);
      {
        std::lock_guard<std::mutex> lk(b->mu);
        b->shape = trial;
      }
      t[c] = time_per_step(b, rp, ci, va, b->nblocks, 1, kSteps);
    }
    if (t[0] <= 0 || t[1] <= 0) {
      measured_all = false;
      continue;
    }
    const int pick = t[1] < 0.98 * t[0] ? cand[1] : cand[0];
    for (int len = lo; len <= kShapeHi[k]; ++len) best.mode[len] = static_cast<int8_t>(pick);
  }
  std::lock_guard<std::mutex> lk(b->mu);
  b->shape = best.valid() ? best : cgh::StepShape();
  b->shape_tuned = measured_all && best.valid();
}

// The autotuner of the group size: measure the cost model's rates and
// per-step overheads on this GPU with synthetic 27-point systems, all CTAs
// busy.  One-CTA systems of two sizes give the rate and overhead of G = 1
// (time per step = bytes / rate + overhead); one size solved by groups of 8
// and of 16 CTAs gives those of groups.  Any measurement that fails or is
// inconsistent keeps the built-in value.  The step shapes are tuned first,
// and the group model is measured with them.
void calibrate(cg_batch_ctx* b) {
  if (!b->shape_fixed) calibrate_shape(b);
  std::vector<int32_t> rp0, ci0, rp1, ci1, rp2, ci2;
  std::vector<double> va0, va1, va2;
  stencil27(10, rp0, ci0, va0);
  stencil27(20, rp1, ci1, va1);
  stencil27(40, rp2, ci2, va2);
  constexpr int kSteps = 40;
  const double t0 = time_per_step(b, rp0, ci0, va0, b->nblocks, 1, kSteps);
  const double t1 = time_per_step(b, rp1, ci1, va1, b->nblocks, 1, kSteps);
  const double t8 = time_per_step(b, rp2, ci2, va2, b->nblocks / 8, 8, kSteps);
  const double t16 = time_per_step(b, rp2, ci2, va2, b->nblocks / 16, 16, kSteps);
  auto bytes = [&](const std::vector<int32_t>& rp, const std::vector<int32_t>& ci) {
    return bytes_per_step(static_cast<int64_t>(rp.size()) - 1, static_cast<int64_t>(ci.size()), b->mixed);
  };
  const double B0 = bytes(rp0, ci0), B1 = bytes(rp1, ci1), B2 = bytes(rp2, ci2);
  GroupModel m = b->model;
  bool got1 = false, got_g = false;
  if (t0 > 0 && t1 > t0) {
    const double rate = (B1 - B0) / (t1 - t0), ov = t0 - B0 / rate;
    if (rate > 0 && ov >= 0) {
      m.cta_rate = rate;
      m.overhead_1 = ov;
      got1 = true;
    }
  }
  if (t8 > 0 && t16 > 0 && t8 > t16) {
    const double rate = B2 / (16.0 * (t8 - t16)), ov = 2.0 * t16 - t8;
    if (rate > 0 && ov >= 0) {
      m.group_rate = rate;
      m.overhead_g = ov;
      got_g = true;
    }
  }
  std::lock_guard<std::mutex> lk(b->mu);
  b->model = m;
  b->autotuned = got1 && got_g;
}

}  // namespace

extern "C" {

void cg_batch_opts_default(cg_batch_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->device = -1;
  o->precision = CG_PREC_FP64;
  o->budget_bytes = 0;
  o->max_systems = 1024;
  o->chunk_iters = 0;
  o->replace_every = 50;
  o->wait_limit_ms = 2000;
  o->max_pending = 65536;
  o->use_graph = 1;
  o->group_override = 0;
  o->validate = 1;
  o->preconditioner = CG_PRECOND_NONE;
  o->autotune = 0;
  o->group_target_ms = 50;
}

const char* cg_batch_last_error(cg_batch b) {
  if (!b) return g_batch_create_err.c_str();
  std::lock_guard<std::mutex> lk(b->mu);
  thread_local std::string copy;
  copy = b->err;
  return copy.c_str();
}

int cg_batch_create(cg_batch* out, const cg_batch_opts* opts) {
  if (!out) return bfail(nullptr, CG_EINVAL, "cg_batch_create: out is NULL");
  *out = nullptr;
  cg_batch_opts o;
  cg_batch_opts_default(&o);
  if (opts) o = *opts;
  if (o.precision != CG_PREC_FP64 && o.precision != CG_PREC_MIXED)
    return bfail(nullptr, CG_EINVAL, "cg_batch_create: unknown precision");
  if (o.max_systems <= 0 || o.max_systems > (1 << 20) || o.chunk_iters < 0 || o.replace_every < 0 ||
      o.budget_bytes < 0 || o.max_pending <= 0 || o.group_override < 0 ||
      (o.preconditioner != CG_PRECOND_NONE && o.preconditioner != CG_PRECOND_JACOBI) || o.autotune < 0 ||
      o.autotune > 1 || o.group_target_ms <= 0 || o.step_shape < 0 || o.step_shape > 3)
    return bfail(nullptr, CG_EINVAL, "cg_batch_create: bad option");
  auto b = std::make_unique<cg_batch_ctx>();
  if (o.step_shape > 0) {
    // 1: the built-in shapes; 2: two lanes per row up to 64 entries; 3: a warp per row
    for (int L = 0; L <= cgh::kShapeMaxLen; ++L) {
      if (o.step_shape == 2) b->shape.mode[L] = static_cast<int8_t>(cgk::kPairPerRow);
      if (o.step_shape == 3) b->shape.mode[L] = static_cast<int8_t>(cgk::kLongRow);
    }
    b->shape_fixed = true;
  }
  if (o.device >= 0) b->device = o.device;
  else if (cudaGetDevice(&b->device) != cudaSuccess) return bfail(nullptr, CG_ECUDA, "cg_batch_create: no device");
  if (cudaSetDevice(b->device) != cudaSuccess) {
    cudaGetLastError();
    return bfail(nullptr, CG_ECUDA, "cg_batch_create: cannot use the device");
  }
  b->mixed = o.precision == CG_PREC_MIXED;
  b->jacobi = o.preconditioner == CG_PRECOND_JACOBI;
  b->max_systems = o.max_systems;
  b->chunk_iters = o.chunk_iters;
  b->replace_every = o.replace_every;
  b->wait_ns = static_cast<unsigned long long>(o.wait_limit_ms > 0 ? o.wait_limit_ms : 2000) * 1000000ull;
  b->max_pending = o.max_pending;
  b->group_override = o.group_override;
  b->model.target_s = 1e-3 * o.group_target_ms;
  b->validate = o.validate != 0;
  b->use_graph = o.use_graph != 0;
  b->t0 = std::chrono::steady_clock::now();

  int sms = 0;
  cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
  const int per_sm = e == cudaSuccess ? cgk::batch_blocks_per_sm(b->mixed, b->jacobi) : -1;
  if (e != cudaSuccess || per_sm <= 0) {
    cudaGetLastError();
    return bfail(nullptr, CG_ECUDA, "cg_batch_create: the batch kernel cannot be resident");
  }
  b->nblocks = sms * per_sm;
  int l2 = 0;
  if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, b->device) != cudaSuccess) {
    cudaGetLastError();
    l2 = 0;
  }
  b->l2_bytes = l2;
  b->model.cta_rate = 6.7e12 / b->nblocks;
  // queue capacity: every resident system once, plus the extra ranks of
  // groups (a round whose groups need more is split over rounds)
  b->task_cap = 2 * b->max_systems + 8 * b->nblocks;
  b->queue_bytes = sizeof(cgk::BatchQueue) + sizeof(cgk::BatchTask) * (b->task_cap - 1);

  size_t budget = static_cast<size_t>(o.budget_bytes);
  if (budget == 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      cudaGetLastError();
      return bfail(nullptr, CG_ECUDA, "cg_batch_create: cudaMemGetInfo");
    }
    budget = fr / 2;
  }
  budget &= ~(kAlign - 1);
  auto fail_cuda = [&](cudaError_t err, const char* what) {
    cudaGetLastError();
    release_all(b.get());
    return bfail(nullptr, err == cudaErrorMemoryAllocation ? CG_ENOMEM : CG_ECUDA, cuda_msg(err, what));
  };
  if ((e = cudaStreamCreateWithFlags(&b->compute, cudaStreamNonBlocking)) != cudaSuccess)
    return fail_cuda(e, "cg_batch_create: stream");
  if ((e = cudaStreamCreateWithFlags(&b->copy, cudaStreamNonBlocking)) != cudaSuccess)
    return fail_cuda(e, "cg_batch_create: stream");
  if ((e = cudaEventCreate(&b->ev0)) != cudaSuccess || (e = cudaEventCreate(&b->ev1)) != cudaSuccess)
    return fail_cuda(e, "cg_batch_create: events");
  if (budget && (e = cudaMalloc(&b->d_arena, budget)) != cudaSuccess)
    return fail_cuda(e, "cg_batch_create: budget allocation");
  b->arena.init(budget);
  if ((e = cudaMalloc(&b->d_sys, sizeof(cgk::SolveParams) * b->max_systems)) != cudaSuccess ||
      (e = cudaMalloc(&b->d_ctrl, sizeof(cgk::SolveCtrl) * b->max_systems)) != cudaSuccess ||
      (e = cudaMalloc(&b->d_queue, b->queue_bytes)) != cudaSuccess ||
      (e = cudaMalloc(&b->d_next, 16)) != cudaSuccess ||
      (e = cudaMalloc(&b->d_admit_err, sizeof(int32_t) * b->max_systems)) != cudaSuccess)
    return fail_cuda(e, "cg_batch_create: tables");
  if ((e = cudaMallocHost(&b->h_sys, sizeof(cgk::SolveParams) * b->max_systems)) != cudaSuccess ||
      (e = cudaMallocHost(&b->h_ctrl, sizeof(cgk::SolveCtrl) * b->max_systems)) != cudaSuccess ||
      (e = cudaMallocHost(&b->h_queue, b->queue_bytes)) != cudaSuccess ||
      (e = cudaMallocHost(&b->h_admit_err, sizeof(int32_t) * b->max_systems)) != cudaSuccess)
    return fail_cuda(e, "cg_batch_create: pinned tables");
  std::memset(b->h_queue, 0, b->queue_bytes);
  if ((e = cudaMemset(b->d_ctrl, 0, sizeof(cgk::SolveCtrl) * b->max_systems)) != cudaSuccess ||
      (e = cudaMemset(b->d_sys, 0, sizeof(cgk::SolveParams) * b->max_systems)) != cudaSuccess)
    return fail_cuda(e, "cg_batch_create: clear");
  b->free_slots.reserve(b->max_systems);
  for (int s = b->max_systems - 1; s >= 0; --s) b->free_slots.push_back(s);
  try_capture(b.get());
  if ((e = cudaDeviceSynchronize()) != cudaSuccess) return fail_cuda(e, "cg_batch_create: synchronize");
  cg_batch_ctx* raw = b.release();
  raw->worker = std::thread(worker_main, raw);
  if (o.autotune) calibrate(raw);
  *out = raw;
  return CG_OK;
}

int cg_batch_destroy(cg_batch b) {
  if (!b) return CG_OK;
  {
    std::lock_guard<std::mutex> lk(b->mu);
    b->stop = true;
  }
  b->cv_work.notify_all();
  if (b->worker.joinable()) b->worker.join();
  int cur = -1;
  cudaGetDevice(&cur);
  cudaSetDevice(b->device);
  cudaStreamSynchronize(b->compute);
  cudaStreamSynchronize(b->copy);
  release_all(b);
  if (cur >= 0) cudaSetDevice(cur);
  delete b;
  return CG_OK;
}

int cg_batch_submit(cg_batch b, const cg_request* reqs, int32_t count, uint64_t* tickets) {
  if (!b) return bfail(nullptr, CG_EINVAL, "cg_batch_submit: NULL batch");
  if (count < 0 || (count > 0 && (!reqs || !tickets))) return bfail(b, CG_EINVAL, "cg_batch_submit: bad arguments");
  for (int32_t i = 0; i < count; ++i) {
    std::string why;
    if (!request_ok(reqs[i], why))
      return bfail(b, CG_EINVAL, "cg_batch_submit: request " + std::to_string(i) + ": " + why);
    const size_t need = footprint_bound(reqs[i].n, reqs[i].nnz, b->mixed, b->jacobi, b->nblocks);
    if (need > b->arena.cap())
      return bfail(b, CG_ENOMEM, "cg_batch_submit: request " + std::to_string(i) + " needs up to " +
                                     std::to_string(need) + " bytes, more than the budget of " +
                                     std::to_string(b->arena.cap()));
  }
  {
    std::lock_guard<std::mutex> lk(b->mu);
    if (b->stop) {
      b->err = "cg_batch_submit: the batch object has stopped";
      return CG_ECUDA;
    }
    if (static_cast<int64_t>(b->queued.size()) + count > b->max_pending) {
      b->err = "cg_batch_submit: pending queue full";
      return CG_EBUSY;
    }
    const double t = now_ms(b->t0);
    for (int32_t i = 0; i < count; ++i) {
      auto j = std::make_unique<Job>();
      j->ticket = b->next_ticket++;
      j->req = reqs[i];
      j->res.ticket = j->ticket;
      j->res.tag = reqs[i].tag;
      j->res.submit_ms = t;
      tickets[i] = j->ticket;
      ++b->submitted;
      if (reqs[i].n == 0) {  // nothing to solve
        j->res.admit_ms = t;
        finish_without_device(b, j.get(), CG_OK);
      } else {
        b->queued.push_back(j->ticket);
      }
      b->jobs.emplace(j->ticket, std::move(j));
    }
  }
  b->cv_work.notify_all();
  b->cv_done.notify_all();
  return CG_OK;
}

int cg_batch_wait(cg_batch b, uint64_t ticket, int32_t timeout_ms, cg_result* res) {
  if (!b || !res) return bfail(b, CG_EINVAL, "cg_batch_wait: bad arguments");
  std::unique_lock<std::mutex> lk(b->mu);
  auto it = b->jobs.find(ticket);
  if (it == b->jobs.end()) {
    b->err = "cg_batch_wait: unknown ticket";
    return CG_EINVAL;
  }
  Job* j = it->second.get();
  auto finished = [&] { return j->state == kFinished || b->stop; };
  if (timeout_ms < 0) b->cv_done.wait(lk, finished);
  else if (timeout_ms > 0) b->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), finished);
  *res = j->res;
  if (j->state == kFinished) b->jobs.erase(it);
  else res->done = 0;
  return CG_OK;
}

int cg_batch_poll(cg_batch b, uint64_t ticket, cg_result* res) { return cg_batch_wait(b, ticket, 0, res); }

int cg_batch_get_stats(cg_batch b, cg_batch_stats* st) {
  if (!b || !st) return bfail(b, CG_EINVAL, "cg_batch_get_stats: bad arguments");
  std::lock_guard<std::mutex> lk(b->mu);
  st->rounds = b->rounds;
  st->submitted = b->submitted;
  st->admitted = b->admitted;
  st->completed = b->completed;
  st->pending = static_cast<int64_t>(b->queued.size());
  st->resident = static_cast<int64_t>(b->resident.size());
  st->bytes_in_use = static_cast<int64_t>(b->arena.in_use);
  st->bytes_peak = static_cast<int64_t>(b->arena.peak);
  st->budget_bytes = static_cast<int64_t>(b->arena.cap());
  st->graph = b->use_graph ? 1 : 0;
  st->nblocks = b->nblocks;
  st->round_ms_total = b->round_ms_total;
  st->last_round_ms = b->last_round_ms;
  st->cta_bytes_per_s = b->model.cta_rate;
  st->group_cta_bytes_per_s = b->model.group_rate;
  st->step_overhead_s = b->model.overhead_1;
  st->group_step_overhead_s = b->model.overhead_g;
  st->autotuned = b->autotuned ? 1 : 0;
  st->shape_tuned = b->shape_tuned ? 1 : 0;
  for (int k = 0; k < kShapeBuckets; ++k) st->step_kind[k] = b->shape.mode[kShapeHi[k]];
  st->pad = 0;
  st->rounds_stream_rows = b->rounds_stream_rows;
  return CG_OK;
}

int cg_batch_group_for(cg_batch b, const int32_t* row_ptr, int64_t n, int32_t* group) {
  if (!b || !row_ptr || !group || n < 0) return bfail(b, CG_EINVAL, "cg_batch_group_for: bad arguments");
  const int64_t nnz = static_cast<int64_t>(row_ptr[n]) - row_ptr[0];
  *group = b->group_override > 0 ? std::min(b->group_override, b->nblocks)
                                 : auto_group(b->model, n, nnz, b->mixed, b->nblocks);
  return CG_OK;
}

}  // extern "C"
