// CSR product and the persistent conjugate-gradient solves.
//
// Classical CG (the paper's Sec. 5.3 solver; no preconditioner), one
// cooperative launch per solve (or, batched, per set of systems):
//   setup     r = b - A x, p = r, rho = r.r, ||b||^2          (product + 2 sums)
//   each step q = A p, gamma = p.q                            (product fused with the sum)
//             alpha = rho/gamma; r -= alpha q, rho' = r.r     (update fused with the sum)
//             stop if sqrt(rho') <= tol ||b||
//             beta = rho'/rho; x += alpha p; p = r + beta p   (x update deferred here)
//   exit      ||b - A x|| / ||b||                             (true residual)
// alpha, beta and the stopping test are computed on the device by every CTA
// from the same deterministic sums, so no host synchronisation happens per
// step and every CTA takes the same branch.  Each CTA owns a fixed range of
// rows (a run of product steps) for all phases, so only the two sums and the
// gather of p need synchronisation across the CTAs that share the system:
// three group barriers per step.  A single-system solve uses the whole grid
// as one group; a batched solve gives each system its own group of CTAs (one
// CTA for most systems) and lets CTAs take systems from a queue.
//
// The mixed-precision variant keeps an FP32 copy of the values and an FP32
// shadow of p: the product is FP32 (FP32 accumulation); sums, alpha, beta, x
// and r stay FP64; every `replace_every` steps, and before accepting
// convergence, r is replaced by the FP64 true residual b - A x.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <set>
#include <utility>
#include "cg_solve.cuh"

namespace cgk {

// One system on the whole grid: CTA c is rank c of the group.  kJacobi:
// preconditioned by M = diag(A) (P.dinv).
template <bool kMixed, bool kJacobi, bool kSmallShare>
__global__ void __launch_bounds__(kBlock, kCtasPerSm) cg_solve_kernel(const __grid_constant__ SolveParams P) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const RingSmem sm{smem_raw, kMixed ? 4u : 8u};  // the step loop streams FP32 values in the mixed solve
  CtaStream cs;
  stream_setup(sm, cs, P.A, blockIdx.x);  // the last barrier of all threads
  if (threadIdx.x >= kConsumers) {
    solve_producer<kMixed>(sm, cs, P);
    return;
  }
  // the neighbour wait at the end of a step pays off on large shares (160^3:
  // 1.6 % faster); on small ones the group barrier is faster (64^3: 1 %, 16^3: 9 %)
  solve_consumers<kMixed, kJacobi, kSmallShare, !kSmallShare>(sm, cs, P, blockIdx.x, &P.stream_rows);
}

// The product alone reads every row pointer once: always evict-first.
__constant__ int32_t kStreamRowsAlways = 1;

// y = A x (same partition and stream as the solve; one pass).
__global__ void __launch_bounds__(kBlock, kCtasPerSm) spmv_kernel(const DevCsr A, const double* __restrict__ x,
                                                                   double* __restrict__ y, int32_t* err) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const RingSmem sm{smem_raw};
  CtaStream cs;
  stream_setup(sm, cs, A, blockIdx.x);
  const unsigned long long lim = 2000000000ull;
  if (threadIdx.x >= kConsumers) {
    if (threadIdx.x == kConsumers && !producer_loop<double>(sm, cs, A.val, A.col_idx, 1, lim)) atomicExch(err, kETIMEOUT);
    return;
  }
  ConsumerCursor cur;
  auto epi = [&](int i, double s, double) { y[i] = s; };
  const bool ok = cta_and(spmv_pass<true, double, double, double>(sm, cs, cur, A, A.val, x, nullptr, epi, lim, &kStreamRowsAlways));
  if (!ok && threadIdx.x == 0) atomicExch(err, kETIMEOUT);
  consumers_done(sm);
}

// Opt a kernel in to `bytes` of dynamic shared memory, and ask for the
// smallest shared-memory carveout that holds them (the rest of the SM's
// 256 KB serves as L1 for the product's gathers), once per (kernel, device).
cudaError_t ensure_smem_attr(const void* kernel, size_t bytes) {
  static std::mutex mu;
  static std::set<std::pair<const void*, int>> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  if (done.count({kernel, dev})) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(bytes));
  int max_sm = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&max_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  if (e == cudaSuccess && max_sm > 0) {
    // a hint: CUDA picks the nearest supported carveout that the launch fits in
    const size_t need = bytes + 1024;  // + the CTA's reserved shared memory
    int pct = static_cast<int>((need * 100 + static_cast<size_t>(max_sm) - 1) / static_cast<size_t>(max_sm));
    if (pct > 100) pct = 100;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
  }
  if (e == cudaSuccess) done.insert({kernel, dev});
  return e;
}

cudaError_t launch_spmv(const DevCsr& A, const double* x, double* y, int32_t* err, cudaStream_t s) {
  constexpr size_t kSmem = ring_smem_bytes<double>();
  cudaError_t e = ensure_smem_attr(reinterpret_cast<const void*>(spmv_kernel), kSmem);
  if (e != cudaSuccess) return e;
  spmv_kernel<<<A.nblocks, kBlock, kSmem, s>>>(A, x, y, err);
  return cudaGetLastError();
}

template <bool kSmallShare>
const void* solve_kernel_ptr_t(bool mixed, bool jacobi) {
  if (mixed) return jacobi ? reinterpret_cast<const void*>(cg_solve_kernel<true, true, kSmallShare>)
                           : reinterpret_cast<const void*>(cg_solve_kernel<true, false, kSmallShare>);
  return jacobi ? reinterpret_cast<const void*>(cg_solve_kernel<false, true, kSmallShare>)
                : reinterpret_cast<const void*>(cg_solve_kernel<false, false, kSmallShare>);
}

const void* solve_kernel_ptr(bool mixed, bool jacobi, bool small_share = false) {
  return small_share ? solve_kernel_ptr_t<true>(mixed, jacobi) : solve_kernel_ptr_t<false>(mixed, jacobi);
}

size_t solve_smem_bytes(bool mixed, bool local) {
  return mixed ? ring_smem_bytes<float>(local) : ring_smem_bytes<double>(local);
}

int solve_blocks_per_sm(bool mixed, bool jacobi) {
  int nb = 0;
  for (const bool small : {false, true}) {  // both must fit (one CTA per SM)
    const void* k = solve_kernel_ptr(mixed, jacobi, small);
    const size_t smem = solve_smem_bytes(mixed, small);
    cudaError_t e = ensure_smem_attr(k, smem);
    int nk = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nk, k, kBlock, smem);
    if (e != cudaSuccess) return -1;
    nb = small ? std::min(nb, nk) : nk;
  }
  return nb;
}

cudaError_t launch_solve(const SolveParams& P, bool mixed, cudaStream_t s) {
  void* args[] = {const_cast<SolveParams*>(&P)};
  // the small-share kernel: every CTA's rows fit its shared r, and the
  // solve runs in this one launch
  const bool small = small_share(P.A, P.chunk_iters);
  const void* k = solve_kernel_ptr(mixed, P.dinv != nullptr, small);
  const size_t smem = solve_smem_bytes(mixed, small);
  cudaError_t e = ensure_smem_attr(k, smem);
  if (e != cudaSuccess) return e;
  return cudaLaunchCooperativeKernel(k, dim3(P.A.nblocks), dim3(kBlock), args, smem, s);
}

// dinv[i] = 1 / diag(A)_i (the diagonal summed over row i's entries in
// column i, in storage order); err <- first row (+1) without a positive one.
__global__ void jacobi_dinv_kernel(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx,
                                   const double* __restrict__ val, int64_t n, double* __restrict__ dinv,
                                   int32_t* err) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    double d = 0.0;
    for (int k = row_ptr[i]; k < row_ptr[i + 1]; ++k)
      if (col_idx[k] == i) d += val[k];
    if (d > 0.0) {
      dinv[i] = 1.0 / d;
    } else {
      dinv[i] = 0.0;
      atomicCAS(err, 0, static_cast<int32_t>(i + 1));
    }
  }
}

cudaError_t launch_jacobi_dinv(const int32_t* row_ptr, const int32_t* col_idx, const double* val, int64_t n,
                               double* dinv, int32_t* err, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int64_t blocks = (n + 255) / 256;
  jacobi_dinv_kernel<<<static_cast<unsigned>(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(row_ptr, col_idx, val, n,
                                                                                        dinv, err);
  return cudaGetLastError();
}

// ---- self-test of the bounded wait: thread 0 of one CTA arrives at the
// group barrier of the solves (group_barrier_t0) for a group of two CTAs that
// no other CTA joins, so its wait must run out after limit_ns, raise the
// abort flag, record the site and report kETIMEOUT through the control block.
__global__ void wait_timeout_selftest_kernel(SolveCtrl* ctrl, unsigned long long limit_ns) {
  __shared__ unsigned long long target;
  if (threadIdx.x == 0) {
    target = 0;
    const bool ok = group_barrier_t0(ctrl, &target, 2u, limit_ns, kSelftestSite);
    ctrl->status = ok ? kOK : kETIMEOUT;
  }
}

cudaError_t launch_wait_timeout_selftest(SolveCtrl* ctrl, unsigned long long limit_ns, cudaStream_t s) {
  wait_timeout_selftest_kernel<<<1, 32, 0, s>>>(ctrl, limit_ns);
  return cudaGetLastError();
}

// ---- cost of the solves' group-wide synchronisations on the whole grid
// (one CTA per SM, the solve kernel's block): `iters` times, between CTA
// barriers as in a solve step, warp 0 of every CTA either meets the others at
// the group barrier (mode 0: group_barrier_t0), or runs a group sum (mode 1:
// publishes the CTA's value in one of two alternating slots, meets the others
// at the barrier, and sums the group's values exactly with
// fx_warp_sum_array, as group_sum in the solve does).  The waits are the
// solves' bounded ones: a wait that gives up raises ctrl->abort, after which
// every CTA stops.  out[rank] keeps the sums live.
__global__ void __launch_bounds__(kBlock, kCtasPerSm)
    sync_probe_kernel(SolveCtrl* ctrl, double* partials, int iters, int mode, unsigned long long limit_ns,
                      double* out) {
  __shared__ unsigned long long target;
  __shared__ int ok;
  __shared__ double total;
  const int nb = static_cast<int>(gridDim.x), rank = static_cast<int>(blockIdx.x);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    target = 0;
    ok = 1;
    total = 0.0;
  }
  __syncthreads();
  double acc = 0.0;
  for (int k = 0; k < iters; ++k) {
    if (warp == 0) {
      double* part = partials + static_cast<size_t>(k & 1) * nb;
      int good = 1;
      if (lane == 0) {
        if (mode == 1) part[rank] = static_cast<double>(rank + k);
        good = group_barrier_t0(ctrl, &target, static_cast<unsigned int>(nb), limit_ns, kProbeSite) ? 1 : 0;
      }
      good = __shfl_sync(0xffffffffu, good, 0);
      if (good && mode == 1) {
        const double sum = fx_warp_sum_array(part, nb);
        if (lane == 0) total = sum;
      }
      if (lane == 0 && !good) ok = 0;
    }
    __syncthreads();
    if (!ok) break;
    acc += total;
    __syncthreads();  // total is rewritten by the next sum
  }
  if (threadIdx.x == 0) out[rank] = acc;
}

cudaError_t launch_sync_probe(SolveCtrl* ctrl, double* partials, int iters, int mode, int nblocks,
                              unsigned long long limit_ns, double* out, cudaStream_t s) {
  void* args[] = {&ctrl, &partials, &iters, &mode, &limit_ns, &out};
  return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(sync_probe_kernel), dim3(nblocks), dim3(kBlock),
                                     args, 0, s);
}

}  // namespace cgk
