// CSR product and the persistent conjugate-gradient solve.
//
// Classical CG (the paper's Sec. 5.3 solver; no preconditioner), one
// cooperative launch per solve:
//   setup     r = b - A x, p = r, rho = r.r, ||b||^2          (product + 2 sums)
//   each step q = A p, gamma = p.q                            (product fused with the sum)
//             alpha = rho/gamma; r -= alpha q, rho' = r.r     (update fused with the sum)
//             stop if sqrt(rho') <= tol ||b||
//             beta = rho'/rho; x += alpha p; p = r + beta p   (x update deferred here)
//   exit      ||b - A x|| / ||b||                             (true residual)
// alpha, beta and the stopping test are computed on the device by every CTA
// from the same deterministic sums, so no host synchronisation happens per
// step and every CTA takes the same branch.  Each CTA owns a fixed range of
// rows (a run of product chunks) for all phases, so only the two sums and the
// gather of p need grid-wide synchronisation: three grid barriers per step.
//
// The mixed-precision variant keeps an FP32 copy of the values and an FP32
// shadow of p: the product is FP32 (FP32 accumulation); sums, alpha, beta, x
// and r stay FP64; every `replace_every` steps, and before accepting
// convergence, r is replaced by the FP64 true residual b - A x.
#include <cmath>
#include <mutex>
#include <set>
#include <utility>
#include "cg_device.cuh"

namespace cgk {

// Consumers leaving the kernel: tell the producer to stop (it then waits for
// its copies in flight and exits).
__device__ __forceinline__ void consumers_done(const RingSmem& sm) {
  cta_sync();
  if (threadIdx.x == 0) *reinterpret_cast<volatile int32_t*>(sm.stop()) = 1;
}

// Leave the kernel after a failed wait: record the status, stop the producer.
__device__ __forceinline__ void solve_fail(const RingSmem& sm, const SolveParams& P) {
  if (threadIdx.x == 0) {
    atomicExch(&P.ctrl->abort, 1);
    atomicExch(&P.ctrl->status, kETIMEOUT);
  }
  __syncwarp();
  if (threadIdx.x == 0) *reinterpret_cast<volatile int32_t*>(sm.stop()) = 1;
}

// CTA sums each thread reads in the grid-wide sum: nblocks <= kMaxCtaSums * kConsumers.
constexpr int kMaxCtaSums = 2;

template <bool kMixed>
__global__ void __launch_bounds__(kBlock, kCtasPerSm) cg_solve_kernel(const SolveParams P) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const RingSmem sm{smem_raw};
  const DevCsr& A = P.A;
  const int bid = blockIdx.x;
  const int tid = threadIdx.x;
  const unsigned long long lim = P.wait_limit_ns;
  CtaStream cs;
  stream_setup(sm, cs, A);  // the last barrier of all threads
  if (tid >= kConsumers) {  // the producer warp
    if (tid == kConsumers) {
      bool ok;
      if constexpr (kMixed) ok = producer_loop<float>(sm, cs, A.val32, A.col_idx, -1, lim);
      else ok = producer_loop<double>(sm, cs, A.val, A.col_idx, -1, lim);
      if (!ok) {
        atomicExch(&P.ctrl->abort, 1);
        atomicExch(&P.ctrl->status, kETIMEOUT);
      }
    }
    return;
  }
  const int row0 = A.block_row[bid], row1 = A.block_row[bid + 1];
  int32_t* flag = sm.flag();
  double* sc = sm.scalars();  // broadcast slots for per-step scalars
  FxScratch* fx = sm.fx();
  SolveCtrl* ctrl = P.ctrl;
  const double* __restrict__ b = P.b;
  double* __restrict__ x = P.x;
  double* __restrict__ r = P.r;
  double* __restrict__ p = P.p;
  double* __restrict__ q = P.q;
  float* __restrict__ p32 = P.p32;
  const int nb = gridDim.x;
  ConsumerCursor cur;
  GridBarrier gb;
  int slot = 0;
  int site = 0;

  // Grid-wide sum of one value per thread, identical in every CTA.  Each CTA
  // sums its threads in fixed point, publishes the result, and after a grid
  // barrier every CTA sums the nb CTA values, again in fixed point (exact and
  // order-independent, hence the same bits everywhere).  Two slots of
  // partials alternate so that a fast CTA publishing the next sum never
  // overwrites values a slow CTA is still reading.
  auto allreduce = [&](double v, double& out) -> bool {
    const double cta = fx_block_sum(v, fx);
    double* part = P.partials + static_cast<size_t>(slot) * nb;
    if (tid == 0) part[bid] = cta;
    if (!gb.sync(ctrl, lim, ++site, flag)) return false;
    double mine[kMaxCtaSums];
#pragma unroll
    for (int j = 0; j < kMaxCtaSums; ++j) {
      const int c = tid + j * kConsumers;
      mine[j] = c < nb ? __ldcg(part + c) : 0.0;
    }
    out = fx_block_sum<kMaxCtaSums>(mine, fx);
    slot ^= 1;
    return true;
  };
  // FP64 products: from the ring in the FP64 solve; read directly from
  // global memory in the mixed solve (whose ring carries the FP32 values).
  // Every product pass ends with a vote of all consumer warps, so that a warp
  // that gave up on a wait and the others leave together.
  auto product64 = [&](const double* xin, const double* aux, auto& epi) -> bool {
    bool ok;
    if constexpr (kMixed) ok = spmv_pass<false, double, double, double>(sm, cs, cur, A, A.val, xin, aux, epi, lim);
    else ok = spmv_pass<true, double, double, double>(sm, cs, cur, A, A.val, xin, aux, epi, lim);
    return cta_and(ok);
  };

  // ---- setup: r = b - A x, p = r, rho = r.r, ||b||^2
  double acc_rr = 0.0, acc_bb = 0.0;
  {
    auto epi = [&](int i, double s, double bi) {
      const double ri = bi - s;
      r[i] = ri;
      p[i] = ri;
      if constexpr (kMixed) p32[i] = static_cast<float>(ri);
      acc_rr = fma(ri, ri, acc_rr);
      acc_bb = fma(bi, bi, acc_bb);
    };
    if (!product64(x, b, epi)) { solve_fail(sm, P); return; }
  }
  double rho, bnorm2;
  if (!allreduce(acc_rr, rho) || !allreduce(acc_bb, bnorm2)) { solve_fail(sm, P); return; }
  if (bnorm2 == 0.0) {  // b = 0: the solution is 0
    for (int i = row0 + tid; i < row1; i += kConsumers) x[i] = 0.0;
    if (bid == 0 && tid == 0) {
      ctrl->status = kOK;
      ctrl->iters = 0;
      ctrl->rho = 0.0;
      ctrl->bnorm2 = 0.0;
      ctrl->relres_rec = 0.0;
      ctrl->relres_true = 0.0;
    }
    consumers_done(sm);
    return;
  }
  // Stopping test sqrt(rho) <= tol ||b|| evaluated as rho <= tol^2 ||b||^2
  // (no square root on the critical path; the same test up to rounding).
  const double thresh2 = (P.tol * P.tol) * bnorm2;
  int64_t k = 0;
  int32_t status = kOK;
  bool done = rho <= thresh2;

  while (!done && k < P.maxit) {
    // ---- q = A p, gamma = p.q
    double acc_g = 0.0;
    bool ok;
    if constexpr (kMixed) {
      auto epi = [&](int i, float s, double pi) {
        const double qi = static_cast<double>(s);
        q[i] = qi;
        acc_g = fma(pi, qi, acc_g);
      };
      ok = cta_and(spmv_pass<true, float, float, float>(sm, cs, cur, A, A.val32, p32, p, epi, lim));
    } else {
      auto epi = [&](int i, double s, double pi) {
        q[i] = s;
        acc_g = fma(pi, s, acc_g);
      };
      ok = cta_and(spmv_pass<true, double, double, double>(sm, cs, cur, A, A.val, p, p, epi, lim));
    }
    double gamma;
    if (!ok || !allreduce(acc_g, gamma)) { solve_fail(sm, P); return; }
    if (!(gamma > 0.0) || !isfinite(gamma)) {  // not SPD, or overflow
      status = kEBREAKDOWN;
      break;
    }
    // alpha = rho / gamma, computed once and broadcast (FP64 division is slow)
    if (tid == 0) sc[0] = rho / gamma;
    cta_sync();
    const double alpha = sc[0];

    // ---- r -= alpha q, rho' = r.r   (four rows per thread in flight)
    double acc_r = 0.0;
    for (int base = row0 + tid; base < row1; base += 4 * kConsumers) {
      double qv[4], rv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = base + u * kConsumers;
        if (i < row1) { qv[u] = q[i]; rv[u] = r[i]; }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = base + u * kConsumers;
        if (i < row1) {
          const double rn = fma(-alpha, qv[u], rv[u]);
          r[i] = rn;
          acc_r = fma(rn, rn, acc_r);
        }
      }
    }
    double rho_new;
    if (!allreduce(acc_r, rho_new)) { solve_fail(sm, P); return; }
    ++k;

    bool replace = false;
    if constexpr (kMixed) replace = (P.replace_every > 0 && k % P.replace_every == 0) || rho_new <= thresh2;
    if (replace) {
      // x += alpha p, then r = b - A x in FP64 (residual replacement)
      for (int i = row0 + tid; i < row1; i += kConsumers) x[i] = fma(alpha, p[i], x[i]);
      if (!gb.sync(ctrl, lim, ++site, flag)) { solve_fail(sm, P); return; }
      double acc_t = 0.0;
      auto epi = [&](int i, double s, double bi) {
        const double ri = bi - s;
        r[i] = ri;
        acc_t = fma(ri, ri, acc_t);
      };
      if (!product64(x, b, epi) || !allreduce(acc_t, rho_new)) { solve_fail(sm, P); return; }
      if (rho_new <= thresh2) {
        rho = rho_new;
        done = true;
        break;
      }
      if (tid == 0) sc[1] = rho_new / rho;
      cta_sync();
      const double beta = sc[1];
      for (int i = row0 + tid; i < row1; i += kConsumers) {
        const double pi = fma(beta, p[i], r[i]);
        p[i] = pi;
        if constexpr (kMixed) p32[i] = static_cast<float>(pi);
      }
      rho = rho_new;
    } else {
      if (!kMixed && rho_new <= thresh2) {
        for (int i = row0 + tid; i < row1; i += kConsumers) x[i] = fma(alpha, p[i], x[i]);
        rho = rho_new;
        done = true;
        break;
      }
      // ---- x += alpha p; p = r + beta p
      if (tid == 0) sc[1] = rho_new / rho;
      cta_sync();
      const double beta = sc[1];
      for (int base = row0 + tid; base < row1; base += 4 * kConsumers) {
        double pv[4], rv[4], xv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = base + u * kConsumers;
          if (i < row1) { pv[u] = p[i]; rv[u] = r[i]; xv[u] = x[i]; }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = base + u * kConsumers;
          if (i < row1) {
            x[i] = fma(alpha, pv[u], xv[u]);
            const double pn = fma(beta, pv[u], rv[u]);
            p[i] = pn;
            if constexpr (kMixed) p32[i] = static_cast<float>(pn);
          }
        }
      }
      rho = rho_new;
    }
    if (!gb.sync(ctrl, lim, ++site, flag)) { solve_fail(sm, P); return; }
  }
  if (status == kOK && !done) status = kENOTCONV;

  // ---- true residual ||b - A x|| / ||b|| (x complete everywhere first)
  if (!gb.sync(ctrl, lim, ++site, flag)) { solve_fail(sm, P); return; }
  double acc_t = 0.0;
  {
    auto epi = [&](int i, double s, double bi) {
      const double d = bi - s;
      acc_t = fma(d, d, acc_t);
    };
    double tsum;
    if (!product64(x, b, epi) || !allreduce(acc_t, tsum)) { solve_fail(sm, P); return; }
    acc_t = tsum;
  }
  if (bid == 0 && tid == 0) {
    ctrl->status = status;
    ctrl->iters = k;
    ctrl->rho = rho;
    ctrl->bnorm2 = bnorm2;
    ctrl->relres_rec = sqrt(rho / bnorm2);
    ctrl->relres_true = sqrt(acc_t / bnorm2);
  }
  consumers_done(sm);
}

// y = A x (same partition and stream as the solve; one pass).
__global__ void __launch_bounds__(kBlock, kCtasPerSm) spmv_kernel(const DevCsr A, const double* __restrict__ x,
                                                                   double* __restrict__ y, int32_t* err) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const RingSmem sm{smem_raw};
  CtaStream cs;
  stream_setup(sm, cs, A);
  const unsigned long long lim = 2000000000ull;
  if (threadIdx.x >= kConsumers) {
    if (threadIdx.x == kConsumers && !producer_loop<double>(sm, cs, A.val, A.col_idx, 1, lim)) atomicExch(err, kETIMEOUT);
    return;
  }
  ConsumerCursor cur;
  auto epi = [&](int i, double s, double) { y[i] = s; };
  const bool ok = cta_and(spmv_pass<true, double, double, double>(sm, cs, cur, A, A.val, x, nullptr, epi, lim));
  if (!ok && threadIdx.x == 0) atomicExch(err, kETIMEOUT);
  consumers_done(sm);
}

namespace {
// Opt a kernel in to the large dynamic shared memory, once per (kernel, device).
cudaError_t ensure_smem_attr(const void* kernel, size_t bytes) {
  static std::mutex mu;
  static std::set<std::pair<const void*, int>> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  if (done.count({kernel, dev})) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(bytes));
  if (e == cudaSuccess) done.insert({kernel, dev});
  return e;
}
}  // namespace

cudaError_t launch_spmv(const DevCsr& A, const double* x, double* y, int32_t* err, cudaStream_t s) {
  cudaError_t e = ensure_smem_attr(reinterpret_cast<const void*>(spmv_kernel), RingSmem::kBytes);
  if (e != cudaSuccess) return e;
  spmv_kernel<<<A.nblocks, kBlock, RingSmem::kBytes, s>>>(A, x, y, err);
  return cudaGetLastError();
}

size_t spmv_smem_bytes() { return RingSmem::kBytes; }

int solve_blocks_per_sm(bool mixed) {
  int nb = 0;
  cudaError_t e;
  if (mixed) {
    e = ensure_smem_attr(reinterpret_cast<const void*>(cg_solve_kernel<true>), RingSmem::kBytes);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, cg_solve_kernel<true>, kBlock, RingSmem::kBytes);
  } else {
    e = ensure_smem_attr(reinterpret_cast<const void*>(cg_solve_kernel<false>), RingSmem::kBytes);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, cg_solve_kernel<false>, kBlock, RingSmem::kBytes);
  }
  return e == cudaSuccess ? nb : -1;
}

cudaError_t launch_solve(const SolveParams& P, bool mixed, cudaStream_t s) {
  void* args[] = {const_cast<SolveParams*>(&P)};
  if (mixed) {
    cudaError_t e = ensure_smem_attr(reinterpret_cast<const void*>(cg_solve_kernel<true>), RingSmem::kBytes);
    if (e != cudaSuccess) return e;
    return cudaLaunchCooperativeKernel(reinterpret_cast<void*>(cg_solve_kernel<true>), dim3(P.A.nblocks),
                                       dim3(kBlock), args, RingSmem::kBytes, s);
  }
  cudaError_t e = ensure_smem_attr(reinterpret_cast<const void*>(cg_solve_kernel<false>), RingSmem::kBytes);
  if (e != cudaSuccess) return e;
  return cudaLaunchCooperativeKernel(reinterpret_cast<void*>(cg_solve_kernel<false>), dim3(P.A.nblocks),
                                     dim3(kBlock), args, RingSmem::kBytes, s);
}

// ---- self-test of the bounded wait: one CTA (of kConsumers threads, the
// grid barrier's CTA size) waits at a grid barrier that expects one more
// arrival than the grid can give, so the wait must run out after limit_ns and
// report kETIMEOUT through the control block.
__global__ void wait_timeout_selftest_kernel(SolveCtrl* ctrl, unsigned long long limit_ns) {
  __shared__ int32_t flag;
  GridBarrier gb;
  gb.target = 1;  // the barrier below now waits for 2 arrivals; only 1 CTA exists
  if (!gb.sync(ctrl, limit_ns, 99, &flag)) {
    if (threadIdx.x == 0) ctrl->status = kETIMEOUT;
  } else if (threadIdx.x == 0) {
    ctrl->status = kOK;
  }
}

cudaError_t launch_wait_timeout_selftest(SolveCtrl* ctrl, unsigned long long limit_ns, cudaStream_t s) {
  wait_timeout_selftest_kernel<<<1, kConsumers, 0, s>>>(ctrl, limit_ns);
  return cudaGetLastError();
}

}  // namespace cgk
