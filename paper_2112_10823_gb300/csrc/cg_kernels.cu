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

// Leave the kernel after a failed wait: drain in-flight copies, record status.
__device__ __forceinline__ void solve_fail(const SpmvSmem& sm, StagePipe& pp, const SolveParams& P) {
  stage_drain(sm, pp, P.wait_limit_ns);
  if (threadIdx.x == 0) {
    atomicExch(&P.ctrl->abort, 1);
    atomicExch(&P.ctrl->status, kETIMEOUT);
  }
}

template <bool kMixed>
__global__ void __launch_bounds__(kBlock, 1) cg_solve_kernel(const SolveParams P) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const SpmvSmem sm{smem_raw};
  const DevCsr& A = P.A;
  const int bid = blockIdx.x;
  const int c0 = A.block_chunk[bid], c1 = A.block_chunk[bid + 1];
  const int row0 = A.chunk_row[c0], row1 = A.chunk_row[c1];
  const unsigned long long lim = P.wait_limit_ns;
  double* red = sm.red();
  int32_t* flag = sm.flag();
  SolveCtrl* ctrl = P.ctrl;
  const double* __restrict__ b = P.b;
  double* __restrict__ x = P.x;
  double* __restrict__ r = P.r;
  double* __restrict__ p = P.p;
  double* __restrict__ q = P.q;
  float* __restrict__ p32 = P.p32;
  const int nb = gridDim.x;

  stage_init(sm);
  StagePipe pp;
  GridBarrier gb;
  int slot = 0;
  int site = 0;

  // Grid-wide sum of one or two per-thread values, identical in every CTA:
  // CTA partials go to partials[slot], a barrier, then every CTA adds the nb
  // partials in block order.  Two slots alternate so that a fast CTA writing
  // the next partials never overwrites ones a slow CTA is still reading.
  auto allreduce2 = [&](double& v0, double& v1) -> bool {
    block_sum2(v0, v1, red);
    double* part = P.partials + static_cast<size_t>(slot) * nb * 2;
    if (threadIdx.x == 0) {
      part[2 * bid] = v0;
      part[2 * bid + 1] = v1;
    }
    if (!gb.sync(ctrl, lim, ++site, flag)) return false;
    double s0 = 0.0, s1 = 0.0;
    for (int j = threadIdx.x; j < nb; j += kBlock) {
      s0 += __ldcg(part + 2 * j);
      s1 += __ldcg(part + 2 * j + 1);
    }
    block_sum2(s0, s1, red);
    v0 = s0;
    v1 = s1;
    slot ^= 1;
    return true;
  };
  auto allreduce = [&](double& v) -> bool {
    double dummy = 0.0;
    return allreduce2(v, dummy);
  };

  // ---- setup: r = b - A x, p = r, rho = r.r, ||b||^2
  double acc_rr = 0.0, acc_bb = 0.0;
  {
    auto epi = [&](int i, double s) {
      const double bi = b[i];
      const double ri = bi - s;
      r[i] = ri;
      p[i] = ri;
      if constexpr (kMixed) p32[i] = static_cast<float>(ri);
      acc_rr = fma(ri, ri, acc_rr);
      acc_bb = fma(bi, bi, acc_bb);
    };
    if (!spmv_pass<double, double, double>(sm, pp, A, A.val, c0, c1, x, epi, lim)) {
      solve_fail(sm, pp, P);
      return;
    }
  }
  if (!allreduce2(acc_rr, acc_bb)) { solve_fail(sm, pp, P); return; }
  double rho = acc_rr;
  const double bnorm2 = acc_bb;
  const double bnorm = sqrt(bnorm2);
  if (bnorm2 == 0.0) {  // b = 0: the solution is 0
    for (int i = row0 + threadIdx.x; i < row1; i += kBlock) x[i] = 0.0;
    if (bid == 0 && threadIdx.x == 0) {
      ctrl->status = kOK;
      ctrl->iters = 0;
      ctrl->rho = 0.0;
      ctrl->bnorm2 = 0.0;
      ctrl->relres_rec = 0.0;
      ctrl->relres_true = 0.0;
    }
    return;
  }
  const double thresh = P.tol * bnorm;
  int64_t k = 0;
  int32_t status = kOK;
  bool done = sqrt(rho) <= thresh;

  while (!done && k < P.maxit) {
    // ---- q = A p, gamma = p.q
    double acc_g = 0.0;
    bool ok;
    if constexpr (kMixed) {
      auto epi = [&](int i, float s) {
        const double qi = static_cast<double>(s);
        q[i] = qi;
        acc_g = fma(p[i], qi, acc_g);
      };
      ok = spmv_pass<float, float, float>(sm, pp, A, A.val32, c0, c1, p32, epi, lim);
    } else {
      auto epi = [&](int i, double s) {
        q[i] = s;
        acc_g = fma(p[i], s, acc_g);
      };
      ok = spmv_pass<double, double, double>(sm, pp, A, A.val, c0, c1, p, epi, lim);
    }
    if (!ok || !allreduce(acc_g)) { solve_fail(sm, pp, P); return; }
    const double gamma = acc_g;
    if (!(gamma > 0.0) || !isfinite(gamma)) {  // not SPD, or overflow
      status = kEBREAKDOWN;
      break;
    }
    const double alpha = rho / gamma;

    // ---- r -= alpha q, rho' = r.r
    double acc_r = 0.0;
    for (int i = row0 + threadIdx.x; i < row1; i += kBlock) {
      const double ri = fma(-alpha, q[i], r[i]);
      r[i] = ri;
      acc_r = fma(ri, ri, acc_r);
    }
    if (!allreduce(acc_r)) { solve_fail(sm, pp, P); return; }
    double rho_new = acc_r;
    ++k;

    bool replace = false;
    if constexpr (kMixed)
      replace = (P.replace_every > 0 && k % P.replace_every == 0) || sqrt(rho_new) <= thresh;
    if (replace) {
      // x += alpha p, then r = b - A x in FP64 (residual replacement)
      for (int i = row0 + threadIdx.x; i < row1; i += kBlock) x[i] = fma(alpha, p[i], x[i]);
      if (!gb.sync(ctrl, lim, ++site, flag)) { solve_fail(sm, pp, P); return; }
      double acc_t = 0.0;
      auto epi = [&](int i, double s) {
        const double ri = b[i] - s;
        r[i] = ri;
        acc_t = fma(ri, ri, acc_t);
      };
      if (!spmv_pass<double, double, double>(sm, pp, A, A.val, c0, c1, x, epi, lim) || !allreduce(acc_t)) {
        solve_fail(sm, pp, P);
        return;
      }
      rho_new = acc_t;
      if (sqrt(rho_new) <= thresh) {
        rho = rho_new;
        done = true;
        break;
      }
      const double beta = rho_new / rho;
      for (int i = row0 + threadIdx.x; i < row1; i += kBlock) {
        const double pi = fma(beta, p[i], r[i]);
        p[i] = pi;
        if constexpr (kMixed) p32[i] = static_cast<float>(pi);
      }
      rho = rho_new;
    } else {
      if (!kMixed && sqrt(rho_new) <= thresh) {
        for (int i = row0 + threadIdx.x; i < row1; i += kBlock) x[i] = fma(alpha, p[i], x[i]);
        rho = rho_new;
        done = true;
        break;
      }
      // ---- x += alpha p; p = r + beta p
      const double beta = rho_new / rho;
      for (int i = row0 + threadIdx.x; i < row1; i += kBlock) {
        const double pi = p[i];
        x[i] = fma(alpha, pi, x[i]);
        const double pn = fma(beta, pi, r[i]);
        p[i] = pn;
        if constexpr (kMixed) p32[i] = static_cast<float>(pn);
      }
      rho = rho_new;
    }
    if (!gb.sync(ctrl, lim, ++site, flag)) { solve_fail(sm, pp, P); return; }
  }
  if (status == kOK && !done) status = kENOTCONV;

  // ---- true residual ||b - A x|| / ||b|| (x complete everywhere first)
  if (!gb.sync(ctrl, lim, ++site, flag)) { solve_fail(sm, pp, P); return; }
  double acc_t = 0.0;
  {
    auto epi = [&](int i, double s) {
      const double d = b[i] - s;
      acc_t = fma(d, d, acc_t);
    };
    if (!spmv_pass<double, double, double>(sm, pp, A, A.val, c0, c1, x, epi, lim) || !allreduce(acc_t)) {
      solve_fail(sm, pp, P);
      return;
    }
  }
  if (bid == 0 && threadIdx.x == 0) {
    ctrl->status = status;
    ctrl->iters = k;
    ctrl->rho = rho;
    ctrl->bnorm2 = bnorm2;
    ctrl->relres_rec = sqrt(rho) / bnorm;
    ctrl->relres_true = sqrt(acc_t) / bnorm;
  }
}

// y = A x over the CTA's chunk range (same partition and staging as the solve).
__global__ void __launch_bounds__(kBlock, 1) spmv_kernel(const DevCsr A, const double* __restrict__ x,
                                                          double* __restrict__ y, int32_t* err) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const SpmvSmem sm{smem_raw};
  stage_init(sm);
  StagePipe pp;
  const int c0 = A.block_chunk[blockIdx.x], c1 = A.block_chunk[blockIdx.x + 1];
  auto epi = [&](int i, double s) { y[i] = s; };
  if (!spmv_pass<double, double, double>(sm, pp, A, A.val, c0, c1, x, epi, 2000000000ull)) {
    stage_drain(sm, pp, 2000000000ull);
    if (threadIdx.x == 0) atomicExch(err, kETIMEOUT);
  }
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
  cudaError_t e = ensure_smem_attr(reinterpret_cast<const void*>(spmv_kernel), SpmvSmem::kBytes);
  if (e != cudaSuccess) return e;
  spmv_kernel<<<A.nblocks, kBlock, SpmvSmem::kBytes, s>>>(A, x, y, err);
  return cudaGetLastError();
}

size_t spmv_smem_bytes() { return SpmvSmem::kBytes; }

int solve_blocks_per_sm(bool mixed) {
  int nb = 0;
  cudaError_t e;
  if (mixed) {
    e = ensure_smem_attr(reinterpret_cast<const void*>(cg_solve_kernel<true>), SpmvSmem::kBytes);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, cg_solve_kernel<true>, kBlock, SpmvSmem::kBytes);
  } else {
    e = ensure_smem_attr(reinterpret_cast<const void*>(cg_solve_kernel<false>), SpmvSmem::kBytes);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, cg_solve_kernel<false>, kBlock, SpmvSmem::kBytes);
  }
  return e == cudaSuccess ? nb : -1;
}

cudaError_t launch_solve(const SolveParams& P, bool mixed, cudaStream_t s) {
  void* args[] = {const_cast<SolveParams*>(&P)};
  if (mixed) {
    cudaError_t e = ensure_smem_attr(reinterpret_cast<const void*>(cg_solve_kernel<true>), SpmvSmem::kBytes);
    if (e != cudaSuccess) return e;
    return cudaLaunchCooperativeKernel(reinterpret_cast<void*>(cg_solve_kernel<true>), dim3(P.A.nblocks),
                                       dim3(kBlock), args, SpmvSmem::kBytes, s);
  }
  cudaError_t e = ensure_smem_attr(reinterpret_cast<const void*>(cg_solve_kernel<false>), SpmvSmem::kBytes);
  if (e != cudaSuccess) return e;
  return cudaLaunchCooperativeKernel(reinterpret_cast<void*>(cg_solve_kernel<false>), dim3(P.A.nblocks),
                                     dim3(kBlock), args, SpmvSmem::kBytes, s);
}

// ---- self-test of the bounded wait: one CTA waits at a grid barrier that
// expects one more arrival than the grid can give, so the wait must run out
// after limit_ns and report kETIMEOUT through the control block.
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
  wait_timeout_selftest_kernel<<<1, 32, 0, s>>>(ctrl, limit_ns);
  return cudaGetLastError();
}

}  // namespace cgk
