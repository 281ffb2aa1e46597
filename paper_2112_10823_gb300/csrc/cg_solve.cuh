// The CG solve body shared by the single-system and the batched kernels:
// the producer side (matrix stream) and the consumer side (the iteration)
// of one CTA's share of one system.
#pragma once
#include <cmath>
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
    atomicExch(&P.ctrl->phase, kPhaseDone);
  }
  __syncwarp();
  if (threadIdx.x == 0) *reinterpret_cast<volatile int32_t*>(sm.stop()) = 1;
}

// CTA sums each thread reads in the grid-wide sum: nblocks <= kMaxCtaSums * kConsumers.
constexpr int kMaxCtaSums = 2;

// Producer side of a solve task: stream the CTA's share of the matrix (FP32
// values in the mixed solve) pass after pass until the consumers stop it.
template <bool kMixed>
__device__ __forceinline__ void solve_producer(const RingSmem& sm, const CtaStream& cs, const SolveParams& P) {
  if (threadIdx.x == kConsumers) {
    bool ok;
    if constexpr (kMixed) ok = producer_loop<float>(sm, cs, P.A.val32, P.A.col_idx, -1, P.wait_limit_ns);
    else ok = producer_loop<double>(sm, cs, P.A.val, P.A.col_idx, -1, P.wait_limit_ns);
    if (!ok) {
      atomicExch(&P.ctrl->abort, 1);
      atomicExch(&P.ctrl->status, kETIMEOUT);
      atomicExch(&P.ctrl->phase, kPhaseDone);
    }
  }
  __syncwarp();
}

// Consumer side of a solve task: share `rank` (of P.group CTAs) of the CG
// iteration on one system, from its start or from the state a previous
// launch saved, for at most P.chunk_iters steps.
template <bool kMixed, bool kJacobi>
__device__ __forceinline__ void solve_consumers(const RingSmem& sm, const CtaStream& cs, const SolveParams& P,
                                                const int rank) {
  const DevCsr& A = P.A;
  const int tid = threadIdx.x;
  const unsigned long long lim = P.wait_limit_ns;
  const int row0 = A.block_row[rank], row1 = A.block_row[rank + 1];
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
  const double* __restrict__ dinv = P.dinv;  // Jacobi (kJacobi): z = dinv .* r; plain CG: z = r
  const int nb = P.group;
  ConsumerCursor cur;
  GridBarrier gb;
  gb.count = static_cast<unsigned int>(nb);
  int slot = 0;
  int site = 0;
  // state saved by an earlier launch of this solve (written by another
  // kernel, so read through L2)
  const int32_t phase0 = __ldcg(&ctrl->phase);
  if (phase0 == kPhaseRunning) {
    gb.target = __ldcg(&ctrl->rounds) * gb.count;
    slot = __ldcg(&ctrl->slot);
  }

  // Group-wide sums of one or two values per thread, identical in every CTA.
  // Each CTA sums its threads in fixed point, publishes the result, and after
  // a group barrier every CTA sums the nb CTA values, again in fixed point
  // (exact and order-independent, hence the same bits everywhere).  Two
  // slots of partials (2 nb values each) alternate so that a fast CTA
  // publishing the next sum never overwrites values a slow CTA is still
  // reading.
  auto group_sum = [&](const double* part) -> double {
    double mine[kMaxCtaSums];
#pragma unroll
    for (int j = 0; j < kMaxCtaSums; ++j) {
      const int c = tid + j * kConsumers;
      mine[j] = c < nb ? __ldcg(part + c) : 0.0;
    }
    return fx_block_sum<kMaxCtaSums>(mine, fx);
  };
  auto allreduce = [&](double v, double& out) -> bool {
    const double cta = fx_block_sum(v, fx);
    if (nb == 1) {  // a one-CTA group: the CTA sum is the sum
      out = cta;
      return true;
    }
    double* part = P.partials + static_cast<size_t>(slot) * 2 * nb;
    if (tid == 0) part[rank] = cta;
    if (!gb.sync(ctrl, lim, ++site, flag)) return false;
    out = group_sum(part);
    slot ^= 1;
    return true;
  };
  auto allreduce2 = [&](double v1, double v2, double& o1, double& o2) -> bool {
    const double c1 = fx_block_sum(v1, fx);
    const double c2 = fx_block_sum(v2, fx);
    if (nb == 1) {
      o1 = c1;
      o2 = c2;
      return true;
    }
    double* part = P.partials + static_cast<size_t>(slot) * 2 * nb;
    if (tid == 0) {
      part[rank] = c1;
      part[nb + rank] = c2;
    }
    if (!gb.sync(ctrl, lim, ++site, flag)) return false;
    o1 = group_sum(part);
    o2 = group_sum(part + nb);
    slot ^= 1;
    return true;
  };
  // r.r and (Jacobi) r.z of per-thread partials: one sum without a
  // preconditioner (r.z = r.r), both in one group barrier with one
  auto sums_rr_rz = [&](double acc_rr, double acc_rz, double& rr, double& rz) -> bool {
    if constexpr (kJacobi) {
      return allreduce2(acc_rr, acc_rz, rr, rz);
    } else {
      if (!allreduce(acc_rr, rr)) return false;
      rz = rr;
      return true;
    }
  };
  // The products outside the step loop (setup, true residual at the end,
  // and the mixed solve's residual replacements) read the FP64 values and
  // columns directly from global memory with a compact per-lane loop: they
  // run once per solve (or once every replace_every steps), and keeping the
  // large unrolled ring product out of them leaves its single copy, in the
  // step loop, the registers it needs.  The ring keeps streaming the values
  // the step loop uses.  Every product pass ends with a vote of all consumer
  // warps, so that a warp that gave up on a wait and the others leave
  // together.
  auto product64 = [&](const double* xin, const double* aux, auto& epi) -> bool {
    const bool ok = spmv_pass<false, double, double, double>(sm, cs, cur, A, A.val, xin, aux, epi, lim);
    return cta_and(ok);
  };

  // rho = r.z (the preconditioned inner product; r.r without a
  // preconditioner), rr = r.r (the stopping test always uses ||r||)
  double rho, bnorm2, rr;
  int64_t k = 0;
  if (phase0 == kPhaseRunning) {
    rho = __ldcg(&ctrl->rho);
    bnorm2 = __ldcg(&ctrl->bnorm2);
    k = __ldcg(&ctrl->iters);
    rr = __ldcg(&ctrl->relres_rec);
    rr = rr * rr * bnorm2;
  } else {
    // ---- setup: r = b - A x, z = dinv .* r, p = z, rho = r.z, ||b||^2
    double acc_rr = 0.0, acc_bb = 0.0, acc_rz = 0.0;
    auto epi = [&](int i, double s, double bi) {
      const double ri = bi - s;
      double zi = ri;
      if constexpr (kJacobi) zi = dinv[i] * ri;
      r[i] = ri;
      p[i] = zi;
      if constexpr (kMixed) p32[i] = static_cast<float>(zi);
      acc_rr = fma(ri, ri, acc_rr);
      if constexpr (kJacobi) acc_rz = fma(ri, zi, acc_rz);
      acc_bb = fma(bi, bi, acc_bb);
    };
    if (!product64(x, b, epi)) { solve_fail(sm, P); return; }
    if (!sums_rr_rz(acc_rr, acc_rz, rr, rho) || !allreduce(acc_bb, bnorm2)) { solve_fail(sm, P); return; }
  }
  if (bnorm2 == 0.0) {  // b = 0: the solution is 0
    for (int i = row0 + tid; i < row1; i += kConsumers) x[i] = 0.0;
    if (rank == 0 && tid == 0) {
      ctrl->status = kOK;
      ctrl->iters = 0;
      ctrl->rho = 0.0;
      ctrl->bnorm2 = 0.0;
      ctrl->relres_rec = 0.0;
      ctrl->relres_true = 0.0;
      ctrl->phase = kPhaseDone;
    }
    consumers_done(sm);
    return;
  }
  // Stopping test sqrt(rho) <= tol ||b|| evaluated as rho <= tol^2 ||b||^2
  // (no square root on the critical path; the same test up to rounding).
  const double thresh2 = (P.tol * P.tol) * bnorm2;
  const int64_t k_end = P.chunk_iters > 0 && P.chunk_iters < P.maxit - k ? k + P.chunk_iters : P.maxit;
  int32_t status = kOK;
  bool done = phase0 != kPhaseRunning && rr <= thresh2;

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

    // ---- r -= alpha q, rr' = r.r, rho' = r.z   (four rows per thread in flight)
    double acc_r = 0.0, acc_z = 0.0;
    {
      constexpr bool jac = kJacobi;
      for (int base = row0 + tid; base < row1; base += 4 * kConsumers) {
        double qv[4], rv[4], dv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = base + u * kConsumers;
          if (i < row1) {
            qv[u] = q[i];
            rv[u] = r[i];
            if constexpr (jac) dv[u] = dinv[i];
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = base + u * kConsumers;
          if (i < row1) {
            const double rn = fma(-alpha, qv[u], rv[u]);
            r[i] = rn;
            acc_r = fma(rn, rn, acc_r);
            if constexpr (jac) acc_z = fma(rn, dv[u] * rn, acc_z);
          }
        }
      }
    }
    double rho_new;
    if (!sums_rr_rz(acc_r, acc_z, rr, rho_new)) { solve_fail(sm, P); return; }
    ++k;

    bool replace = false;
    if constexpr (kMixed) replace = (P.replace_every > 0 && k % P.replace_every == 0) || rr <= thresh2;
    if (replace) {
      // x += alpha p, then r = b - A x in FP64 (residual replacement).  The
      // direction keeps the recurrence's beta = rho_rec / rho (rho_rec: the
      // recursive r.z of this step); r, rr and rho take the true residual's
      // values.
      if (tid == 0) sc[1] = rho_new / rho;
      for (int i = row0 + tid; i < row1; i += kConsumers) x[i] = fma(alpha, p[i], x[i]);
      if (!gb.sync(ctrl, lim, ++site, flag)) { solve_fail(sm, P); return; }
      const double beta = sc[1];
      double acc_t = 0.0, acc_tz = 0.0;
      auto epi = [&](int i, double s, double bi) {
        const double ri = bi - s;
        r[i] = ri;
        acc_t = fma(ri, ri, acc_t);
        if constexpr (kJacobi) acc_tz = fma(ri, dinv[i] * ri, acc_tz);
      };
      if (!product64(x, b, epi) || !sums_rr_rz(acc_t, acc_tz, rr, rho_new)) { solve_fail(sm, P); return; }
      if (rr <= thresh2) {
        rho = rho_new;
        done = true;
        break;
      }
      for (int i = row0 + tid; i < row1; i += kConsumers) {
        double zi = r[i];
        if constexpr (kJacobi) zi = dinv[i] * zi;
        const double pi = fma(beta, p[i], zi);
        p[i] = pi;
        if constexpr (kMixed) p32[i] = static_cast<float>(pi);
      }
      rho = rho_new;
    } else {
      if (!kMixed && rr <= thresh2) {
        for (int i = row0 + tid; i < row1; i += kConsumers) x[i] = fma(alpha, p[i], x[i]);
        rho = rho_new;
        done = true;
        break;
      }
      // ---- x += alpha p; p = z + beta p   (z = dinv .* r, or r)
      if (tid == 0) sc[1] = rho_new / rho;
      cta_sync();
      const double beta = sc[1];
      for (int base = row0 + tid; base < row1; base += 4 * kConsumers) {
        double pv[4], rv[4], xv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = base + u * kConsumers;
          if (i < row1) {
            pv[u] = p[i];
            rv[u] = r[i];
            if constexpr (kJacobi) rv[u] = dinv[i] * rv[u];
            xv[u] = x[i];
          }
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
    if (k >= k_end && k < P.maxit) {
      // end of this launch's share of the solve: save the state (identical
      // in every CTA of the group; x, r, p are complete after the barrier)
      if (rank == 0 && tid == 0) {
        ctrl->iters = k;
        ctrl->rho = rho;
        ctrl->bnorm2 = bnorm2;
        ctrl->relres_rec = sqrt(rr / bnorm2);
        ctrl->rounds = gb.target / gb.count;
        ctrl->slot = slot;
        ctrl->phase = kPhaseRunning;
      }
      consumers_done(sm);
      return;
    }
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
  if (rank == 0 && tid == 0) {
    ctrl->status = status;
    ctrl->iters = k;
    ctrl->rho = rho;
    ctrl->bnorm2 = bnorm2;
    ctrl->relres_rec = sqrt(rr / bnorm2);
    ctrl->relres_true = sqrt(acc_t / bnorm2);
    ctrl->phase = kPhaseDone;
  }
  consumers_done(sm);
}

}  // namespace cgk
