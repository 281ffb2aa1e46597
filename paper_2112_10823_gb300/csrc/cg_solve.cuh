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

// Systems whose CTAs hold at most kLocalRows rows each (small, L2-resident
// shares), solved in one launch, use the small-share kernels: r of the CTA's
// rows lives in shared memory (only the owning CTA ever reads it; three
// accesses per step), and x is updated behind the barrier of the r.r sum,
// where the wait is longer than the update.  Larger shares keep r in global
// memory and update x together with p (one pass over p).  Both compute the
// same bits.

// Rows per thread in flight in the vector phases (all loads of a batch
// issued before any is used): as many as the registers that the product
// leaves allow without spilling (128 per thread at 16 warps per CTA; the
// Jacobi variants carry dinv as well, the fused x and p update three vectors).
template <bool kJacobi, bool kSmallShare>
__host__ __device__ constexpr int vec_rows() {
  return kSmallShare ? (kJacobi ? 3 : 4) : (kJacobi ? 2 : 3);
}

// Consumer side of a solve task: share `rank` (of P.group CTAs) of the CG
// iteration on one system, from its start or from the state a previous
// launch saved, for at most P.chunk_iters steps.  kSmallShare: the small-share
// kernel (above): r in shared memory, x updated by warps 1.. behind the
// barrier of the r.r sum; it runs a solve in one launch.
//
// Scalars live in the CTA state in shared memory (thread 0 updates them
// between CTA barriers; every thread reads them after one), so that the
// registers of the step loop's product are the product's own.
template <bool kMixed, bool kJacobi, bool kSmallShare, bool kNeighborWait>
__device__ __forceinline__ void solve_consumers(const RingSmem& sm, const CtaStream& cs, const SolveParams& P,
                                                const int rank, const int32_t* stream_rows) {
  // kNeighborWait: the single-system kernel for large shares (P.flags set
  // when the group has several CTAs); the small-share and batched kernels
  // always use the group barrier.
  const bool neighbor = kNeighborWait && P.flags != nullptr;
  const DevCsr& A = P.A;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int row0 = A.block_row[rank], row1 = A.block_row[rank + 1];
  const int nb = P.group;
  CtaState* st = sm.state();
  SumScratch* ss = sm.sums();
  SolveCtrl* ctrl = P.ctrl;
  double* __restrict__ x = P.x;
  double* __restrict__ r = P.r;
  double* __restrict__ p = P.p;
  ConsumerCursor cur;
  constexpr int kVR = vec_rows<kJacobi, kSmallShare>();
  // r_i of the CTA's rows: shared memory in the small-share kernel
  double* const r_loc = sm.local() - row0;
  auto R = [&](int i) -> double& {
    if constexpr (kSmallShare) return r_loc[i];
    else return r[i];
  };

  // Group-wide sum of nv values per thread (nv <= 3), fused with the vote of
  // the consumer warps (`ok`: this thread's waits all succeeded).  Each warp
  // sums its lanes exactly in fixed point; warp 0 combines the warps,
  // publishes the CTA's values, meets the other CTAs of the group at the
  // barrier and sums the group's CTA values in fixed point (exact and
  // order-independent: the same bits in every CTA); lane 0 then runs
  // fin(sums), which updates the CTA state; one CTA barrier publishes it.
  // Two slots of partials (3 nb values each) alternate so that a fast CTA
  // publishing the next sum never overwrites values a slow CTA still reads.
  // `side()` runs in warps 1.. while warp 0 does this: work of the step that
  // needs no group-wide value yet, hidden behind the barrier.
  // Returns false in every thread if a wait gave up, here or anywhere before.
  auto group_sum = [&](bool ok, int nv, double v0, double v1, double v2, auto&& fin, auto&& side) -> bool {
    const double vin[kMaxSumValues] = {v0, v1, v2};
    FxPart fp[kMaxSumValues];
#pragma unroll
    for (int j = 0; j < kMaxSumValues; ++j)
      if (j < nv) fp[j] = fx_warp(vin[j]);
    const bool wok = __all_sync(0xffffffffu, ok);
    if (lane == 0) {
#pragma unroll
      for (int j = 0; j < kMaxSumValues; ++j)
        if (j < nv) ss->part[j][warp] = fp[j];
      ss->ok[warp] = wok ? 1 : 0;
    }
    cta_sync();
    if (warp == 0) {
      const bool valid = lane < kWarps;
      bool good = __all_sync(0xffffffffu, valid ? ss->ok[lane] != 0 : true);
      double sum[kMaxSumValues] = {0.0, 0.0, 0.0};
#pragma unroll
      for (int j = 0; j < kMaxSumValues; ++j)
        if (j < nv) sum[j] = fx_combine(valid ? ss->part[j][lane] : FxPart{0, 0, 0}, valid);
      if (good && nb > 1) {
        const int slot = st->slot;
        double* part = P.partials + static_cast<size_t>(slot) * kMaxSumValues * nb;
        int bar_ok = 1;
        if (lane == 0) {
#pragma unroll
          for (int j = 0; j < kMaxSumValues; ++j)
            if (j < nv) part[j * nb + rank] = sum[j];
          bar_ok = group_barrier_t0(ctrl, &st->target, static_cast<unsigned int>(nb), P.wait_limit_ns, ++st->site);
        }
        good = __shfl_sync(0xffffffffu, bar_ok, 0) != 0;
        __syncwarp();
        if (good) {
#pragma unroll
          for (int j = 0; j < kMaxSumValues; ++j)
            if (j < nv) sum[j] = fx_warp_sum_array(part + j * nb, nb);
          if (lane == 0) st->slot = slot ^ 1;
        }
      }
      if (lane == 0) {
        st->ok = good ? 1 : 0;
        if (good) fin(sum);
      }
    } else {
      side();
    }
    cta_sync();
    return st->ok != 0;
  };
  auto no_side = [] {};
  // Group barrier of all threads: every write before it is visible to every
  // CTA of the group after it.
  auto group_sync = [&]() -> bool {
    cta_sync();
    if (tid == 0)
      st->ok = group_barrier_t0(ctrl, &st->target, static_cast<unsigned int>(nb), P.wait_limit_ns, ++st->site) ? 1
                                                                                                                : 0;
    cta_sync();
    return st->ok != 0;
  };
  // End of a step in a single-system solve (P.flags set): instead of a group
  // barrier, the CTA publishes this step's number in its epoch flag once its
  // p is written (release pattern as in the group barrier) and waits until
  // the CTAs that own the columns its rows reach (ranks dep_lo..dep_hi) have
  // published the same step: the next product gathers p only from them.
  // Reusing p in place is safe: a CTA overwrites its p only after the r.r
  // barrier of the step, which every CTA reaches after its product.
  auto neighbor_sync = [&]() -> bool {
    cta_sync();
    if (warp == 0) {
      const unsigned long long epoch = static_cast<unsigned long long>(st->k);
      if (lane == 0) {
        asm volatile("fence.acq_rel.gpu;" ::: "memory");
        asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(P.flags + rank), "l"(epoch) : "memory");
      }
      bool good = true;
      unsigned long long t0 = 0;
      uint32_t spins = 0;
      for (int q0 = st->dep_lo; q0 <= st->dep_hi && good; q0 += 32) {
        const int q = q0 + lane;
        if (q <= st->dep_hi && q != rank) {
          for (;;) {
            unsigned long long v;
            asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(P.flags + q) : "memory");
            if (v >= epoch) break;
            if ((++spins & 255u) == 0) {
              if (*reinterpret_cast<const volatile int32_t*>(&ctrl->abort)) { good = false; break; }
              const unsigned long long now = global_timer_ns();
              if (t0 == 0) t0 = now;
              else if (now - t0 > P.wait_limit_ns) {
                atomicExch(&ctrl->abort, 1);
                atomicExch(&ctrl->timeout_site, kNeighborSite);
                good = false;
                break;
              }
            }
          }
        }
      }
      good = __all_sync(0xffffffffu, good);
      asm volatile("fence.acq_rel.gpu;" ::: "memory");
      if (lane == 0) st->ok = good ? 1 : 0;
    }
    cta_sync();
    return st->ok != 0;
  };
  // Products outside the step loop (setup, the final true residual, the
  // mixed solve's residual replacements) read the FP64 values and columns
  // directly from global memory with a compact per-lane loop: they run once
  // per solve (or every replace_every steps), and keeping the unrolled ring
  // product out of them leaves its single copy, in the step loop, the
  // registers it needs.  The ring keeps streaming what the step loop uses.
  auto product64 = [&](const double* xin, const double* aux, auto& epi) -> bool {
    return spmv_pass<false, double, double, double>(sm, cs, cur, A, A.val, xin, aux, epi, P.wait_limit_ns, stream_rows);
  };

  // ---- state: saved by an earlier launch of this solve (written by another
  // kernel, so read through L2), or fresh
  if (tid == 0) {
    st->slot = 0;
    st->site = 0;
    st->ok = 1;
    st->flags = 0;
    st->target = 0;
    st->k = 0;
    if (__ldcg(&ctrl->phase) == kPhaseRunning) {
      st->target = __ldcg(&ctrl->rounds) * static_cast<unsigned long long>(nb);
      st->slot = __ldcg(&ctrl->slot);
      st->rho = __ldcg(&ctrl->rho);
      st->bnorm2 = __ldcg(&ctrl->bnorm2);
      st->k = __ldcg(&ctrl->iters);
      const double rel = __ldcg(&ctrl->relres_rec);
      st->rr = rel * rel * st->bnorm2;  // reported only (the next step recomputes it)
      st->flags = kFlagResumed;
    }
    st->dep_lo = 0x7fffffff;  // smallest and largest column of the CTA's rows, first
    st->dep_hi = -1;
  }
  cta_sync();
  if (neighbor) {
    // the CTAs whose p the product gathers: ranks owning the CTA's column range
    int cmin = 0x7fffffff, cmax = -1;
    for (int k = A.row_ptr[row0] + tid; k < A.row_ptr[row1]; k += kConsumers) {
      const int c = A.col_idx[k];
      cmin = min(cmin, c);
      cmax = max(cmax, c);
    }
    cmin = static_cast<int>(__reduce_min_sync(0xffffffffu, static_cast<unsigned int>(cmin)));
    cmax = __reduce_max_sync(0xffffffffu, cmax);
    if (lane == 0) {
      atomicMin(&st->dep_lo, cmin);
      atomicMax(&st->dep_hi, cmax);
    }
    cta_sync();
    if (tid == 0) {
      auto owner = [&](int c) {  // the rank whose row range holds row c
        int lo = 0, hi = nb - 1;
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (A.block_row[mid] <= c) lo = mid;
          else hi = mid - 1;
        }
        return lo;
      };
      if (st->dep_hi < 0) {  // no entries: nothing to wait for
        st->dep_lo = 1;
        st->dep_hi = 0;
      } else {
        st->dep_lo = owner(st->dep_lo);
        st->dep_hi = owner(st->dep_hi);
      }
    }
    cta_sync();
  }
  if (!(st->flags & kFlagResumed)) {
    // ---- setup: r = b - A x, z = dinv .* r (Jacobi) or r, p = z,
    //      rho = r.z, rr = r.r, ||b||^2
    double acc_rr = 0.0, acc_bb = 0.0, acc_rz = 0.0;
    auto epi = [&](int i, double s, double bi) {
      const double ri = bi - s;
      double zi = ri;
      if constexpr (kJacobi) zi = P.dinv[i] * ri;
      R(i) = ri;
      p[i] = zi;
      if constexpr (kMixed) P.p32[i] = static_cast<float>(zi);
      acc_rr = fma(ri, ri, acc_rr);
      if constexpr (kJacobi) acc_rz = fma(ri, zi, acc_rz);
      acc_bb = fma(bi, bi, acc_bb);
    };
    const bool ok = product64(x, P.b, epi);
    if (!group_sum(ok, kJacobi ? 3 : 2, acc_rr, acc_bb, acc_rz, [&](const double* sum) {
          st->rr = sum[0];
          st->bnorm2 = sum[1];
          st->rho = kJacobi ? sum[2] : sum[0];
        }, no_side)) {
      solve_fail(sm, P);
      return;
    }
  }
  if (st->bnorm2 == 0.0) {  // b = 0: the solution is 0
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
  if (tid == 0) {
    // Stopping test sqrt(rr) <= tol ||b|| evaluated as rr <= tol^2 ||b||^2
    // (no square root on the critical path; the same test up to rounding).
    st->thresh2 = (P.tol * P.tol) * st->bnorm2;
    const long long k = st->k;
    st->k_end = P.chunk_iters > 0 && P.chunk_iters < P.maxit - k ? k + P.chunk_iters : P.maxit;
    if (!(st->flags & kFlagResumed) && st->rr <= st->thresh2) st->flags |= kFlagDone;
  }
  cta_sync();

  for (;;) {
    if ((st->flags & kFlagDone) || st->k >= P.maxit) break;
    // ---- q = A p, gamma = p.q
    double acc_g = 0.0;
    bool ok;
    if constexpr (kMixed) {
      auto epi = [&](int i, float s, double pi) {
        const double qi = static_cast<double>(s);
        P.q[i] = qi;
        acc_g = fma(pi, qi, acc_g);
      };
      ok = spmv_pass<true, float, float, float>(sm, cs, cur, A, A.val32, P.p32, p, epi, P.wait_limit_ns,
                                                  stream_rows);
    } else {
      auto epi = [&](int i, double s, double pi) {
        P.q[i] = s;
        acc_g = fma(pi, s, acc_g);
      };
      ok = spmv_pass<true, double, double, double>(sm, cs, cur, A, A.val, p, p, epi, P.wait_limit_ns,
                                                     stream_rows);
    }
    // alpha = rho / gamma, once per CTA (an FP64 division is slow)
    if (!group_sum(ok, 1, acc_g, 0.0, 0.0, [&](const double* sum) {
          const double gamma = sum[0];
          if (!(gamma > 0.0) || !isfinite(gamma)) st->flags |= kFlagBreakdown;  // not SPD, or overflow
          else st->alpha = st->rho / gamma;
        }, no_side)) {
      solve_fail(sm, P);
      return;
    }
    if (st->flags & kFlagBreakdown) break;
    const double alpha = st->alpha;

    // ---- r -= alpha q; rr = r.r and (Jacobi) r.z   (kVR rows per thread in flight)
    double acc_r = 0.0, acc_z = 0.0;
    for (int base = row0 + tid; base < row1; base += kVR * kConsumers) {
      double qv[kVR], rv[kVR], dv[kVR];
#pragma unroll
      for (int u = 0; u < kVR; ++u) {
        const int i = base + u * kConsumers;
        if (i < row1) {
          qv[u] = P.q[i];
          rv[u] = R(i);
          if constexpr (kJacobi) dv[u] = P.dinv[i];
        }
      }
#pragma unroll
      for (int u = 0; u < kVR; ++u) {
        const int i = base + u * kConsumers;
        if (i < row1) {
          const double rn = fma(-alpha, qv[u], rv[u]);
          R(i) = rn;
          acc_r = fma(rn, rn, acc_r);
          if constexpr (kJacobi) acc_z = fma(rn, dv[u] * rn, acc_z);
        }
      }
    }
    // kSmallShare: x += alpha p by warps 1.. while warp 0 does the sum below (x is
    // needed again only by the next residual replacement or at the end)
    auto side_x = [&] {
      if constexpr (kSmallShare) {
        for (int base = row0 + tid - 32; base < row1; base += 2 * (kConsumers - 32)) {
          double pv[2], xv[2];
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const int i = base + u * (kConsumers - 32);
            if (i < row1) {
              pv[u] = p[i];
              xv[u] = x[i];
            }
          }
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const int i = base + u * (kConsumers - 32);
            if (i < row1) x[i] = fma(alpha, pv[u], xv[u]);
          }
        }
      }
    };
    if (!group_sum(true, kJacobi ? 2 : 1, acc_r, acc_z, 0.0, [&](const double* sum) {
          const long long k = st->k + 1;
          st->k = k;
          const double rr = sum[0], rho_new = kJacobi ? sum[1] : sum[0];
          st->rr = rr;
          // beta keeps the recurrence's own ratio (rho_new: the recursive r.z
          // of this step), also when r is replaced below
          st->beta = rho_new / st->rho;
          bool replace = false;
          if constexpr (kMixed) replace = (P.replace_every > 0 && k % P.replace_every == 0) || rr <= st->thresh2;
          if (replace) {
            st->flags |= kFlagReplace;
          } else {
            if (rr <= st->thresh2) st->flags |= kFlagDone;
            st->rho = rho_new;
          }
        }, side_x)) {
      solve_fail(sm, P);
      return;
    }
    const int32_t f = st->flags;
    const double beta = st->beta;
    if (f & kFlagReplace) {
      // x += alpha p (unless done behind the sum), then r = b - A x in FP64
      // (residual replacement); r, rr and rho take the true residual's values
      if constexpr (!kSmallShare)
        for (int i = row0 + tid; i < row1; i += kConsumers) x[i] = fma(alpha, p[i], x[i]);
      if (!group_sync()) { solve_fail(sm, P); return; }
      double acc_t = 0.0, acc_tz = 0.0;
      auto epi = [&](int i, double s, double bi) {
        const double ri = bi - s;
        R(i) = ri;
        acc_t = fma(ri, ri, acc_t);
        if constexpr (kJacobi) acc_tz = fma(ri, P.dinv[i] * ri, acc_tz);
      };
      const bool okr = product64(x, P.b, epi);
      if (!group_sum(okr, kJacobi ? 2 : 1, acc_t, acc_tz, 0.0, [&](const double* sum) {
            st->rr = sum[0];
            st->rho = kJacobi ? sum[1] : sum[0];
            st->flags &= ~kFlagReplace;
            if (sum[0] <= st->thresh2) st->flags |= kFlagDone;
          }, no_side)) {
        solve_fail(sm, P);
        return;
      }
      if (st->flags & kFlagDone) break;
      for (int i = row0 + tid; i < row1; i += kConsumers) {
        double zi = R(i);
        if constexpr (kJacobi) zi = P.dinv[i] * zi;
        const double pi = fma(beta, p[i], zi);
        p[i] = pi;
        if constexpr (kMixed) P.p32[i] = static_cast<float>(pi);
      }
    } else if (f & kFlagDone) {
      if constexpr (!kSmallShare)
        for (int i = row0 + tid; i < row1; i += kConsumers) x[i] = fma(alpha, p[i], x[i]);
      break;
    } else if constexpr (kSmallShare) {
      // ---- p = z + beta p   (z = dinv .* r, or r; x was updated behind the sum)
      for (int base = row0 + tid; base < row1; base += kVR * kConsumers) {
        double pv[kVR], zv[kVR];
#pragma unroll
        for (int u = 0; u < kVR; ++u) {
          const int i = base + u * kConsumers;
          if (i < row1) {
            pv[u] = p[i];
            zv[u] = R(i);
            if constexpr (kJacobi) zv[u] = P.dinv[i] * zv[u];
          }
        }
#pragma unroll
        for (int u = 0; u < kVR; ++u) {
          const int i = base + u * kConsumers;
          if (i < row1) {
            const double pn = fma(beta, pv[u], zv[u]);
            p[i] = pn;
            if constexpr (kMixed) P.p32[i] = static_cast<float>(pn);
          }
        }
      }
    } else {
      // ---- x += alpha p; p = z + beta p   (z = dinv .* r, or r)
      for (int base = row0 + tid; base < row1; base += kVR * kConsumers) {
        double pv[kVR], zv[kVR], xv[kVR];
#pragma unroll
        for (int u = 0; u < kVR; ++u) {
          const int i = base + u * kConsumers;
          if (i < row1) {
            pv[u] = p[i];
            zv[u] = R(i);
            if constexpr (kJacobi) zv[u] = P.dinv[i] * zv[u];
            xv[u] = __ldcs(x + i);  // x is not read again this step: evict-first
          }
        }
#pragma unroll
        for (int u = 0; u < kVR; ++u) {
          const int i = base + u * kConsumers;
          if (i < row1) {
            __stcs(x + i, fma(alpha, pv[u], xv[u]));
            const double pn = fma(beta, pv[u], zv[u]);
            p[i] = pn;
            if constexpr (kMixed) P.p32[i] = static_cast<float>(pn);
          }
        }
      }
    }
    bool synced;
    if constexpr (kNeighborWait) synced = neighbor ? neighbor_sync() : group_sync();
    else synced = group_sync();
    if (!synced) { solve_fail(sm, P); return; }
    if (st->k >= st->k_end && st->k < P.maxit) {
      // end of this launch's share of the solve: save the state (identical in
      // every CTA of the group; x, r, p are complete after the barrier)
      if (rank == 0 && tid == 0) {
        ctrl->iters = st->k;
        ctrl->rho = st->rho;
        ctrl->bnorm2 = st->bnorm2;
        ctrl->relres_rec = sqrt(st->rr / st->bnorm2);
        ctrl->rounds = st->target / static_cast<unsigned long long>(nb);
        ctrl->slot = st->slot;
        ctrl->phase = kPhaseRunning;
      }
      consumers_done(sm);
      return;
    }
  }

  // ---- true residual ||b - A x|| / ||b|| (x complete everywhere first)
  if (!group_sync()) { solve_fail(sm, P); return; }
  double acc_t = 0.0;
  auto epi = [&](int i, double s, double bi) {
    const double d = bi - s;
    acc_t = fma(d, d, acc_t);
  };
  const bool okt = product64(x, P.b, epi);
  if (!group_sum(okt, 1, acc_t, 0.0, 0.0, [&](const double* sum) {
        if (rank == 0) {
          const int32_t f = st->flags;
          ctrl->status = (f & kFlagBreakdown) ? kEBREAKDOWN : ((f & kFlagDone) ? kOK : kENOTCONV);
          ctrl->iters = st->k;
          ctrl->rho = st->rho;
          ctrl->bnorm2 = st->bnorm2;
          ctrl->relres_rec = sqrt(st->rr / st->bnorm2);
          ctrl->relres_true = sqrt(sum[0] / st->bnorm2);
          ctrl->phase = kPhaseDone;
        }
      }, no_side)) {
    solve_fail(sm, P);
    return;
  }
  consumers_done(sm);
}

}  // namespace cgk
