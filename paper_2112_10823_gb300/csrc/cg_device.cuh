// Device-side building blocks of the CG kernels: PTX wrappers for 1-D TMA
// bulk copies and mbarriers, deterministic reductions, the bounded grid
// barrier of the persistent solve, and the shared-memory-staged CSR product.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "cg_internal.h"

namespace cgk {

// ------------------------------------------------------------------ PTX

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long global_timer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Makes mbarrier initialisation visible to the async (TMA) proxy.
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Orders this thread's earlier generic-proxy shared-memory accesses (made
// visible to it by a CTA barrier) before later async-proxy writes.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// 1-D bulk copy global -> shared (TMA), completion counted on `bar`.
// dst and src 16-byte aligned, bytes a non-zero multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void red_release_add_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ int ld_volatile_i32(const int32_t* p) {
  return *reinterpret_cast<const volatile int32_t*>(p);
}

// ------------------------------------------------------------ reductions

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;  // identical in every lane (IEEE addition is commutative)
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum of `v` over the CTA, in a fixed order; every thread gets the same value.
// The per-thread values go through shared memory and only warp 0 adds them
// (8 sequential adds per lane, then a butterfly), which keeps the number of
// FP64 warp instructions small: FP64 issue is scarce on this GPU.
// `red` holds at least kBlock + 1 doubles.  Must be called by all threads.
__device__ __forceinline__ double block_sum(double v, double* red) {
  __syncthreads();  // earlier users of `red` are done
  red[threadIdx.x] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double s = red[threadIdx.x];
#pragma unroll
    for (int j = 1; j < kWarps; ++j) s += red[threadIdx.x + 32 * j];
    s = warp_sum(s);
    if (threadIdx.x == 0) red[kBlock] = s;
  }
  __syncthreads();
  return red[kBlock];
}

// Two sums at once (same order rules as block_sum).  `red` holds 2*kBlock+2.
__device__ __forceinline__ void block_sum2(double& a, double& b, double* red) {
  __syncthreads();
  red[threadIdx.x] = a;
  red[kBlock + threadIdx.x] = b;
  __syncthreads();
  if (threadIdx.x < 32) {
    double s = red[threadIdx.x], t = red[kBlock + threadIdx.x];
#pragma unroll
    for (int j = 1; j < kWarps; ++j) {
      s += red[threadIdx.x + 32 * j];
      t += red[kBlock + threadIdx.x + 32 * j];
    }
    s = warp_sum(s);
    t = warp_sum(t);
    if (threadIdx.x == 0) {
      red[2 * kBlock] = s;
      red[2 * kBlock + 1] = t;
    }
  }
  __syncthreads();
  a = red[2 * kBlock];
  b = red[2 * kBlock + 1];
}

// ------------------------------------------------------------ grid barrier

// Bounded grid-wide barrier for a cooperative (co-resident) launch.  Thread 0
// of each CTA adds one arrival to a monotonic 64-bit counter with release
// semantics and spins with acquire loads until all CTAs of this round have
// arrived; the fence afterwards makes every write that preceded any CTA's
// arrival visible to all threads of this CTA.  A wait longer than
// `limit_ns`, or an abort raised by another CTA, makes it return false in
// every thread of the CTA (the caller then leaves the kernel).
struct GridBarrier {
  unsigned long long target = 0;

  __device__ __forceinline__ bool sync(SolveCtrl* ctrl, unsigned long long limit_ns, int site,
                                       int32_t* flag_smem) {
    __syncthreads();
    if (threadIdx.x == 0) {
      target += gridDim.x;
      __threadfence();
      red_release_add_u64(&ctrl->barrier, 1ull);
      int32_t ok = 1;
      unsigned long long t0 = 0;
      uint32_t spins = 0;
      while (ld_acquire_u64(&ctrl->barrier) < target) {
        if ((++spins & 255u) == 0) {
          if (ld_volatile_i32(&ctrl->abort)) { ok = 0; break; }
          unsigned long long now = global_timer_ns();
          if (t0 == 0) t0 = now;
          else if (now - t0 > limit_ns) {
            atomicExch(&ctrl->abort, 1);
            atomicExch(&ctrl->timeout_site, site);
            ok = 0;
            break;
          }
        }
      }
      __threadfence();
      *flag_smem = ok;
    }
    __syncthreads();
    return *flag_smem != 0;
  }
};

// ------------------------------------------------------- staged CSR product

// Shared memory of the staged product: kStages stages of values + column
// indices, their mbarriers, a reduction scratch and a broadcast flag, laid out
// by offsets in one dynamic shared-memory buffer.  The value area of a stage
// is sized for FP64; the FP32 product of the mixed-precision solve uses the
// first half of it, so both products share the same stages and mbarriers.
struct SpmvSmem {
  static constexpr size_t kValBytes = (sizeof(double) * kStageVal + 15) & ~size_t(15);
  static constexpr size_t kColBytes = (sizeof(int32_t) * kStageCol + 15) & ~size_t(15);
  static constexpr size_t kStageBytes = kValBytes + kColBytes;
  static constexpr size_t kRedBytes = sizeof(double) * (2 * kBlock + 4);
  static constexpr size_t kBytes = kStages * kStageBytes + kRedBytes + 8 * kStages + 16;

  unsigned char* base;
  template <typename T>
  __device__ T* val(int s) const { return reinterpret_cast<T*>(base + s * kStageBytes); }
  __device__ int32_t* col(int s) const {
    return reinterpret_cast<int32_t*>(base + s * kStageBytes + kValBytes);
  }
  __device__ double* red() const { return reinterpret_cast<double*>(base + kStages * kStageBytes); }
  __device__ uint64_t* bar(int s) const {
    return reinterpret_cast<uint64_t*>(base + kStages * kStageBytes + kRedBytes) + s;
  }
  __device__ int32_t* flag() const {
    return reinterpret_cast<int32_t*>(base + kStages * kStageBytes + kRedBytes + 8 * kStages);
  }
};

// Per-CTA pipeline state of the staged product; lives in registers and is
// uniform across the CTA.
struct StagePipe {
  uint32_t phase = 0;     // bit s: parity the next completion of stage s will have
  uint32_t issued = 0;    // staged chunks issued so far
  uint32_t consumed = 0;  // staged chunks consumed so far
};

__device__ __forceinline__ void stage_init(const SpmvSmem& sm) {
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) mbar_init(sm.bar(s), 1);
    fence_mbar_init();
  }
  __syncthreads();
}

// Issue the bulk copies of chunk c (values of type T, column indices) into
// stage `s`.  Called by one thread.
template <typename T>
__device__ __forceinline__ void stage_issue(const SpmvSmem& sm, int s, const int32_t* row_ptr,
                                            const int32_t* col_idx, const T* val, int r0, int r1) {
  constexpr int kAlignV = 16 / sizeof(T);
  const int k0 = row_ptr[r0], k1 = row_ptr[r1];
  const int kv0 = k0 & ~(kAlignV - 1);
  const int kc0 = k0 & ~3;
  const uint32_t bv = (static_cast<uint32_t>(k1 - kv0) * sizeof(T) + 15u) & ~15u;
  const uint32_t bc = (static_cast<uint32_t>(k1 - kc0) * 4u + 15u) & ~15u;
  fence_proxy_async_smem();
  mbar_arrive_expect_tx(sm.bar(s), bv + bc);
  if (bv) bulk_g2s(sm.val<T>(s), val + kv0, bv, sm.bar(s));
  if (bc) bulk_g2s(sm.col(s), col_idx + kc0, bc, sm.bar(s));
}

// Wait (bounded) for stage s.  The outcome is made uniform over the CTA:
// false in every thread if any thread gave up.
__device__ __forceinline__ bool stage_wait(const SpmvSmem& sm, int s, uint32_t parity,
                                           unsigned long long limit_ns) {
  uint32_t spins = 0;
  unsigned long long t0 = 0;
  int ok = 1;
  while (!mbar_try_wait(sm.bar(s), parity)) {
    if ((++spins & 63u) == 0) {
      unsigned long long now = global_timer_ns();
      if (t0 == 0) t0 = now;
      else if (now - t0 > limit_ns) { ok = 0; break; }
    }
  }
  return __syncthreads_and(ok) != 0;
}

// Gather-multiply-accumulate of one row held in shared memory: with
// jv = k - kv0 and jc = k - kc0 the stage positions of entry k,
//   s = sum_{k in [ks, ke)} sv[jv] * x[sc[jc]], in order, with FMA.
// Gathers are issued 8 at a time to keep several loads in flight.
template <typename T, typename X, typename Acc>
__device__ __forceinline__ Acc row_dot_smem(const T* sv, const int32_t* sc, int jv, int jc, int len,
                                            const X* x) {
  Acc s = Acc(0);
  int t = 0;
  for (; t + 8 <= len; t += 8) {
    int c[8];
    X xv[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) c[u] = sc[jc + t + u];
#pragma unroll
    for (int u = 0; u < 8; ++u) xv[u] = x[c[u]];
#pragma unroll
    for (int u = 0; u < 8; ++u) s = fma(Acc(sv[jv + t + u]), Acc(xv[u]), s);
  }
  for (; t < len; ++t) s = fma(Acc(sv[jv + t]), Acc(x[sc[jc + t]]), s);
  return s;
}

// y rows of chunk [r0, r1) from stage s (thread- or warp-per-row), each result
// handed to epi(i, yi) by the thread that computed it.
template <typename T, typename X, typename Acc, typename Epi>
__device__ __forceinline__ void chunk_compute_staged(const SpmvSmem& sm, int s, int mode,
                                                     const int32_t* row_ptr, int r0, int r1, const X* x,
                                                     Epi& epi) {
  constexpr int kAlignV = 16 / sizeof(T);
  const int k0 = row_ptr[r0];
  const int kv0 = k0 & ~(kAlignV - 1), kc0 = k0 & ~3;
  const T* sv = sm.val<T>(s);
  const int32_t* sc = sm.col(s);
  if (mode == kThreadPerRow) {
    const int i = r0 + static_cast<int>(threadIdx.x);
    if (i < r1) {
      const int ks = row_ptr[i], ke = row_ptr[i + 1];
      epi(i, row_dot_smem<T, X, Acc>(sv, sc, ks - kv0, ks - kc0, ke - ks, x));
    }
  } else {  // kWarpPerRow
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = r0 + w; i < r1; i += kWarps) {
      const int ks = row_ptr[i], ke = row_ptr[i + 1];
      Acc acc = Acc(0);
      for (int k = ks + lane; k < ke; k += 32) acc = fma(Acc(sv[k - kv0]), Acc(x[sc[k - kc0]]), acc);
      if constexpr (sizeof(Acc) == 8) acc = warp_sum(acc);
      else acc = warp_sum_f(acc);
      if (lane == 0) epi(i, acc);
    }
  }
}

// One row longer than a stage, streamed from global memory by the whole CTA.
template <typename T, typename X, typename Acc, typename Epi>
__device__ __forceinline__ void chunk_compute_long(const int32_t* row_ptr, const int32_t* col_idx,
                                                   const T* val, int i, const X* x, double* red, Epi& epi) {
  const int ks = row_ptr[i], ke = row_ptr[i + 1];
  Acc acc = Acc(0);
  for (int k = ks + static_cast<int>(threadIdx.x); k < ke; k += kBlock)
    acc = fma(Acc(val[k]), Acc(x[col_idx[k]]), acc);
  const double tot = block_sum(static_cast<double>(acc), red);
  if (threadIdx.x == 0) epi(i, static_cast<Acc>(tot));
}

// The product over chunks [c0, c1) of A (values `val` of type T), staged
// through shared memory with one chunk in flight ahead of the one being
// computed.  Returns false if a wait gave up (the caller leaves the kernel).
template <typename T, typename X, typename Acc, typename Epi>
__device__ __forceinline__ bool spmv_pass(const SpmvSmem& sm, StagePipe& pp, const DevCsr& A, const T* val,
                                          int c0, int c1, const X* x, Epi& epi, unsigned long long limit_ns) {
  const int32_t* row_ptr = A.row_ptr;
  const int32_t* cr = A.chunk_row;
  const int32_t* cm = A.chunk_mode;
  // next staged chunk at or after c
  auto next_staged = [&](int c) {
    while (c < c1 && cm[c] == kBlockPerRow) ++c;
    return c;
  };
  int nxt = next_staged(c0);
  if (nxt < c1 && threadIdx.x == 0)
    stage_issue<T>(sm, static_cast<int>(pp.issued & 1u), row_ptr, A.col_idx, val, cr[nxt], cr[nxt + 1]);
  if (nxt < c1) pp.issued++;
  for (int c = c0; c < c1; ++c) {
    const int mode = cm[c];
    if (mode == kBlockPerRow) {
      chunk_compute_long<T, X, Acc>(row_ptr, A.col_idx, val, cr[c], x, sm.red(), epi);
      continue;
    }
    // c is the staged chunk number pp.consumed; put the next one in flight.
    nxt = next_staged(c + 1);
    if (nxt < c1) {
      if (threadIdx.x == 0)
        stage_issue<T>(sm, static_cast<int>(pp.issued & 1u), row_ptr, A.col_idx, val, cr[nxt], cr[nxt + 1]);
      pp.issued++;
    }
    const int s = static_cast<int>(pp.consumed & 1u);
    const uint32_t parity = (pp.phase >> s) & 1u;
    if (!stage_wait(sm, s, parity, limit_ns)) return false;
    pp.phase ^= (1u << s);
    chunk_compute_staged<T, X, Acc>(sm, s, mode, row_ptr, cr[c], cr[c + 1], x, epi);
    __syncthreads();  // stage s is free again before it is refilled
    pp.consumed++;
  }
  return true;
}

// Before leaving the kernel on an error path: wait (bounded) for every copy
// this CTA still has in flight, so no bulk copy lands in shared memory after
// the CTA is gone.
__device__ __forceinline__ void stage_drain(const SpmvSmem& sm, StagePipe& pp, unsigned long long limit_ns) {
  while (pp.consumed < pp.issued) {
    const int s = static_cast<int>(pp.consumed & 1u);
    stage_wait(sm, s, (pp.phase >> s) & 1u, limit_ns);
    pp.phase ^= (1u << s);
    pp.consumed++;
  }
}

}  // namespace cgk
