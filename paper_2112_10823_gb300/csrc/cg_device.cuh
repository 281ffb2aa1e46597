// Device-side building blocks of the CG kernels: PTX wrappers for 1-D TMA
// bulk copies and mbarriers, deterministic reductions, the bounded grid
// barrier of the persistent solve, and the CSR product fed by a TMA ring.
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

// Sum of `v` over the CTA in a fixed order (FP64 adds); every thread gets the
// same value.  `red` holds blockDim.x + 1 doubles (blockDim.x a multiple of
// 32, at most 1024).  All threads must call it.
__device__ __forceinline__ double block_sum(double v, double* red) {
  const int nt = blockDim.x;
  __syncthreads();
  red[threadIdx.x] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double s = red[threadIdx.x];
    for (int j = 32 + threadIdx.x; j < nt; j += 32) s += red[j];
    s = warp_sum(s);
    if (threadIdx.x == 0) red[nt] = s;
  }
  __syncthreads();
  return red[nt];
}

// Scratch of the fixed-point CTA sum (shared memory).
struct FxScratch {
  long long m[kWarps];
  int32_t e[kWarps];
  int32_t nf[kWarps];
  double result;
};

// Sum over the CTA of K doubles per thread, exactly in fixed point.
//
// FP64 adds cost 64 cycles of latency each on this GPU, so a tree of them over
// hundreds of values sits on the critical path of every CG step.  Instead each
// value is rounded to a common fixed-point grid set by the largest exponent E
// among all values (spacing 2^(E-1074), i.e. about 2^-51 of the largest value,
// leaving 10 bits of headroom for up to 1024 terms), the integers are added
// exactly with integer adds (order-independent, so the sum is deterministic
// whatever the order of arrival), and the total is rounded once back to FP64.
// Zero and subnormal values count as zero; an infinite or NaN value makes the
// sum NaN.  Thread 0 converts the total; every thread receives it through
// shared memory.  Requires blockDim.x == kBlock and K * kBlock <= 1024.
template <int K>
__device__ __forceinline__ double fx_block_sum(const double (&v)[K], FxScratch* sc) {
  static_assert(K * kBlock <= 1024, "fixed-point headroom is 10 bits");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long bits[K];
  int e[K];
  int emax = 0, nfl = 0;
#pragma unroll
  for (int j = 0; j < K; ++j) {
    bits[j] = static_cast<unsigned long long>(__double_as_longlong(v[j]));
    e[j] = static_cast<int>((bits[j] >> 52) & 0x7ffull);
    emax = max(emax, e[j]);
    nfl |= (e[j] == 0x7ff);
  }
  const unsigned int ew = __reduce_max_sync(0xffffffffu, static_cast<unsigned int>(emax));
  const int nfw = __any_sync(0xffffffffu, nfl);
  __syncthreads();  // earlier users of sc are done
  if (lane == 0) {
    sc->e[warp] = static_cast<int32_t>(ew);
    sc->nf[warp] = nfw;
  }
  __syncthreads();
  int E = 0, nf = 0;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) {
    E = max(E, static_cast<int>(sc->e[w]));
    nf |= sc->nf[w];
  }
  long long m = 0;
#pragma unroll
  for (int j = 0; j < K; ++j) {
    if (e[j] != 0 && !nf) {
      const int s = E - e[j] + 1;  // >= 1
      if (s < 64) {
        const unsigned long long M = (bits[j] & 0xFFFFFFFFFFFFFull) | (1ull << 52);
        const unsigned long long rnd = (M + (1ull << (s - 1))) >> s;
        m += (bits[j] >> 63) ? -static_cast<long long>(rnd) : static_cast<long long>(rnd);
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m += __shfl_xor_sync(0xffffffffu, m, o);
  if (lane == 0) sc->m[warp] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long tot = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) tot += sc->m[w];
    double r;
    if (nf) r = __longlong_as_double(0x7ff8000000000000ll);  // NaN
    else if (E == 0) r = 0.0;
    else r = ldexp(static_cast<double>(tot), E - 1074);
    sc->result = r;
  }
  __syncthreads();
  return sc->result;
}

__device__ __forceinline__ double fx_block_sum(double v, FxScratch* sc) {
  const double a[1] = {v};
  return fx_block_sum<1>(a, sc);
}

// ------------------------------------------------------------ grid barrier

// Bounded grid-wide barrier for a cooperative (co-resident) launch, split in
// an arrive and a wait half so that a CTA can do independent work between
// them.  Thread 0 of each CTA adds one arrival to a monotonic 64-bit counter
// with release semantics and later spins with acquire loads until all CTAs of
// this round have arrived; the fence afterwards makes every write that
// preceded any CTA's arrival visible to all threads of this CTA.  A wait
// longer than `limit_ns`, or an abort raised by another CTA, makes wait()
// return false in every thread of the CTA (the caller then leaves the kernel).
struct GridBarrier {
  unsigned long long target = 0;

  // All threads call; the CTA's writes before this point are published.
  __device__ __forceinline__ void arrive(SolveCtrl* ctrl) {
    __syncthreads();
    target += gridDim.x;
    if (threadIdx.x == 0) {
      __threadfence();
      red_release_add_u64(&ctrl->barrier, 1ull);
    }
  }

  __device__ __forceinline__ bool wait(SolveCtrl* ctrl, unsigned long long limit_ns, int site,
                                       int32_t* flag_smem) {
    if (threadIdx.x == 0) {
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

  __device__ __forceinline__ bool sync(SolveCtrl* ctrl, unsigned long long limit_ns, int site,
                                       int32_t* flag_smem) {
    arrive(ctrl);
    return wait(ctrl, limit_ns, site, flag_smem);
  }
};

// ------------------------------------------------------ streamed CSR product

// Shared memory of the streamed product: the value ring (sized for FP64; the
// FP32 product uses its first half), the column-index ring, one mbarrier per
// ring slot, reduction scratch and a few broadcast words.
struct RingSmem {
  static constexpr size_t kValBytes = sizeof(double) * kRing;
  static constexpr size_t kColBytes = sizeof(int32_t) * kRing;
  static constexpr size_t kBarOff = kValBytes + kColBytes;
  static constexpr size_t kRedOff = kBarOff + 8 * kSlots;
  static constexpr size_t kRedBytes = sizeof(double) * (kBlock + 8);
  static constexpr size_t kFxOff = kRedOff + kRedBytes;
  static constexpr size_t kFxBytes = (sizeof(FxScratch) + 15) & ~size_t(15);
  static constexpr size_t kMiscOff = kFxOff + kFxBytes;
  static constexpr size_t kBytes = kMiscOff + 64;

  unsigned char* base;
  template <typename T>
  __device__ T* val() const { return reinterpret_cast<T*>(base); }
  __device__ int32_t* col() const { return reinterpret_cast<int32_t*>(base + kValBytes); }
  __device__ uint64_t* bar(int s) const { return reinterpret_cast<uint64_t*>(base + kBarOff) + s; }
  __device__ double* red() const { return reinterpret_cast<double*>(base + kRedOff); }
  __device__ FxScratch* fx() const { return reinterpret_cast<FxScratch*>(base + kFxOff); }
  __device__ int32_t* flag() const { return reinterpret_cast<int32_t*>(base + kMiscOff); }
  __device__ double* scalars() const { return reinterpret_cast<double*>(base + kMiscOff + 16); }
};

// Per-CTA state of the matrix stream; in registers, uniform across the CTA.
// Pieces are numbered globally (across passes) so that the slot of a piece is
// (global number % kSlots) and its mbarrier phase (global number / kSlots) & 1.
struct RingState {
  int kb = 0;            // first entry of the CTA's range, rounded down to a multiple of 4
  int ke = 0;            // end of the CTA's entry range
  int npieces = 0;       // pieces per pass
  uint32_t gbase = 0;    // global number of piece 0 of the current pass
  int issued = 0;        // pieces of the current pass issued
  int waited = 0;        // pieces of the current pass seen complete
  int released = 0;      // pieces of the current pass whose slots may be refilled
  int pre_type = 0;      // value size (4 or 8) of pieces prefetched for the next pass, 0 = none
  int pre_count = 0;     // pieces of the next pass already issued
};

__device__ __forceinline__ void ring_init(const RingSmem& sm, RingState& rs, const DevCsr& A, int row0,
                                          int row1) {
  if (threadIdx.x == 0) {
    for (int s = 0; s < kSlots; ++s) mbar_init(sm.bar(s), 1);
    fence_mbar_init();
  }
  __syncthreads();
  rs.kb = A.row_ptr[row0] & ~3;
  rs.ke = A.row_ptr[row1];
  // a CTA without rows streams nothing (kb may sit below ke after rounding)
  rs.npieces = row1 > row0 ? (rs.ke - rs.kb + kPiece - 1) >> kPieceLog : 0;
}

// Ring position of the first entry of piece 0 of the pass starting at gbase.
__device__ __forceinline__ int ring_pos_of_piece0(uint32_t gbase) {
  return static_cast<int>((gbase % kSlots) * kPiece);
}

// Issue piece j of the pass starting at gbase (values of type T).  One thread.
template <typename T>
__device__ __forceinline__ void ring_issue(const RingSmem& sm, const RingState& rs, uint32_t gbase, int j,
                                           const T* val, const int32_t* col) {
  const int e0 = rs.kb + j * kPiece;
  int e1 = e0 + kPiece;
  const int ke4 = (rs.ke + 3) & ~3;  // copy whole 16-byte groups (<= 3 padding entries)
  if (e1 > ke4) e1 = ke4;
  const int slot = static_cast<int>((gbase + static_cast<uint32_t>(j)) % kSlots);
  const int pos = slot * kPiece;
  const uint32_t bv = static_cast<uint32_t>(e1 - e0) * sizeof(T);
  const uint32_t bc = static_cast<uint32_t>(e1 - e0) * 4u;
  fence_proxy_async_smem();
  mbar_arrive_expect_tx(sm.bar(slot), bv + bc);
  bulk_g2s(sm.val<T>() + pos, val + e0, bv, sm.bar(slot));
  bulk_g2s(sm.col() + pos, col + e0, bc, sm.bar(slot));
}

// Wait (bounded) for global piece g; returns false if the wait gave up.
__device__ __forceinline__ bool ring_wait_global(const RingSmem& sm, uint32_t g, unsigned long long limit_ns) {
  const int slot = static_cast<int>(g % kSlots);
  const uint32_t parity = (g / kSlots) & 1u;
  uint32_t spins = 0;
  unsigned long long t0 = 0;
  while (!mbar_try_wait(sm.bar(slot), parity)) {
    if ((++spins & 63u) == 0) {
      const unsigned long long now = global_timer_ns();
      if (t0 == 0) t0 = now;
      else if (now - t0 > limit_ns) return false;
    }
  }
  return true;
}

// Wait for pieces [rs.waited, upto) of the current pass, in order.  Called by
// all threads; the outcome is made uniform over the CTA.
__device__ __forceinline__ bool ring_wait_upto(const RingSmem& sm, RingState& rs, int upto,
                                               unsigned long long limit_ns) {
  int ok = 1;
  for (int j = rs.waited; j < upto; ++j)
    if (!ring_wait_global(sm, rs.gbase + static_cast<uint32_t>(j), limit_ns)) ok = 0;
  if (upto > rs.waited) rs.waited = upto;
  return __syncthreads_and(ok) != 0;
}

// Keep the ring full: issue pieces while slots are free.  Thread 0 issues;
// the counters advance in every thread.
template <typename T>
__device__ __forceinline__ void ring_fill(const RingSmem& sm, RingState& rs, const T* val, const int32_t* col) {
  int lim = rs.released + kSlots;
  if (lim > rs.npieces) lim = rs.npieces;
  if (threadIdx.x == 0)
    for (int j = rs.issued; j < lim; ++j) ring_issue<T>(sm, rs, rs.gbase, j, val, col);
  if (lim > rs.issued) rs.issued = lim;
}

// Start a pass over values of type T: adopt the pieces prefetched for it, or
// first wait out prefetched pieces of the other type and skip past them.
template <typename T>
__device__ __forceinline__ bool ring_begin_pass(const RingSmem& sm, RingState& rs, const T* val,
                                                const int32_t* col, unsigned long long limit_ns) {
  if (rs.pre_count > 0 && rs.pre_type != static_cast<int>(sizeof(T))) {
    int ok = 1;
    for (int j = 0; j < rs.pre_count; ++j)
      if (!ring_wait_global(sm, rs.gbase + static_cast<uint32_t>(j), limit_ns)) ok = 0;
    if (!__syncthreads_and(ok)) return false;
    rs.gbase += static_cast<uint32_t>(rs.pre_count);
    rs.pre_count = 0;
  }
  rs.issued = rs.pre_count;
  rs.waited = 0;
  rs.released = 0;
  rs.pre_count = 0;
  rs.pre_type = 0;
  __syncthreads();  // no thread still reads the ring from an earlier pass
  ring_fill<T>(sm, rs, val, col);
  return true;
}

// End a pass: every piece of it has been consumed.  Optionally issue the
// first pieces of the next pass (values of type Tn) so that they load during
// whatever the CTA does before that pass.
template <typename Tn>
__device__ __forceinline__ void ring_end_pass(const RingSmem& sm, RingState& rs, const Tn* next_val,
                                              const int32_t* col) {
  rs.gbase += static_cast<uint32_t>(rs.npieces);
  rs.issued = rs.waited = rs.released = 0;
  rs.pre_count = 0;
  rs.pre_type = 0;
  if (next_val != nullptr && rs.npieces > 0) {
    const int cnt = rs.npieces < kSlots ? rs.npieces : kSlots;
    __syncthreads();  // every thread is done reading the ring
    if (threadIdx.x == 0)
      for (int j = 0; j < cnt; ++j) ring_issue<Tn>(sm, rs, rs.gbase, j, next_val, col);
    rs.pre_count = cnt;
    rs.pre_type = static_cast<int>(sizeof(Tn));
  }
}

// Before leaving the kernel on an error path: wait (bounded) for the copies
// this CTA still has in flight, so no bulk copy lands after the CTA is gone.
__device__ __forceinline__ void ring_drain(const RingSmem& sm, RingState& rs, unsigned long long limit_ns) {
  for (int j = rs.waited; j < rs.issued; ++j) ring_wait_global(sm, rs.gbase + static_cast<uint32_t>(j), limit_ns);
  for (int j = 0; j < rs.pre_count; ++j) ring_wait_global(sm, rs.gbase + static_cast<uint32_t>(j), limit_ns);
}

// Dot product of one row segment held in the ring: entries at ring positions
// pos, pos+1, ... (masked), len of them, in storage order, with FMA.  Up to U
// entries take a fully unrolled path that issues every gather before the
// first multiply-add; longer segments go 8 at a time.
template <typename T, typename X, typename Acc, int U>
__device__ __forceinline__ Acc seg_dot(const T* rv, const int32_t* rc, int pos, int len, const X* x) {
  Acc s = Acc(0);
  // Called by all 32 lanes of the warp (len = 0 for lanes without a row).
  // The unroll bound is the warp's longest segment, so no FP64 instruction is
  // issued for a slot that no lane needs: FP64 issue is the scarce resource.
  const int wmax = static_cast<int>(__reduce_max_sync(0xffffffffu, static_cast<unsigned int>(len)));
  if (wmax <= U) {
    // all gathers first (only they have long latency), then the FMAs with
    // the values read from shared memory as they are consumed
    X xv[U];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (u < wmax && u < len) xv[u] = x[rc[(pos + u) & kRingMask]];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (u < wmax && u < len) s = fma(Acc(rv[(pos + u) & kRingMask]), Acc(xv[u]), s);
    return s;
  }
  int t = 0;
  for (; t + 8 <= len; t += 8) {
    X xv[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) xv[u] = x[rc[(pos + t + u) & kRingMask]];
#pragma unroll
    for (int u = 0; u < 8; ++u) s = fma(Acc(rv[(pos + t + u) & kRingMask]), Acc(xv[u]), s);
  }
  for (; t < len; ++t) {
    const int p = (pos + t) & kRingMask;
    s = fma(Acc(rv[p]), Acc(x[rc[p]]), s);
  }
  return s;
}

// Rows of chunk [r0, r1) from the ring; each result goes to epi(i, yi) from
// the thread that holds it.  Entry k sits at ring position (k - kb + off) &
// kRingMask.
template <typename T, typename X, typename Acc, typename Epi>
__device__ __forceinline__ void chunk_compute_ring(const RingSmem& sm, int mode, const int32_t* row_ptr, int r0,
                                                   int r1, int kb, int off, const X* x, Epi& epi) {
  const T* rv = sm.val<T>();
  const int32_t* rc = sm.col();
  if (mode == kThreadPerRow) {
    const int i = r0 + static_cast<int>(threadIdx.x);
    int ks = 0, len = 0;
    if (i < r1) {
      ks = row_ptr[i];
      len = row_ptr[i + 1] - ks;
    }
    const Acc s = seg_dot<T, X, Acc, 16>(rv, rc, ks - kb + off, len, x);
    if (i < r1) epi(i, s);
  } else if (mode == kPairPerRow) {
    const int i = r0 + static_cast<int>(threadIdx.x >> 1);
    const int h = threadIdx.x & 1;
    int a = 0, len = 0;
    if (i < r1) {
      const int ks = row_ptr[i], ke = row_ptr[i + 1];
      const int half = (ke - ks + 1) >> 1;
      a = h ? ks + half : ks;
      len = h ? (ke - ks - half) : half;
    }
    const Acc part = seg_dot<T, X, Acc, 16>(rv, rc, a - kb + off, len, x);
    // first half + second half: the same value in both lanes (commutative add)
    const Acc other = __shfl_xor_sync(0xffffffffu, part, 1);
    const Acc s = part + other;
    if (h == 0 && i < r1) epi(i, s);
  } else {  // kWarpPerRow
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = r0 + w; i < r1; i += kWarps) {
      const int ks = row_ptr[i], ke = row_ptr[i + 1];
      Acc acc = Acc(0);
      for (int k = ks + lane; k < ke; k += 32) {
        const int p = (k - kb + off) & kRingMask;
        acc = fma(Acc(rv[p]), Acc(x[rc[p]]), acc);
      }
      if constexpr (sizeof(Acc) == 8) acc = warp_sum(acc);
      else acc = warp_sum_f(acc);
      if (lane == 0) epi(i, acc);
    }
  }
}

// One row longer than kChunkNnz, streamed from global memory by the whole CTA.
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

// The product over the CTA's chunks [c0, c1) with values `val` of type T,
// gathering x.  The pass starts from the pieces prefetched for it (if any)
// and ends by prefetching the first pieces of the next pass (next_val, of
// type Tn; nullptr for none).  Returns false if a wait gave up.
template <typename T, typename X, typename Acc, typename Tn, typename Epi>
__device__ __forceinline__ bool spmv_pass(const RingSmem& sm, RingState& rs, const DevCsr& A, const T* val,
                                          int c0, int c1, const X* x, Epi& epi, const Tn* next_val,
                                          unsigned long long limit_ns) {
  const int32_t* row_ptr = A.row_ptr;
  const int32_t* cr = A.chunk_row;
  const int32_t* cm = A.chunk_mode;
  if (!ring_begin_pass<T>(sm, rs, val, A.col_idx, limit_ns)) return false;
  const int off = ring_pos_of_piece0(rs.gbase);
  for (int c = c0; c < c1; ++c) {
    const int mode = cm[c];
    const int r0 = cr[c], r1 = cr[c + 1];
    const int k1 = row_ptr[r1];
    if (mode == kBlockPerRow) {
      chunk_compute_long<T, X, Acc>(row_ptr, A.col_idx, val, r0, x, sm.red(), epi);
    } else {
      const int k0 = row_ptr[r0];
      if (k1 > k0 && !ring_wait_upto(sm, rs, ((k1 - 1 - rs.kb) >> kPieceLog) + 1, limit_ns)) return false;
      chunk_compute_ring<T, X, Acc>(sm, mode, row_ptr, r0, r1, rs.kb, off, x, epi);
    }
    __syncthreads();  // the chunk's ring entries are consumed
    // Release the pieces that end before the next chunk's first entry.  A slot
    // is refilled only after its piece is complete, so pieces are waited for
    // before release; a row longer than the ring (streamed from global memory)
    // advances the ring in steps of at most kSlots pieces.
    const int rel = (c + 1 == c1) ? rs.npieces : ((k1 - rs.kb) >> kPieceLog);
    while (rel > rs.released) {
      const int upto = rel < rs.issued ? rel : rs.issued;
      if (!ring_wait_upto(sm, rs, upto, limit_ns)) return false;
      rs.released = upto;
      ring_fill<T>(sm, rs, val, A.col_idx);
    }
  }
  ring_end_pass<Tn>(sm, rs, next_val, A.col_idx);
  return true;
}

}  // namespace cgk
