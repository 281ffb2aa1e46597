// Device-side building blocks of the CG kernels: PTX wrappers for 1-D TMA
// bulk copies and mbarriers, deterministic reductions, the bounded grid
// barrier of the persistent solve, and the CSR product fed by a TMA ring.
#pragma once
#include <cstdint>
#include <type_traits>
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

// The same copy with an L2 eviction policy (createpolicy): used for data read
// once per pass, so that it does not push reused data out of L2.
__device__ __forceinline__ void bulk_g2s_hint(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                              uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
      : "memory");
}

__device__ __forceinline__ uint64_t l2_evict_first_policy() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
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



__device__ __forceinline__ int ld_volatile_i32(const int32_t* p) {
  return *reinterpret_cast<const volatile int32_t*>(p);
}

// Barrier of the consumer warps only (named barrier 1): the producer warp of
// a solve CTA never takes part in CTA-wide synchronisation.
__device__ __forceinline__ void cta_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(kConsumers) : "memory");
}

// AND of a per-thread condition over the consumer warps (named barrier 1).
// Every consumer thread must reach it; used after each product pass so that a
// warp that gave up on a wait and the others leave the kernel together.
__device__ __forceinline__ bool cta_and(bool v) {
  int r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.s32 p, %1, 0;\n\t"
      "bar.red.and.pred q, 1, %2, p;\n\t"
      "selp.s32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"(static_cast<int>(v)), "n"(kConsumers)
      : "memory");
  return r != 0;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
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

// -------------------------------------------- warp-level fixed-point sums

// A partial of an exact fixed-point sum: the integer m at scale 2^(e - 1074),
// e being the largest biased exponent among the values summed; nf: a NaN or
// an infinity was among them.
struct FxPart {
  long long m;
  int32_t e;
  int32_t nf;
};

// Sum over the warp of one double per lane, exactly, in fixed point at the
// warp's largest exponent E (spacing 2^(E-1074), about 2^-51 of the largest
// value; 32 values leave ample headroom).  Every lane gets the same result.
__device__ __forceinline__ FxPart fx_warp(double v) {
  const unsigned long long bits = static_cast<unsigned long long>(__double_as_longlong(v));
  const int e = static_cast<int>((bits >> 52) & 0x7ffull);
  const int E = static_cast<int>(__reduce_max_sync(0xffffffffu, static_cast<unsigned int>(e)));
  const int nf = __any_sync(0xffffffffu, e == 0x7ff);
  long long m = 0;
  if (e != 0 && !nf) {
    const int s = E - e + 1;  // >= 1
    if (s < 64) {
      const unsigned long long M = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
      const unsigned long long rnd = (M + (1ull << (s - 1))) >> s;
      m = (bits >> 63) ? -static_cast<long long>(rnd) : static_cast<long long>(rnd);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m += __shfl_xor_sync(0xffffffffu, m, o);
  return FxPart{m, E, nf};
}

// Sum of up to 32 partials, one per lane (`valid` lanes), realigned to the
// largest exponent (each partial rounded once, to nearest, ties away from
// zero) and converted to double once.  The result depends only on the
// partials, not on their order.  Every lane gets it.
__device__ __forceinline__ double fx_combine(FxPart p, bool valid) {
  const int E = static_cast<int>(__reduce_max_sync(0xffffffffu, valid ? static_cast<unsigned int>(p.e) : 0u));
  const int nf = __any_sync(0xffffffffu, valid && p.nf);
  long long m = 0;
  if (valid && p.m != 0) {
    const int d = E - p.e;  // >= 0
    if (d == 0) {
      m = p.m;
    } else if (d < 63) {
      const long long a = p.m < 0 ? -p.m : p.m;
      const long long r = (a + (1ll << (d - 1))) >> d;
      m = p.m < 0 ? -r : r;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m += __shfl_xor_sync(0xffffffffu, m, o);
  if (nf) return __longlong_as_double(0x7ff8000000000000ll);
  if (E == 0) return 0.0;
  return ldexp(static_cast<double>(m), E - 1074);
}

// Exact fixed-point sum, over the calling warp, of src[0 .. count), read
// through L2 (values written by other CTAs); lane j takes entries j, j + 32,
// ...; count <= 1024 keeps the integer sum within 63 bits.  The loads of a
// batch of 8 entries per lane are all issued before any is used (one L2
// round trip for up to 256 entries); the batch stays in registers for both
// steps (the largest exponent, then the rounded integers).  Every lane gets
// the result.
__device__ __forceinline__ double fx_warp_sum_array(const double* src, int count) {
  constexpr int kB = 8;
  const int lane = threadIdx.x & 31;
  long long m = 0;
  int E = 0, nf = 0;
  // the exponent of the whole array first (so that all batches share one grid)
  {
    unsigned int emax = 0;
    int nfl = 0;
    for (int j0 = 0; j0 < count; j0 += 32 * kB) {
      double v[kB];
#pragma unroll
      for (int u = 0; u < kB; ++u) {
        const int j = j0 + lane + 32 * u;
        v[u] = j < count ? __ldcg(src + j) : 0.0;
      }
#pragma unroll
      for (int u = 0; u < kB; ++u) {
        const unsigned long long bits = static_cast<unsigned long long>(__double_as_longlong(v[u]));
        const unsigned int e = static_cast<unsigned int>((bits >> 52) & 0x7ffull);
        emax = e > emax ? e : emax;
        nfl |= (e == 0x7ffu);
      }
      if (j0 + 32 * kB >= count) {
        // last (usually only) batch: sum it from the registers
        E = static_cast<int>(__reduce_max_sync(0xffffffffu, emax));
        nf = __any_sync(0xffffffffu, nfl);
        if (j0 == 0 && !nf) {
#pragma unroll
          for (int u = 0; u < kB; ++u) {
            const unsigned long long bits = static_cast<unsigned long long>(__double_as_longlong(v[u]));
            const int e = static_cast<int>((bits >> 52) & 0x7ffull);
            const int sh = E - e + 1;
            if (e != 0 && sh < 64) {
              const unsigned long long M = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
              const unsigned long long rnd = (M + (1ull << (sh - 1))) >> sh;
              m += (bits >> 63) ? -static_cast<long long>(rnd) : static_cast<long long>(rnd);
            }
          }
        }
      }
    }
  }
  if (count > 32 * kB && !nf) {
    // more than one batch: a second pass over the array at the common grid
    for (int j0 = 0; j0 < count; j0 += 32 * kB) {
      double v[kB];
#pragma unroll
      for (int u = 0; u < kB; ++u) {
        const int j = j0 + lane + 32 * u;
        v[u] = j < count ? __ldcg(src + j) : 0.0;
      }
#pragma unroll
      for (int u = 0; u < kB; ++u) {
        const unsigned long long bits = static_cast<unsigned long long>(__double_as_longlong(v[u]));
        const int e = static_cast<int>((bits >> 52) & 0x7ffull);
        const int sh = E - e + 1;
        if (e != 0 && sh < 64) {
          const unsigned long long M = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
          const unsigned long long rnd = (M + (1ull << (sh - 1))) >> sh;
          m += (bits >> 63) ? -static_cast<long long>(rnd) : static_cast<long long>(rnd);
        }
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m += __shfl_xor_sync(0xffffffffu, m, o);
  if (nf) return __longlong_as_double(0x7ff8000000000000ll);
  if (E == 0) return 0.0;
  return ldexp(static_cast<double>(m), E - 1074);
}

// Arrival and bounded wait of thread 0 at the group barrier of a system
// (the caller synchronises its own CTA around it).  `target` is the CTA's
// running target (in shared memory: thread 0 alone keeps it).  The arrival is
// a release pattern (an acq_rel fence, cumulative over what the CTA wrote
// before the CTA barrier that precedes it, then a relaxed add); the wait
// polls with relaxed loads and ends with an acquire pattern (an acq_rel
// fence).  These fences are lighter than the sequentially consistent one of
// __threadfence().  Returns false after a wait longer than limit_ns or an
// abort raised by another CTA.
__device__ __forceinline__ bool group_barrier_t0(SolveCtrl* ctrl, unsigned long long* target, unsigned int count,
                                                 unsigned long long limit_ns, int site) {
  *target += count;
  if (count <= 1) return true;
  asm volatile("fence.acq_rel.gpu;" ::: "memory");
  asm volatile("red.relaxed.gpu.global.add.u64 [%0], %1;" ::"l"(&ctrl->barrier), "l"(1ull) : "memory");
  unsigned long long t0 = 0;
  uint32_t spins = 0;
  const unsigned long long tgt = *target;
  for (;;) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(&ctrl->barrier) : "memory");
    if (v >= tgt) break;
    if ((++spins & 255u) == 0) {
      if (*reinterpret_cast<const volatile int32_t*>(&ctrl->abort)) return false;
      const unsigned long long now = global_timer_ns();
      if (t0 == 0) t0 = now;
      else if (now - t0 > limit_ns) {
        atomicExch(&ctrl->abort, 1);
        atomicExch(&ctrl->timeout_site, site);
        return false;
      }
    }
  }
  asm volatile("fence.acq_rel.gpu;" ::: "memory");
  return true;
}

// ------------------------------------------------------ streamed CSR product

// Per-CTA state of a solve, in shared memory: written by thread 0 (between
// CTA barriers), read by all.  Keeping it out of registers leaves the
// product in the step loop the registers it needs.
struct CtaState {
  double rho;                  // r.z (r.r without a preconditioner)
  double rr;                   // r.r of the current iterate
  double bnorm2;               // b.b
  double thresh2;              // tol^2 b.b
  double alpha, beta;
  long long k;                 // steps done
  long long k_end;             // last step of this launch
  unsigned long long target;   // group-barrier target of this CTA
  int32_t slot;                // partial-sum slot of the next group sum
  int32_t site;                // diagnostics: group waits so far
  int32_t ok;                  // the last group sum or barrier succeeded
  int32_t flags;               // kFlag* below
  int32_t dep_lo, dep_hi;      // CTAs whose rows this CTA's columns reach (columns first, then ranks)
};
enum : int32_t { kFlagDone = 1, kFlagBreakdown = 2, kFlagReplace = 4, kFlagResumed = 8 };

// Warp partials of a CTA sum (up to three values per thread) and each
// warp's vote.
constexpr int kMaxSumValues = 3;
struct SumScratch {
  FxPart part[kMaxSumValues][kWarps];
  int32_t ok[kWarps];
};

// Dynamic shared memory of a persistent CTA: the value ring (values of vb
// bytes: 8 for FP64, 4 for FP32, so that an FP32 stream leaves more of the
// SM's 256 KB to L1 for the gathers) and the column-index ring, each followed
// by its kMirror-entry mirror, the full/empty mbarriers of every slot, the
// CTA state of a solve, the warp partials of its sums, a few words (stop
// flag), and in the small-share solve the r of the CTA's rows.
struct RingSmem {
  static constexpr int kRingAlloc = kRing + kMirror;
  static constexpr size_t kColBytes = sizeof(int32_t) * kRingAlloc;
  static constexpr size_t kStateBytes = (sizeof(CtaState) + 15) & ~size_t(15);
  static constexpr size_t kSumBytes = (sizeof(SumScratch) + 15) & ~size_t(15);
  __host__ __device__ static constexpr size_t bar_off(size_t vb) {
    return (vb * kRingAlloc + kColBytes + 15) & ~size_t(15);
  }
  __host__ __device__ static constexpr size_t state_off(size_t vb) { return bar_off(vb) + 16 * kSlots; }
  __host__ __device__ static constexpr size_t sum_off(size_t vb) { return state_off(vb) + kStateBytes; }
  __host__ __device__ static constexpr size_t misc_off(size_t vb) { return sum_off(vb) + kSumBytes; }
  // Bytes of the whole layout for ring values of vb bytes.
  __host__ __device__ static constexpr size_t bytes(size_t vb) { return misc_off(vb) + 64; }

  unsigned char* base;
  uint32_t vb = sizeof(double);  // bytes per value in the ring
  template <typename T>
  __device__ T* val() const { return reinterpret_cast<T*>(base); }
  __device__ int32_t* col() const { return reinterpret_cast<int32_t*>(base + static_cast<size_t>(vb) * kRingAlloc); }
  __device__ uint64_t* full(int s) const { return reinterpret_cast<uint64_t*>(base + bar_off(vb)) + s; }
  __device__ uint64_t* empty(int s) const { return reinterpret_cast<uint64_t*>(base + bar_off(vb)) + kSlots + s; }
  __device__ CtaState* state() const { return reinterpret_cast<CtaState*>(base + state_off(vb)); }
  __device__ SumScratch* sums() const { return reinterpret_cast<SumScratch*>(base + sum_off(vb)); }
  __device__ int32_t* flag() const { return reinterpret_cast<int32_t*>(base + misc_off(vb)); }
  __device__ int32_t* stop() const { return reinterpret_cast<int32_t*>(base + misc_off(vb) + 4); }
  __device__ double* scalars() const { return reinterpret_cast<double*>(base + misc_off(vb) + 16); }
  // r of the CTA's rows in a small-share solve, behind the layout
  // (kLocalRows entries).
  __device__ double* local() const { return reinterpret_cast<double*>(base + bytes(vb)); }
};

// Dynamic shared memory of the kernels whose step-loop product streams
// values of type T; `local`: with the small-share solve's r.
template <typename T>
constexpr size_t ring_smem_bytes(bool local = false) {
  return RingSmem::bytes(sizeof(T)) + (local ? sizeof(double) * kLocalRows : 0);
}

// The CTA's part of the matrix stream (identical in every thread).  Pieces
// are numbered globally across passes (piece j of pass k is k * npieces + j);
// global piece g sits in slot g % kSlots and completes phase g / kSlots of
// that slot's full barrier.
struct CtaStream {
  int kb = 0;        // first entry of the CTA's range, rounded down to a multiple of 4
  int ke = 0;        // end of the CTA's entry range
  int npieces = 0;   // pieces per pass
  int s0 = 0, s1 = 0;  // the CTA's steps [s0, s1)
};

__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Initialise the ring barriers for the CTA's share `rank` of A's partition
// (all threads of the CTA call; ends with a full CTA barrier).  `reinit`:
// the barriers hold a previous stream, already drained (a CTA taking another
// task of a batched solve); they are invalidated first.
__device__ __forceinline__ void stream_setup(const RingSmem& sm, CtaStream& cs, const DevCsr& A, int rank,
                                             bool reinit = false) {
  if (threadIdx.x < kSlots) {
    if (reinit) {
      mbar_inval(sm.full(threadIdx.x));
      mbar_inval(sm.empty(threadIdx.x));
    }
    mbar_init(sm.full(threadIdx.x), 1);
    mbar_init(sm.empty(threadIdx.x), kConsumerWarps);
  }
  if (threadIdx.x == 0) *sm.stop() = 0;
  if (threadIdx.x < kSlots) fence_mbar_init();
  __syncthreads();
  cs.s0 = A.block_step[rank];
  cs.s1 = A.block_step[rank + 1];
  cs.kb = cs.ke = cs.npieces = 0;
  if (cs.s1 > cs.s0) {
    cs.kb = A.step[cs.s0].z & ~3;
    cs.ke = A.step[cs.s1 - 1].w;
    cs.npieces = (cs.ke - cs.kb + kPiece - 1) >> kPieceLog;
  }
}

// Bounded wait on an mbarrier phase; false if it gave up.  If `stop` is
// given, also gives up as soon as *stop becomes non-zero.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, unsigned long long limit_ns,
                                                  const int32_t* stop) {
  uint32_t spins = 0;
  unsigned long long t0 = 0;
  while (!mbar_try_wait(bar, parity)) {
    if ((++spins & 63u) == 0) {
      if (stop && ld_volatile_i32(stop)) return false;
      const unsigned long long now = global_timer_ns();
      if (t0 == 0) t0 = now;
      else if (now - t0 > limit_ns) return false;
    }
  }
  return true;
}

// Producer (one lane of the producer warp): stream the CTA's range pass after
// pass (max_passes < 0: until told to stop) with values of type T.  Before
// refilling a slot it waits for every consumer warp to release the slot's
// previous piece.  On stop it waits for its copies still in flight, so no
// bulk copy lands after the CTA is gone.  Returns false on a timeout.
template <typename T>
__device__ __forceinline__ bool producer_loop(const RingSmem& sm, const CtaStream& cs, const T* val,
                                              const int32_t* col, int max_passes, unsigned long long limit_ns) {
  bool ok = true;
  uint32_t g = 0;
  const uint64_t pol = l2_evict_first_policy();
  if (cs.npieces > 0) {
    const int ke4 = (cs.ke + 3) & ~3;  // copy whole 16-byte groups (<= 3 padding entries)
    for (int pass = 0; ok && (max_passes < 0 || pass < max_passes); ++pass) {
      for (int j = 0; j < cs.npieces; ++j, ++g) {
        const int slot = static_cast<int>(g % kSlots);
        if (g >= kSlots && !mbar_wait_bounded(sm.empty(slot), ((g / kSlots) - 1) & 1u, limit_ns, sm.stop())) {
          ok = ld_volatile_i32(sm.stop()) != 0;  // a stop is the normal way out
          goto drain;
        }
        const int e0 = cs.kb + j * kPiece;
        const int e1 = e0 + kPiece < ke4 ? e0 + kPiece : ke4;
        const int pos = slot * kPiece;
        const uint32_t bv = static_cast<uint32_t>(e1 - e0) * sizeof(T);
        const uint32_t bc = static_cast<uint32_t>(e1 - e0) * 4u;
        // slot 0 also fills the mirror behind the ring end with its first entries
        const int nm = slot == 0 ? (e1 - e0 < kMirror ? e1 - e0 : kMirror) : 0;  // a multiple of 4
        const uint32_t mv = static_cast<uint32_t>(nm) * sizeof(T), mc = static_cast<uint32_t>(nm) * 4u;
        mbar_arrive_expect_tx(sm.full(slot), bv + bc + mv + mc);
        bulk_g2s_hint(sm.val<T>() + pos, val + e0, bv, sm.full(slot), pol);
        bulk_g2s_hint(sm.col() + pos, col + e0, bc, sm.full(slot), pol);
        if (nm) {
          bulk_g2s_hint(sm.val<T>() + kRing, val + e0, mv, sm.full(slot), pol);
          bulk_g2s_hint(sm.col() + kRing, col + e0, mc, sm.full(slot), pol);
        }
      }
    }
  }
drain:
  // the newest piece of every slot may still be in flight
  for (uint32_t k = g > kSlots ? g - kSlots : 0; k < g; ++k)
    mbar_wait_bounded(sm.full(k % kSlots), (k / kSlots) & 1u, limit_ns, nullptr);
  return ok;
}

// Consumer-side position of the CTA in the stream (identical in all
// consumer threads): global number of piece 0 of the next ring pass.
struct ConsumerCursor {
  uint32_t gbase = 0;
};

// Gathers of one lane's row segment: xv[u] = x[cp[u]] for its len entries,
// cp pointing at the segment's column indices in the ring (contiguous thanks
// to the mirror).  N is the step's longest per-lane segment (lanes with a
// shorter segment, or none, are predicated off for the tail), so the code is
// branch-free and no instruction is issued for a slot no lane needs.
template <typename X, int N, int U>
__device__ __forceinline__ void seg_gather_n(const int32_t* cp, int len, const X* x, X (&xv)[U]) {
#pragma unroll
  for (int u = 0; u < N; ++u)
    if (u < len) xv[u] = x[cp[u]];
}

// Multiply-adds of a gathered segment, in storage order, with FMA.
template <typename T, typename X, typename Acc, int N, int U>
__device__ __forceinline__ Acc seg_fma_n(const T* vp, int len, const X (&xv)[U], Acc s) {
#pragma unroll
  for (int u = 0; u < N; ++u)
    if (u < len) s = fma(Acc(vp[u]), Acc(xv[u]), s);
  return s;
}

// The step's longest per-lane segment (1..32) selects the unrolled code once
// per step (dispatch_tree below).

// The multiply-adds of a lane's first 16 entries (xv holds their gathered
// values), each followed by the gather of entry 16 + u into the register it
// frees (N2 = entries of the second batch the step needs, at most 16): the
// second batch's loads are in flight during the first batch's FMA chain.
template <typename T, typename X, typename Acc, int N2>
__device__ __forceinline__ Acc seg_fma_refill_n(const T* vp, const int32_t* cp2, int len, const X* x, X (&xv)[16]) {
  Acc s = Acc(0);
#pragma unroll
  for (int u = 0; u < 16; ++u) {
    if (u < len) s = fma(Acc(vp[u]), Acc(xv[u]), s);
    if (u < N2 && 16 + u < len) xv[u] = x[cp2[u]];
  }
  return s;
}

// Calls f(std::integral_constant<int, v>) for v in [LO, HI] (values below LO
// call f with LO) through a binary tree of warp-uniform conditional branches:
// no indirect jump (a jump table's target must be resolved before the warp
// can go on).
template <int LO, int HI, typename F>
__device__ __forceinline__ void dispatch_tree(int v, F&& f) {
  if constexpr (LO == HI) {
    f(std::integral_constant<int, LO>{});
  } else {
    constexpr int MID = (LO + HI) / 2;
    if (v <= MID) dispatch_tree<LO, MID>(v, f);
    else dispatch_tree<MID + 1, HI>(v, f);
  }
}

template <typename T, typename X, typename Acc>
__device__ __forceinline__ Acc seg_fma_refill(const T* vp, const int32_t* cp2, int len, int n2, const X* x,
                                              X (&xv)[16]) {
  Acc s = Acc(0);
  dispatch_tree<1, 16>(n2, [&](auto N) { s = seg_fma_refill_n<T, X, Acc, decltype(N)::value>(vp, cp2, len, x, xv); });
  return s;
}

template <typename X, int U>
__device__ __forceinline__ void seg_gather(const int32_t* cp, int len, int wmax, const X* x, X (&xv)[U]) {
  static_assert(U == 32 || U == 16, "dispatch covers 1..U");
  dispatch_tree<1, U>(wmax, [&](auto N) { seg_gather_n<X, decltype(N)::value, U>(cp, len, x, xv); });
}

template <typename T, typename X, typename Acc, int U>
__device__ __forceinline__ Acc seg_fma(const T* vp, int len, int wmax, const X (&xv)[U], Acc s) {
  static_assert(U == 32 || U == 16, "dispatch covers 1..U");
  dispatch_tree<1, U>(wmax, [&](auto N) { s = seg_fma_n<T, X, Acc, decltype(N)::value, U>(vp, len, xv, s); });
  return s;
}

// A segment longer than the unrolled capacity (up to kMirror entries: rows of
// 17..64 entries split over two lanes), contiguous in the ring: gathers and
// multiply-adds 8 at a time.
template <typename T, typename X, typename Acc>
__device__ __forceinline__ Acc seg_dot_loop(const T* vp, const int32_t* cp, int len, const X* x) {
  Acc s = Acc(0);
  int t = 0;
  for (; t + 8 <= len; t += 8) {
    X xv[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) xv[u] = x[cp[t + u]];
#pragma unroll
    for (int u = 0; u < 8; ++u) s = fma(Acc(vp[t + u]), Acc(xv[u]), s);
  }
  for (; t < len; ++t) s = fma(Acc(vp[t]), Acc(x[cp[t]]), s);
  return s;
}

// Lane-private part of a lane-per-row or pair-per-row step.  The row
// pointers are loaded when a step is two steps ahead and only consumed one
// step later, so their latency stays off the critical path.  *stream != 0:
// load them with the evict-first policy (__ldcs), so that in a solve whose
// vectors and row pointers together outgrow the L2 the row pointers, read
// once per product, give way to the vectors that the step reads again.  The
// flag is read where it is used (a kernel parameter or an L1 hit) rather
// than held in a register through the product.
struct LaneRaw {
  int row;   // row whose (partial) sum this lane computes, -1 if none
  int ks;    // row_ptr[row]
  int ke;    // row_ptr[row + 1]
};

__device__ __forceinline__ LaneRaw lane_raw(const int32_t* row_ptr, int4 d, int mode, bool valid,
                                            const int32_t* stream) {
  const int lane = threadIdx.x & 31;
  LaneRaw r{-1, 0, 0};
  if (valid && mode != kLongRow) {
    const int i = d.x + (mode == kLanePerRow ? lane : (lane >> 1));
    if (i < d.y) {
      r.row = i;
      if (*stream) {
        r.ks = __ldcs(row_ptr + i);
        r.ke = __ldcs(row_ptr + i + 1);
      } else {
        r.ks = row_ptr[i];
        r.ke = row_ptr[i + 1];
      }
    }
  }
  return r;
}

// This lane's entries [a, a + len) of its row (half of it in a pair step).
__device__ __forceinline__ void lane_span(const LaneRaw& r, int mode, int& a, int& len) {
  if (r.row < 0) {
    a = 0;
    len = 0;
  } else if (mode == kLanePerRow) {
    a = r.ks;
    len = r.ke - r.ks;
  } else {
    const int half = (r.ke - r.ks + 1) >> 1;
    const bool second = threadIdx.x & 1;
    a = second ? r.ks + half : r.ks;
    len = second ? (r.ke - r.ks - half) : half;
  }
}

// The product over the CTA's steps with values `val` (type T), gathering x;
// consumer warp w computes steps s0 + w, s0 + w + kConsumerWarps, ...  Each
// row's result goes to epi(i, yi, aux[i]) from one lane (aux[i] = 0 when aux
// is nullptr).  kRingPass: entries come from the ring (the producer streams
// them; the warp waits on the full barrier of the pieces a step spans and
// releases pieces on the empty barriers once its next step starts beyond
// them); otherwise entries are read directly from global memory (values
// `val`, column indices A.col_idx).  Step descriptors are loaded two steps
// ahead, row pointers and aux values one step ahead; *stream_rows != 0: row
// pointers with the evict-first policy (lane_raw).  Returns false
// (uniformly over the warp) if a wait gave up.
template <bool kRingPass, typename T, typename X, typename Acc, typename Epi>
__device__ __forceinline__ bool spmv_pass(const RingSmem& sm, const CtaStream& cs, ConsumerCursor& cur,
                                          const DevCsr& A, const T* val, const X* x, const double* aux, Epi& epi,
                                          unsigned long long limit_ns, const int32_t* stream_rows) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const T* rv = kRingPass ? sm.val<T>() : val;
  const int32_t* rc = kRingPass ? sm.col() : A.col_idx;
  const int32_t* row_ptr = A.row_ptr;
  const uint32_t gbase = cur.gbase;
  // entry k sits at rv[pos(k)]: in the ring at (k + off) & kRingMask
  const int off = static_cast<int>((gbase % kSlots) * kPiece) - cs.kb;
  auto pos = [&](int k) { return kRingPass ? ((k + off) & kRingMask) : k; };
  auto wait_piece = [&](int j) {
    const uint32_t g = gbase + static_cast<uint32_t>(j);
    return __all_sync(0xffffffffu, mbar_wait_bounded(sm.full(g % kSlots), (g / kSlots) & 1u, limit_ns, nullptr));
  };
  int released = 0;  // pieces of this pass this warp has released
  auto release_upto = [&](int upto) -> bool {
    for (; released < upto; ++released) {
      if (!wait_piece(released)) return false;  // the piece must be the slot's current one
      __syncwarp();
      if (lane == 0) mbar_arrive(sm.empty((gbase + static_cast<uint32_t>(released)) % kSlots));
    }
    return true;
  };
  auto sd = [&](int k) { return k < A.nsteps + 2 ? k : A.nsteps + 1; };  // two sentinels follow the last step
  auto holds_result = [&](int mode, const LaneRaw& r) {
    return r.row >= 0 && (mode == kLanePerRow || (lane & 1) == 0);
  };
  constexpr int kStride = kConsumerWarps;
  int s = cs.s0 + w;
  int4 d0 = A.step[sd(s)], d1 = A.step[sd(s + kStride)];
  int m0 = A.step_mode[sd(s)], m1 = A.step_mode[sd(s + kStride)];
  LaneRaw r0 = lane_raw(row_ptr, d0, m0 & 3, s < cs.s1, stream_rows);
  double a0 = (aux != nullptr && s < cs.s1 && holds_result(m0 & 3, r0)) ? aux[r0.row] : 0.0;
  for (; s < cs.s1; s += kStride) {
    const bool has1 = s + kStride < cs.s1;
    // prefetch: descriptor two steps ahead, row pointers and aux value of the next step
    const int4 d2 = A.step[sd(s + 2 * kStride)];
    const int m2 = A.step_mode[sd(s + 2 * kStride)];
    const LaneRaw r1 = lane_raw(row_ptr, d1, m1 & 3, has1, stream_rows);
    const double a1 = (aux != nullptr && has1 && holds_result(m1 & 3, r1)) ? aux[r1.row] : 0.0;
    const int mode = m0 & 3;
    if (kRingPass && d0.w > d0.z) {
      // release what lies before this step; a short step then waits for the
      // (at most two) pieces it spans
      if (!release_upto((d0.z - cs.kb) >> kPieceLog)) return false;
      if (mode != kLongRow) {
        const int jh = (d0.w - 1 - cs.kb) >> kPieceLog;
        for (int j = (d0.z - cs.kb) >> kPieceLog; j <= jh; ++j)
          if (!wait_piece(j)) return false;
      }
    }
    if (mode == kLongRow) {
      // lanes stride the row; in a ring pass piece by piece, each piece
      // released once done (the warp's next step starts after this row)
      Acc acc = Acc(0);
      if (kRingPass) {
        const int jl = (d0.z - cs.kb) >> kPieceLog, jh = (d0.w - 1 - cs.kb) >> kPieceLog;
        for (int j = jl; j <= jh; ++j) {
          if (!wait_piece(j)) return false;
          const int lo = max(d0.z, cs.kb + j * kPiece), hi = min(d0.w, cs.kb + (j + 1) * kPiece);
          for (int k = lo + lane; k < hi; k += 32) {
            const int p = pos(k);
            acc = fma(Acc(rv[p]), Acc(x[rc[p]]), acc);
          }
          if (j < jh && !release_upto(j + 1)) return false;
        }
      } else {
        for (int k = d0.z + lane; k < d0.w; k += 32) acc = fma(Acc(rv[k]), Acc(x[rc[k]]), acc);
      }
      Acc tot;
      if constexpr (sizeof(Acc) == 8) tot = warp_sum(acc);
      else tot = warp_sum_f(acc);
      if (lane == 0) epi(d0.x, tot, aux != nullptr ? aux[d0.x] : 0.0);
    } else {
      int a, len;
      lane_span(r0, mode, a, len);
      const int p0 = pos(a);
      Acc part;
      if constexpr (kRingPass) {
        const int wmax = (m0 >> kWmaxShift) & 0xff;
        if constexpr (sizeof(X) == 8) {
          // FP64 gathers in batches of 16 (the same FMAs in the same order;
          // half the registers held by gathered values); the second batch is
          // loaded during the first batch's FMAs
          X xv[16];
          const int w0 = wmax < 16 ? wmax : 16;
          seg_gather<X, 16>(rc + p0, len, w0, x, xv);
          if (wmax > 16) {
            part = seg_fma_refill<T, X, Acc>(rv + p0, rc + p0 + 16, len, wmax - 16, x, xv);
            part = seg_fma<T, X, Acc, 16>(rv + p0 + 16, len - 16, wmax - 16, xv, part);
          } else {
            part = seg_fma<T, X, Acc, 16>(rv + p0, len, w0, xv, Acc(0));
          }
        } else {
          X xv[kLaneMax];
          seg_gather<X, kLaneMax>(rc + p0, len, wmax, x, xv);
          part = seg_fma<T, X, Acc, kLaneMax>(rv + p0, len, wmax, xv, Acc(0));
        }
      } else {
        // the direct pass (rare: residual replacements) uses the compact
        // loop: the same FMAs in the same order, far fewer registers
        part = seg_dot_loop<T, X, Acc>(rv + p0, rc + p0, len, x);
      }
      if (mode == kPairPerRow) {
        // first half + second half: the same value in both lanes (commutative add)
        const Acc sum = part + __shfl_xor_sync(0xffffffffu, part, 1);
        if (holds_result(mode, r0)) epi(r0.row, sum, a0);
      } else if (holds_result(mode, r0)) {
        epi(r0.row, part, a0);
      }
    }
    d0 = d1; m0 = m1; r0 = r1; a0 = a1;
    d1 = d2; m1 = m2;
  }
  if (kRingPass) {
    if (!release_upto(cs.npieces)) return false;
    cur.gbase = gbase + static_cast<uint32_t>(cs.npieces);
  }
  return true;
}

}  // namespace cgk
