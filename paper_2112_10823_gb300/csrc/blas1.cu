// Vector kernels benchmarked by the paper (Sec. 5.2): dot product, addition
// of vectors (y <- a x + y) and element-wise product (z = x o y).  All three
// stream HBM; the dot product is deterministic for a given length (fixed grid,
// fixed per-thread order, fixed combine order).
#include "cg_device.cuh"

namespace cgk {

// Threads per CTA of the vector kernels.
constexpr int kVecBlock = 384;

// Grid of the dot kernel: enough CTAs to fill the GPU for long vectors, no
// more than needed for short ones.  Depends only on n and the SM count.
int dot_grid(int64_t n, int num_sms) {
  const int64_t per_cta = static_cast<int64_t>(kVecBlock) * 8;
  int64_t g = (n + per_cta - 1) / per_cta;
  const int64_t cap = static_cast<int64_t>(num_sms) * 4;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return static_cast<int>(g);
}

// Each thread sums x_i y_i over i = t, t + T, t + 2T, ... (T = threads in the
// grid, four independent accumulators combined in a fixed order), the CTA sums
// its threads, and the last CTA to finish adds the CTA partials in CTA order
// and resets the arrival counter for the next call.
__global__ void __launch_bounds__(kVecBlock) dot_kernel(int64_t n, const double* __restrict__ x,
                                                     const double* __restrict__ y, double* __restrict__ out,
                                                     double* __restrict__ partials, unsigned int* counter) {
  __shared__ double red[kVecBlock + 4];
  __shared__ unsigned int is_last;
  const int64_t T = static_cast<int64_t>(gridDim.x) * kVecBlock;
  int64_t i = static_cast<int64_t>(blockIdx.x) * kVecBlock + threadIdx.x;
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  for (; i + 3 * T < n; i += 4 * T) {
    a0 = fma(x[i], y[i], a0);
    a1 = fma(x[i + T], y[i + T], a1);
    a2 = fma(x[i + 2 * T], y[i + 2 * T], a2);
    a3 = fma(x[i + 3 * T], y[i + 3 * T], a3);
  }
  for (; i < n; i += T) a0 = fma(x[i], y[i], a0);
  double s = block_sum((a0 + a1) + (a2 + a3), red);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = s;
    __threadfence();
    const unsigned int ticket = atomicAdd(counter, 1u);
    is_last = (ticket == gridDim.x - 1) ? 1u : 0u;
  }
  __syncthreads();
  if (is_last) {
    __threadfence();
    double t = 0.0;
    for (int j = threadIdx.x; j < static_cast<int>(gridDim.x); j += kVecBlock) t += __ldcg(partials + j);
    t = block_sum(t, red);
    if (threadIdx.x == 0) {
      *out = t;
      *counter = 0u;
    }
  }
}

cudaError_t launch_dot(int64_t n, const double* x, const double* y, double* out, double* partials,
                       unsigned int* counter, int grid, cudaStream_t s) {
  dot_kernel<<<grid, kVecBlock, 0, s>>>(n, x, y, out, partials, counter);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Streamed dot product: the kernel of cg_dot when x and y are 16-byte aligned
// and long enough.  One CTA per SM.  A producer warp copies chunks of x and y
// (kDotChunk elements each) into a ring of kDotSlots shared-memory slots with
// 1-D bulk copies, completion counted on each slot's "full" mbarrier; eight
// consumer warps read a slot with 16-byte shared loads, run one FMA per
// element into eight per-thread accumulators, and release the slot on its
// "empty" mbarrier.  The copy engine keeps up to kDotSlots * 32 KB in flight
// per SM whatever the consumers are doing, so the FP64 pipe (one FMA per 16
// bytes streamed: about two thirds of its peak at the HBM rate) and the
// memory stream overlap.  Chunk c goes to CTA c mod G; the elements past the
// last whole chunk to the last CTA.  Every thread sums its accumulators in a
// fixed order, the CTA in a fixed tree, the last CTA to finish the CTA sums in
// CTA order: the same bits for a given n.
constexpr int kDotWarps = 8;
constexpr int kDotThreads = (kDotWarps + 1) * 32;
constexpr int kDotChunk = 2048;
constexpr int kDotSlots = 4;
constexpr int kDotPerThread = kDotChunk / (kDotWarps * 32);  // 8 elements per slot and thread
static_assert(kDotPerThread == 8, "the consumer loop reads four double2 of x and of y per slot");
constexpr size_t kDotSmem = 2 * sizeof(double) * kDotChunk * kDotSlots + 16 * kDotSlots + 16;

int64_t dot_stream_min_n() { return static_cast<int64_t>(kDotChunk) * 16; }

__global__ void __launch_bounds__(kDotThreads, 1)
    dot_stream_kernel(int64_t n, const double* __restrict__ x, const double* __restrict__ y, double* __restrict__ out,
                      double* __restrict__ partials, unsigned int* counter, int32_t* err,
                      unsigned long long limit_ns) {
  extern __shared__ __align__(128) unsigned char dsm[];
  double* xs = reinterpret_cast<double*>(dsm);
  double* ys = xs + kDotChunk * kDotSlots;
  uint64_t* full = reinterpret_cast<uint64_t*>(ys + kDotChunk * kDotSlots);
  uint64_t* empty = full + kDotSlots;
  int32_t* stop = reinterpret_cast<int32_t*>(empty + kDotSlots);
  __shared__ double red[kDotThreads + 1];
  __shared__ unsigned int is_last;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t G = gridDim.x;
  const int64_t nchunks = n / kDotChunk;
  const uint32_t mine = nchunks > blockIdx.x ? static_cast<uint32_t>((nchunks - 1 - blockIdx.x) / G + 1) : 0u;
  if (threadIdx.x < kDotSlots) {
    mbar_init(&full[threadIdx.x], 1);
    mbar_init(&empty[threadIdx.x], kDotWarps);
  }
  if (threadIdx.x == 0) *stop = 0;
  if (threadIdx.x < kDotSlots) fence_mbar_init();
  __syncthreads();
  double acc = 0.0;
  if (warp == kDotWarps) {
    if (lane == 0) {
      constexpr uint32_t kBytes = kDotChunk * sizeof(double);
      uint32_t g = 0;
      for (; g < mine; ++g) {
        const int s = static_cast<int>(g % kDotSlots);
        if (g >= kDotSlots && !mbar_wait_bounded(&empty[s], ((g / kDotSlots) - 1) & 1u, limit_ns, stop)) break;
        const int64_t c = static_cast<int64_t>(blockIdx.x) + static_cast<int64_t>(g) * G;
        mbar_arrive_expect_tx(&full[s], 2 * kBytes);
        bulk_g2s(xs + s * kDotChunk, x + c * kDotChunk, kBytes, &full[s]);
        bulk_g2s(ys + s * kDotChunk, y + c * kDotChunk, kBytes, &full[s]);
      }
      // copies still in flight land before the CTA leaves
      for (uint32_t k = g > kDotSlots ? g - kDotSlots : 0; k < g; ++k)
        mbar_wait_bounded(&full[k % kDotSlots], (k / kDotSlots) & 1u, limit_ns, nullptr);
    }
  } else {
    double a[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (uint32_t g = 0; g < mine; ++g) {
      const int s = static_cast<int>(g % kDotSlots);
      if (!mbar_wait_bounded(&full[s], (g / kDotSlots) & 1u, limit_ns, stop)) {
        atomicExch(stop, 1);
        break;
      }
      const double2* xv = reinterpret_cast<const double2*>(xs + s * kDotChunk);
      const double2* yv = reinterpret_cast<const double2*>(ys + s * kDotChunk);
      double2 u[4], v[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        u[j] = xv[threadIdx.x + kDotWarps * 32 * j];
        v[j] = yv[threadIdx.x + kDotWarps * 32 * j];
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[s]);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        a[2 * j] = fma(u[j].x, v[j].x, a[2 * j]);
        a[2 * j + 1] = fma(u[j].y, v[j].y, a[2 * j + 1]);
      }
    }
    if (blockIdx.x == G - 1)
      for (int64_t i = nchunks * kDotChunk + threadIdx.x; i < n; i += kDotWarps * 32) a[0] = fma(x[i], y[i], a[0]);
    acc = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
  }
  double s = block_sum(acc, red);
  if (threadIdx.x == 0) {
    if (ld_volatile_i32(stop)) atomicExch(err, 1);
    partials[blockIdx.x] = s;
    __threadfence();
    const unsigned int ticket = atomicAdd(counter, 1u);
    is_last = (ticket == gridDim.x - 1) ? 1u : 0u;
  }
  __syncthreads();
  if (is_last) {
    __threadfence();
    double t = 0.0;
    for (int j = threadIdx.x; j < static_cast<int>(gridDim.x); j += kDotThreads) t += __ldcg(partials + j);
    t = block_sum(t, red);
    if (threadIdx.x == 0) {
      // err[0]: raised by any CTA of this call; err[1]: the outcome of the
      // last call (read by the host after a synchronising call).  Both
      // words are left ready for the next call, like the counter.
      const int32_t bad = __ldcg(err);
      err[1] = bad;
      err[0] = 0;
      *out = bad ? __longlong_as_double(0x7ff8000000000000ll) : t;
      *counter = 0u;
    }
  }
}

cudaError_t launch_dot_stream(int64_t n, const double* x, const double* y, double* out, double* partials,
                              unsigned int* counter, int32_t* err, int grid, unsigned long long limit_ns,
                              cudaStream_t s) {
  cudaError_t e = ensure_smem_attr(reinterpret_cast<const void*>(dot_stream_kernel), kDotSmem);
  if (e != cudaSuccess) return e;
  dot_stream_kernel<<<grid, kDotThreads, kDotSmem, s>>>(n, x, y, out, partials, counter, err, limit_ns);
  return cudaGetLastError();
}

// Grid of the streamed dot product: one CTA per SM, fewer if there are fewer
// whole chunks.
int dot_stream_grid(int64_t n, int num_sms) {
  const int64_t nchunks = n / kDotChunk;
  int64_t g = nchunks < num_sms ? nchunks : num_sms;
  return g < 1 ? 1 : static_cast<int>(g);
}

// ---------------------------------------------------------------------------
// FP64 multiply-add throughput probe (the ceiling of the ALU roofline): every
// thread runs eight independent FMA chains a = a * m + c, whose fixed point is
// c / (1 - m) = 1, so the values stay finite; the sum is stored only if it
// takes a value it cannot take, which keeps the compiler from dropping the
// work without writing anything.  m and c are moved into registers first
// (adding 1e-300 * threadIdx.x changes neither value but hides that from
// the compiler): with an operand read from the constant bank, FMAs issue at
// only 1.68 per clock per SM on GB300 instead of 2.
__global__ void __launch_bounds__(256) fp64_probe_kernel(int64_t iters, double m_in, double c_in, double* sink) {
  const double m = m_in + 1e-300 * threadIdx.x, c = c_in + 1e-300 * blockIdx.x;
  double a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = 0.5 + 1e-3 * k + 1e-9 * threadIdx.x;
  // 32 FMAs per trip of the loop, so its counter and branch are a small
  // share of the issued instructions
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
#pragma unroll
      for (int k = 0; k < 8; ++k) a[k] = fma(a[k], m, c);
    }
  }
  const double t = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
  if (t == -1.0) sink[blockIdx.x] = t;
}


cudaError_t launch_fp64_probe(int64_t iters, int grid, double* sink, cudaStream_t s) {
  fp64_probe_kernel<<<grid, 256, 0, s>>>(iters, 1.0 - 1.0 / 1024.0, 1.0 / 1024.0, sink);
  return cudaGetLastError();
}

namespace {
inline int stream_grid(int64_t n) {
  int dev = 0, sms = 148;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t want = (n / 2 + kVecBlock - 1) / kVecBlock;
  const int64_t cap = static_cast<int64_t>(sms) * 8;
  int64_t g = want < cap ? want : cap;
  return g < 1 ? 1 : static_cast<int>(g);
}
inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }
}  // namespace

// y <- a x + y.  Pairs of elements move as 16-byte loads/stores when both
// vectors are 16-byte aligned; otherwise element by element.
template <bool kVec>
__global__ void __launch_bounds__(kVecBlock) axpy_kernel(int64_t n, double a, const double* __restrict__ x,
                                                      double* __restrict__ y) {
  const int64_t T = static_cast<int64_t>(gridDim.x) * kVecBlock;
  int64_t t = static_cast<int64_t>(blockIdx.x) * kVecBlock + threadIdx.x;
  if constexpr (kVec) {
    const int64_t n2 = n / 2;
    const double2* x2 = reinterpret_cast<const double2*>(x);
    double2* y2 = reinterpret_cast<double2*>(y);
    for (int64_t i = t; i < n2; i += T) {
      const double2 xv = x2[i];
      double2 yv = y2[i];
      yv.x = fma(a, xv.x, yv.x);
      yv.y = fma(a, xv.y, yv.y);
      y2[i] = yv;
    }
    if (t == 0 && (n & 1)) y[n - 1] = fma(a, x[n - 1], y[n - 1]);
  } else {
    for (int64_t i = t; i < n; i += T) y[i] = fma(a, x[i], y[i]);
  }
}

template <bool kVec>
__global__ void __launch_bounds__(kVecBlock) ewmul_kernel(int64_t n, const double* x, const double* y,
                                                       double* z) {  // z may alias x or y
  const int64_t T = static_cast<int64_t>(gridDim.x) * kVecBlock;
  int64_t t = static_cast<int64_t>(blockIdx.x) * kVecBlock + threadIdx.x;
  if constexpr (kVec) {
    const int64_t n2 = n / 2;
    const double2* x2 = reinterpret_cast<const double2*>(x);
    const double2* y2 = reinterpret_cast<const double2*>(y);
    double2* z2 = reinterpret_cast<double2*>(z);
    for (int64_t i = t; i < n2; i += T) {
      const double2 xv = x2[i], yv = y2[i];
      z2[i] = make_double2(xv.x * yv.x, xv.y * yv.y);
    }
    if (t == 0 && (n & 1)) z[n - 1] = x[n - 1] * y[n - 1];
  } else {
    for (int64_t i = t; i < n; i += T) z[i] = x[i] * y[i];
  }
}

cudaError_t launch_axpy(int64_t n, double a, const double* x, double* y, cudaStream_t s) {
  const int g = stream_grid(n);
  if (aligned16(x) && aligned16(y)) axpy_kernel<true><<<g, kVecBlock, 0, s>>>(n, a, x, y);
  else axpy_kernel<false><<<g, kVecBlock, 0, s>>>(n, a, x, y);
  return cudaGetLastError();
}

cudaError_t launch_ewmul(int64_t n, const double* x, const double* y, double* z, cudaStream_t s) {
  const int g = stream_grid(n);
  if (aligned16(x) && aligned16(y) && aligned16(z)) ewmul_kernel<true><<<g, kVecBlock, 0, s>>>(n, x, y, z);
  else ewmul_kernel<false><<<g, kVecBlock, 0, s>>>(n, x, y, z);
  return cudaGetLastError();
}

}  // namespace cgk

namespace cgk {

// FP32 copy of the matrix values (mixed-precision handles), round to nearest.
__global__ void f64_to_f32_kernel(int64_t n, const double* __restrict__ src, float* __restrict__ dst) {
  const int64_t T = static_cast<int64_t>(gridDim.x) * kVecBlock;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * kVecBlock + threadIdx.x; i < n; i += T)
    dst[i] = __double2float_rn(src[i]);
}

cudaError_t launch_f64_to_f32(int64_t n, const double* src, float* dst, cudaStream_t s) {
  f64_to_f32_kernel<<<stream_grid(n), kVecBlock, 0, s>>>(n, src, dst);
  return cudaGetLastError();
}

}  // namespace cgk

// ---------------------------------------------------------------------------
// Dot product without any allocation (cg_dot_noalloc).
//
// Same kernel as cg_dot, launched with one CTA per kNoAllocElemsPerCta
// elements, with its scratch in a fixed device array compiled into the
// library instead of memory the caller or a handle allocates.  The array holds
// kNoAllocMaxCtas per-CTA partial sums followed by the arrival counter, so the
// largest accepted length is kNoAllocMaxCtas * kNoAllocElemsPerCta elements.
// Every GPU that loads the library keeps this array (about 128 KB) until the
// process exits.
#include <mutex>

namespace cgk {

constexpr int kNoAllocMaxCtas = 16384;
constexpr int64_t kNoAllocElemsPerCta = 2048;
constexpr int64_t kNoAllocMaxN = static_cast<int64_t>(kNoAllocMaxCtas) * kNoAllocElemsPerCta;

// [0, kNoAllocMaxCtas): partial sums; the next slot holds the arrival counter.
static __device__ __align__(256) double g_dot_noalloc_scratch[kNoAllocMaxCtas + 32];

int64_t dot_noalloc_max_n() { return kNoAllocMaxN; }

// Device address of the scratch on the current device.  In host code the
// array's name is only a stand-in, so the address comes from
// cudaGetSymbolAddress, once per device (with that device current), and is
// cached.  The first call on a device therefore makes a runtime call that must
// not happen inside a stream capture.
static cudaError_t noalloc_scratch(double** out) {
  static std::mutex mu;
  static double* cache[64] = {nullptr};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  if (!cache[dev]) {
    double* p = nullptr;
    e = cudaGetSymbolAddress(reinterpret_cast<void**>(&p), g_dot_noalloc_scratch);
    if (e != cudaSuccess) return e;
    cache[dev] = p;
  }
  *out = cache[dev];
  return cudaSuccess;
}

cudaError_t launch_dot_noalloc(int64_t n, const double* x, const double* y, double* out, cudaStream_t s) {
  if (n < 0 || n > kNoAllocMaxN) return cudaErrorInvalidValue;
  double* scratch = nullptr;
  cudaError_t e = noalloc_scratch(&scratch);
  if (e != cudaSuccess) return e;
  unsigned int* counter = reinterpret_cast<unsigned int*>(scratch + kNoAllocMaxCtas);
  // The counter must start at zero; the kernel's last CTA also resets it, but a
  // call that never finished would leave it set.
  e = cudaMemsetAsync(counter, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  int64_t grid = (n + kNoAllocElemsPerCta - 1) / kNoAllocElemsPerCta;
  if (grid < 1) grid = 1;
  dot_kernel<<<static_cast<unsigned int>(grid), kVecBlock, 0, s>>>(n, x, y, out, scratch, counter);
  return cudaGetLastError();
}

}  // namespace cgk
