// Classical CG (the paper's Sec. 5.3 solver) for small systems on one
// thread-block cluster.  A whole-grid solve of a system with a few thousand
// rows is a chain of grid-wide synchronisations (each CTA holds a few dozen
// rows); here sixteen CTAs hold the system in shared memory instead: each CTA
// its contiguous range of rows, their CSR entries, and p and x of those rows.
// The product gathers p from the owning CTA's shared memory (distributed
// shared memory), the two sums of a step are exchanged through it, and the
// synchronisations are hardware cluster barriers.  Every CTA computes the
// same scalars from the same exact fixed-point sums, so all CTAs take the
// same branches and reach the same barriers (there is no spin-wait).  The
// arithmetic per row and per sum is the other kernels': each row summed in
// storage order with FMA, sums exact in fixed point.
#include <cmath>
#include "cg_device.cuh"

namespace cgk {

namespace {

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// Every thread of every CTA of the cluster; writes before it (shared memory
// of any CTA of the cluster) are visible to all after it.
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Address, in the cluster's shared window, of `p` in the CTA of rank `rank`.
__device__ __forceinline__ uint32_t cluster_addr(const void* p, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
  return r;
}

__device__ __forceinline__ double cluster_ld(uint32_t addr) {
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(addr) : "memory");
  return v;
}

__device__ __forceinline__ void cluster_st(uint32_t addr, double v) {
  asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(addr), "d"(v) : "memory");
}

// Shared-memory layout of a cluster CTA for R rows and E entries per CTA.
struct ClusterLayout {
  int R, E;
  __host__ __device__ size_t off_p() const { return 0; }
  __host__ __device__ size_t off_x() const { return off_p() + 8 * static_cast<size_t>(R); }
  __host__ __device__ size_t off_val() const { return off_x() + 8 * static_cast<size_t>(R); }
  __host__ __device__ size_t off_sums() const { return off_val() + 8 * static_cast<size_t>(E); }  // [2 sets][2 values][CTAs]
  __host__ __device__ size_t off_part() const { return off_sums() + 8 * 2 * 2 * kClusterCtas; }   // [2 values][16 warps] FxPart
  __host__ __device__ size_t off_scal() const { return off_part() + sizeof(FxPart) * 2 * 16; }    // 8 doubles
  __host__ __device__ size_t off_col() const { return off_scal() + 8 * 8; }
  __host__ __device__ size_t off_rp() const { return off_col() + ((4 * static_cast<size_t>(E) + 15) & ~size_t(15)); }
  __host__ __device__ size_t bytes() const { return off_rp() + ((4 * (static_cast<size_t>(R) + 1) + 15) & ~size_t(15)); }
};

}  // namespace

struct ClusterParams {
  const int32_t* row_ptr;  // the handle's 0-based CSR
  const int32_t* col_idx;
  const double* val;
  const double* b;
  double* x;               // initial guess in, solution out
  SolveCtrl* ctrl;         // status and results (written by rank 0)
  double tol;
  int64_t maxit;
  int32_t n;
  int32_t R;               // rows per CTA, a power of two (the last CTAs may hold fewer)
  int32_t E;               // capacity of a CTA's entry arrays
  int32_t log2R;
};

__global__ void __launch_bounds__(kClusterThreads, 1) cg_cluster_kernel(const __grid_constant__ ClusterParams P) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const ClusterLayout L{P.R, P.E};
  double* const p_s = reinterpret_cast<double*>(smem_raw + L.off_p());
  double* const x_s = reinterpret_cast<double*>(smem_raw + L.off_x());
  double* const val_s = reinterpret_cast<double*>(smem_raw + L.off_val());
  double* const sums = reinterpret_cast<double*>(smem_raw + L.off_sums());
  FxPart* const part = reinterpret_cast<FxPart*>(smem_raw + L.off_part());
  double* const scal = reinterpret_cast<double*>(smem_raw + L.off_scal());
  int32_t* const col_s = reinterpret_cast<int32_t*>(smem_raw + L.off_col());
  int32_t* const rp_s = reinterpret_cast<int32_t*>(smem_raw + L.off_rp());
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t rank = cluster_rank();
  const int row0 = min(static_cast<int>(rank) * P.R, P.n), row1 = min(row0 + P.R, P.n);
  const int nr = row1 - row0;
  constexpr int kRowsPerThread = (kClusterMaxRows + kClusterThreads - 1) / kClusterThreads;

  // ---- the CTA's rows: entries and row pointers (local), x0, into shared memory
  const int e0 = P.row_ptr[row0];
  const int ne = P.row_ptr[row1] - e0;
  for (int k = tid; k < ne; k += kClusterThreads) {
    val_s[k] = P.val[e0 + k];
    col_s[k] = P.col_idx[e0 + k];
  }
  for (int i = tid; i <= nr; i += kClusterThreads) rp_s[i] = P.row_ptr[row0 + i] - e0;
  for (int i = tid; i < nr; i += kClusterThreads) x_s[i] = P.x[row0 + i];
  cluster_sync_all();

  // y_i = (A v)_i for the CTA's local row i, v (p or x) gathered from the
  // owning CTAs' shared memory (CTA c >> log2R, entry c & (R - 1)), in
  // storage order with FMA; the loads of 8 entries go out before their FMAs
  const int lg = P.log2R;
  const int rmask = (1 << lg) - 1;
  auto row_product = [&](const double* v_s, int i) -> double {
    double acc = 0.0;
    const int k1 = rp_s[i + 1];
    for (int kb = rp_s[i]; kb < k1; kb += 8) {
      double vc[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        if (kb + u < k1) {
          const int c = col_s[kb + u];
          vc[u] = cluster_ld(cluster_addr(v_s + (c & rmask), static_cast<uint32_t>(c >> lg)));
        }
      }
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (kb + u < k1) acc = fma(val_s[kb + u], vc[u], acc);
    }
    return acc;
  };

  // Cluster-wide sum of nv (<= 2) values per thread, exact in fixed point:
  // warps, then the CTA (warp 0), then the kClusterCtas CTA values, which
  // warp 0 of every CTA writes into slot `rank` of set `set` in every CTA's
  // shared memory; after the cluster barrier each CTA sums the same values
  // the same way.  The two sets alternate so that a CTA writing the next sum
  // never overwrites values a slower CTA still reads (between two uses of a
  // set every CTA passes a cluster barrier after reading it).
  int set = 0;
  auto cluster_sum = [&](int nv, double v0, double v1, double* out) {
    const double vin[2] = {v0, v1};
#pragma unroll
    for (int j = 0; j < 2; ++j)
      if (j < nv) {
        const FxPart f = fx_warp(vin[j]);
        if (lane == 0) part[j * 16 + warp] = f;
      }
    __syncthreads();
    if (warp == 0) {
      const bool valid = lane < kClusterThreads / 32;
#pragma unroll
      for (int j = 0; j < 2; ++j)
        if (j < nv) {
          const double c = fx_combine(valid ? part[j * 16 + lane] : FxPart{0, 0, 0}, valid);
          if (lane < kClusterCtas)
            cluster_st(cluster_addr(sums + (set * 2 + j) * kClusterCtas + rank, static_cast<uint32_t>(lane)), c);
        }
    }
    cluster_sync_all();
    if (warp == 0) {
#pragma unroll
      for (int j = 0; j < 2; ++j)
        if (j < nv) {
          const bool valid = lane < kClusterCtas;
          const FxPart f = fx_warp(valid ? sums[(set * 2 + j) * kClusterCtas + lane] : 0.0);
          const double tot = f.nf ? __longlong_as_double(0x7ff8000000000000ll)
                                  : (f.e == 0 ? 0.0 : ldexp(static_cast<double>(f.m), f.e - 1074));
          if (lane == 0) scal[j] = tot;
        }
    }
    __syncthreads();
    out[0] = scal[0];
    if (nv > 1) out[1] = scal[1];
    set ^= 1;
    __syncthreads();  // scal is rewritten by the next sum
  };

  // ---- setup: r = b - A x0, p = r, rho = r.r, ||b||^2
  double rr_[kRowsPerThread], xr[kRowsPerThread], pr[kRowsPerThread];
  double acc_rr = 0.0, acc_bb = 0.0;
#pragma unroll
  for (int t = 0; t < kRowsPerThread; ++t) {
    const int i = tid + t * kClusterThreads;
    rr_[t] = xr[t] = pr[t] = 0.0;
    if (i < nr) {
      const double bi = P.b[row0 + i];
      const double ri = bi - row_product(x_s, i);
      rr_[t] = ri;
      pr[t] = ri;
      xr[t] = x_s[i];
      acc_rr = fma(ri, ri, acc_rr);
      acc_bb = fma(bi, bi, acc_bb);
    }
  }
  double s2[2];
  cluster_sum(2, acc_rr, acc_bb, s2);
  double rho = s2[0];
  const double bnorm2 = s2[1];
  const double thresh2 = (P.tol * P.tol) * bnorm2;
  int status = kENOTCONV;
  long long k = 0;
  double rr = rho;
  if (bnorm2 == 0.0) {  // b = 0: the solution is 0
#pragma unroll
    for (int t = 0; t < kRowsPerThread; ++t) xr[t] = 0.0;
    status = kOK;
  } else if (rr <= thresh2) {
    status = kOK;
  }
#pragma unroll
  for (int t = 0; t < kRowsPerThread; ++t) {
    const int i = tid + t * kClusterThreads;
    if (i < nr) p_s[i] = pr[t];
  }
  cluster_sync_all();  // p visible to every CTA

  while (status == kENOTCONV && k < P.maxit) {
    // ---- q = A p, gamma = p.q
    double qr[kRowsPerThread];
    double acc_g = 0.0;
#pragma unroll
    for (int t = 0; t < kRowsPerThread; ++t) {
      const int i = tid + t * kClusterThreads;
      qr[t] = 0.0;
      if (i < nr) {
        qr[t] = row_product(p_s, i);
        acc_g = fma(pr[t], qr[t], acc_g);
      }
    }
    double g[2];
    cluster_sum(1, acc_g, 0.0, g);
    if (!(g[0] > 0.0) || !isfinite(g[0])) {  // not SPD, or overflow
      status = kEBREAKDOWN;
      break;
    }
    const double alpha = rho / g[0];
    // ---- x += alpha p; r -= alpha q; rr = r.r
    double acc_r = 0.0;
#pragma unroll
    for (int t = 0; t < kRowsPerThread; ++t) {
      const int i = tid + t * kClusterThreads;
      if (i < nr) {
        xr[t] = fma(alpha, pr[t], xr[t]);
        rr_[t] = fma(-alpha, qr[t], rr_[t]);
        acc_r = fma(rr_[t], rr_[t], acc_r);
      }
    }
    double rs[2];
    cluster_sum(1, acc_r, 0.0, rs);
    ++k;
    rr = rs[0];
    if (rr <= thresh2) {
      status = kOK;
      break;
    }
    const double beta = rr / rho;
    rho = rr;
    // ---- p = r + beta p; visible to every CTA after the barrier
#pragma unroll
    for (int t = 0; t < kRowsPerThread; ++t) {
      const int i = tid + t * kClusterThreads;
      if (i < nr) {
        pr[t] = fma(beta, pr[t], rr_[t]);
        p_s[i] = pr[t];
      }
    }
    cluster_sync_all();
  }

  // ---- x out; the true residual ||b - A x|| / ||b||
#pragma unroll
  for (int t = 0; t < kRowsPerThread; ++t) {
    const int i = tid + t * kClusterThreads;
    if (i < nr) {
      x_s[i] = xr[t];
      P.x[row0 + i] = xr[t];
    }
  }
  cluster_sync_all();
  double acc_t = 0.0;
#pragma unroll
  for (int t = 0; t < kRowsPerThread; ++t) {
    const int i = tid + t * kClusterThreads;
    if (i < nr) {
      const double d = P.b[row0 + i] - row_product(x_s, i);
      acc_t = fma(d, d, acc_t);
    }
  }
  double ts[2];
  cluster_sum(1, acc_t, 0.0, ts);
  if (rank == 0 && tid == 0) {
    SolveCtrl* c = P.ctrl;
    c->status = status;
    c->iters = k;
    c->rho = rho;
    c->bnorm2 = bnorm2;
    c->relres_rec = bnorm2 > 0.0 ? sqrt(rr / bnorm2) : 0.0;
    c->relres_true = bnorm2 > 0.0 ? sqrt(ts[0] / bnorm2) : 0.0;
    c->phase = kPhaseDone;
  }
  cluster_sync_all();  // no CTA leaves while another may still read its shared memory
}

size_t cluster_smem_bytes(int R, int E) { return ClusterLayout{R, E}.bytes(); }

namespace {
cudaLaunchConfig_t cluster_config(size_t smem, cudaStream_t s, cudaLaunchAttribute* attr) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kClusterCtas);
  cfg.blockDim = dim3(kClusterThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kClusterCtas;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}
}  // namespace

// The layout's size depends on the system; the kernel is opted in once to
// the largest layout that cg_create accepts.
constexpr size_t kClusterSmemMax = size_t(220) << 10;

// Clusters above 8 CTAs need the kernel's opt-in to non-portable sizes.
cudaError_t cluster_attrs() {
  cudaError_t e = ensure_smem_attr(reinterpret_cast<const void*>(cg_cluster_kernel), kClusterSmemMax);
  if (e == cudaSuccess && kClusterCtas > 8)
    e = cudaFuncSetAttribute(reinterpret_cast<const void*>(cg_cluster_kernel),
                             cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  return e;
}

int cluster_max_active(int R, int E) {
  const size_t smem = cluster_smem_bytes(R, E);
  if (smem > kClusterSmemMax || cluster_attrs() != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  cudaLaunchAttribute attr[1];
  const cudaLaunchConfig_t cfg = cluster_config(smem, nullptr, attr);
  int num = 0;
  if (cudaOccupancyMaxActiveClusters(&num, reinterpret_cast<const void*>(cg_cluster_kernel), &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return num;
}

cudaError_t launch_cluster_solve(const int32_t* row_ptr, const int32_t* col_idx, const double* val,
                                 const double* b, double* x, SolveCtrl* ctrl, double tol, int64_t maxit, int32_t n,
                                 int32_t R, int32_t E, cudaStream_t s) {
  const size_t smem = cluster_smem_bytes(R, E);
  if (smem > kClusterSmemMax) return cudaErrorInvalidValue;
  cudaError_t e = cluster_attrs();
  if (e != cudaSuccess) return e;
  int lg = 0;
  while ((1 << lg) < R) ++lg;
  if ((1 << lg) != R) return cudaErrorInvalidValue;  // R must be a power of two
  ClusterParams P{row_ptr, col_idx, val, b, x, ctrl, tol, maxit, n, R, E, lg};
  cudaLaunchAttribute attr[1];
  const cudaLaunchConfig_t cfg = cluster_config(smem, s, attr);
  return cudaLaunchKernelEx(&cfg, cg_cluster_kernel, P);
}

}  // namespace cgk
