// The batched persistent solve: many systems in one cooperative launch.
// Each CTA takes tasks (a system and its rank in the system's group of CTAs)
// from a queue; the CG arithmetic of every task is the single-system solve's
// (cg_solve.cuh).
#include "cg_solve.cuh"

namespace cgk {

// Many systems in one persistent launch: each CTA takes tasks (a system and
// its rank in the system's group) from the queue, in queue order, until it is
// empty.  The host orders the queue longest estimated time per CTA first,
// with a group's ranks next to each other; a group's first ranks wait at its
// first group barrier until CTAs that free up have taken the rest.  Between
// tasks the whole CTA (producer included) joins, the producer having drained
// its copies, and the ring barriers are reset.
template <bool kMixed, bool kJacobi>
__global__ void __launch_bounds__(kBlock, kCtasPerSm) cg_batch_kernel(const __grid_constant__ BatchParams B) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const RingSmem sm{smem_raw, kMixed ? 4u : 8u};  // FP32 values in the mixed solve's stream
  __shared__ int32_t task_id;
  bool reinit = false;
  for (;;) {
    if (threadIdx.x == 0) task_id = atomicAdd(B.next, 1);
    __syncthreads();
    const int t = task_id;
    if (t >= B.queue->ntasks) break;
    const BatchTask tk = B.queue->task[t];
    const SolveParams& P = B.sys[tk.sys];
    CtaStream cs;
    stream_setup(sm, cs, P.A, tk.rank, reinit);
    reinit = true;
    if (threadIdx.x >= kConsumers) solve_producer<kMixed>(sm, cs, P);
    else solve_consumers<kMixed, kJacobi, false, false>(sm, cs, P, tk.rank, &B.queue->stream_rows);
    __syncthreads();  // producer drained, consumers done: the CTA is free
  }
}

const void* batch_kernel_ptr(bool mixed, bool jacobi) {
  if (mixed) return jacobi ? reinterpret_cast<const void*>(cg_batch_kernel<true, true>)
                           : reinterpret_cast<const void*>(cg_batch_kernel<true, false>);
  return jacobi ? reinterpret_cast<const void*>(cg_batch_kernel<false, true>)
                : reinterpret_cast<const void*>(cg_batch_kernel<false, false>);
}

int batch_blocks_per_sm(bool mixed, bool jacobi) {
  int nb = 0;
  const void* k = batch_kernel_ptr(mixed, jacobi);
  const size_t smem = solve_smem_bytes(mixed);
  cudaError_t e = ensure_smem_attr(k, smem);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, kBlock, smem);
  return e == cudaSuccess ? nb : -1;
}

// Cooperative launch (all CTAs co-resident: the ranks of a group wait on
// each other), through cudaLaunchKernelEx so that it can be captured in a
// CUDA graph.
cudaError_t launch_batch(const BatchParams& B, bool mixed, bool jacobi, int nblocks, cudaStream_t s) {
  const void* k = batch_kernel_ptr(mixed, jacobi);
  const size_t smem = solve_smem_bytes(mixed);
  cudaError_t e = ensure_smem_attr(k, smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nblocks);
  cfg.blockDim = dim3(kBlock);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  void* args[] = {const_cast<BatchParams*>(&B)};
  return cudaLaunchKernelExC(&cfg, k, args);
}

}  // namespace cgk
