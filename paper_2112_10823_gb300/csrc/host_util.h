// Host-side helpers shared by the single-system and batched entry points:
// the step partition of a CSR matrix for the persistent kernels.
#pragma once
#include <cstdint>
#include <vector>
#include <vector_types.h>

namespace cgh {

// Row partition of the persistent kernels for `nblocks` CTAs: CTA ranges of
// about equal cost (block_row), each split into steps (block_step, step,
// step_mode; see cg_internal.h), plus two sentinel steps.
struct Partition {
  std::vector<int4> step;
  std::vector<int32_t> step_mode;
  std::vector<int32_t> block_step;
  std::vector<int32_t> block_row;
};

void build_partition(const std::vector<int32_t>& rp, int64_t n, int nblocks, Partition& P);

}  // namespace cgh
