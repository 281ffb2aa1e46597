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

// Which kind of step (cgk::StepMode: one lane per row, two lanes per row, or
// a warp per row) rows of each length 0..64 go to; longer rows always take a
// warp each.  A step's kind is the widest kind among its rows; a one-lane
// step holds up to 32 rows, a two-lane step up to 16.  The built-in table is
// one lane for rows of up to 32 entries and two lanes for 33..64.  A lane
// computes at most 32 entries, so mode[L] may be "one lane" only for L <= 32.
constexpr int kShapeMaxLen = 64;
struct StepShape {
  int8_t mode[kShapeMaxLen + 1];
  StepShape();
  bool valid() const;
};

void build_partition(const std::vector<int32_t>& rp, int64_t n, int nblocks, Partition& P,
                     const StepShape& shape = StepShape());

}  // namespace cgh
