// mixed.cuh -- the rotation search with a tensor-core Gram shortlist (internal).
#pragma once

#include <vector>

#include "stage.cuh"

namespace pmmf {

// Rotation search of every cluster of a dense stage with the Gram matrices
// formed in TF32 or BF16 (PMMF_PREC_*) and FP64 re-scoring; stats[4]
// accumulates (candidates re-scored, full-row fallbacks, steps, largest
// shortlist).
pmmf_status mixed_stage_select(const DBuf<double> &D, int64_t s, const int32_t *pos,
                               const StageClusters &cls, const std::vector<int64_t> &hcoff,
                               int64_t cmax, int precision, uint64_t seed, int64_t stage,
                               StageRotations &rot, int32_t *elimflag, unsigned long long *stats,
                               unsigned *status, cudaStream_t st);

}  // namespace pmmf
