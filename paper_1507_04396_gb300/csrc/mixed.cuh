// mixed.cuh -- the rotation search with a tensor-core Gram shortlist (internal).
#pragma once

#include <vector>

#include "stage.cuh"

namespace pmmf {

// s + x kept as the FP32 pair (hi, lo): hi takes the rounded sum, lo gathers
// the exact rounding errors of those additions (Knuth's TwoSum; the cascaded
// summation "Sum2" of Ogita, Rump and Oishi, 2005).  FP32 instructions only,
// where an FP64 add per chunk and output would load the SM's small FP64 pipe.
__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float x) {
    const float s = __fadd_rn(hi, x);
    const float bp = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(x, bp));
    hi = s;
    lo = __fadd_rn(lo, err);
}

// G~ of every cluster (rows [hcoff[u], hcoff[u + 1]) of the split slab XH,
// XL: rows x sp elements, sp a multiple of 8) into G at goff[u] (c x c,
// FP32) on the tcgen05 tensor cores; TF32 or BF16 (PMMF_PREC_*).  A bounded
// wait that runs out sets ST_TIMEOUT in *status (device).
pmmf_status tc_gram_tcgen05(int precision, const void *XH, const void *XL, int64_t rows, int64_t sp,
                            const int64_t *coff, const std::vector<int64_t> &hcoff,
                            const int64_t *goff, float *G, unsigned *status, cudaStream_t st);

// The same with the kernel chosen by PMMF_TUNE_TC_GRAM (2 = tcgen05, the
// default; 1 = the warp-level mma.sync kernel).
pmmf_status tc_gram(int precision, const void *XH, const void *XL, int64_t rows, int64_t sp,
                    const int64_t *coff, const std::vector<int64_t> &hcoff, const int64_t *goff,
                    float *G, unsigned *status, cudaStream_t st);

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
