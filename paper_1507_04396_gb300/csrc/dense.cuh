// dense.cuh -- the stage on a dense active matrix (internal).
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>

#include <vector>

#include "rotmath.cuh"
#include "stage.cuh"

namespace pmmf {

// The stage's rotations across all clusters, grouped by dependency level,
// with row positions in place of cluster-local indices (passed by value).
struct DenseRotList {
    int K = 2;
    Rot2 *g2 = nullptr;               // k = 2: positions and (c, s)
    int64_t *gt = nullptr;            // k >= 3: step-order rotation of each slot
    int32_t *gpos = nullptr;          // k >= 3: K positions per slot (-1 unused)
    int32_t *gkk = nullptr;           // k = 3: tuple size per slot
    double *gO3 = nullptr;            // k = 3: the slot's block O, stride 3 (a * 3 + b)
    const Rot2 *lvlrot = nullptr;     // per-cluster sources
    const int32_t *lvlidx = nullptr, *kkv = nullptr, *kidx = nullptr;
    const double *kO = nullptr;
};

struct DenseLevels {
    int nlv = 0;
    DBuf<int64_t> goffL;              // nlv + 1: slots of level L at [goffL[L-1], goffL[L])
    DBuf<Rot2> g2;
    DBuf<int64_t> gt;
    DBuf<int32_t> gpos;
    DBuf<int32_t> gkk;
    DBuf<double> gO3;
    DenseRotList L;
};

// D = the caller's n x ld matrix, contiguous; status: ST_NONFINITE,
// ST_NOT_SYMMETRIC (bitwise, +0 and -0 equal).
pmmf_status dense_load(const double *A, int64_t n, int64_t ld, DBuf<double> &D, unsigned *status,
                       cudaStream_t st);
// Gram and local blocks of every cluster from the dense active matrix.
pmmf_status dense_gram(const DBuf<double> &D, int64_t s, const int32_t *pos,
                       const StageClusters &cls, const std::vector<int64_t> &hcoff,
                       GramBlocks &gb, cudaStream_t st);
pmmf_status dense_levels(const StageClusters &cls, const StageRotations &rot, const int32_t *pos,
                         int nlv, DenseLevels &out, cudaStream_t st);
// A_p = (A Q^T)^T Q^T in D (overwritten), residual and H diagonal of the
// eliminated coordinates, then the survivors' block in Dnext (s2 x s2) and
// their ids in nact.
pmmf_status dense_update(DBuf<double> &D, int64_t s, const DenseLevels &lv, const int32_t *act,
                         const int32_t *elimflag, int64_t stage, double *hdiag, double *contrib,
                         DBuf<double> &Dnext, DBuf<int32_t> &nact, int64_t &s2, cudaStream_t st);
// The same update with the block laid out in padded cluster order and moved
// in tiles by TMA (the rotations staged once per CTA).  *used = false (and
// nothing done) when a cluster's tiles do not fit shared memory or the tensor
// map call is unavailable; the caller then runs dense_update.
pmmf_status dense_update_tiles(DBuf<double> &D, int64_t s, const StageClusters &cls,
                               const std::vector<int64_t> &hc, const StageRotations &rot,
                               const int32_t *pos, const int32_t *act, const int32_t *elimflag,
                               int64_t stage, double *hdiag, double *contrib, DBuf<double> &Dnext,
                               DBuf<int32_t> &nact, int64_t &s2, unsigned *status, cudaStream_t st,
                               bool *used);
// cuTensorMapEncodeTiled from the driver, looked up once; nullptr when the
// driver does not export it.
PFN_cuTensorMapEncodeTiled_v12000 encode_fn();
// Number of entries that are not +-0.
pmmf_status dense_nonzeros(const double *D, int64_t cnt, int64_t *out, cudaStream_t st);
pmmf_status dense_core(const double *D, int64_t s, const int32_t *act, double *core, double *hdiag,
                       cudaStream_t st);
// CSR copy of D (exact zeros dropped) with global column ids.
pmmf_status dense_record(const double *D, int64_t s, const int32_t *act, Csr &out,
                         cudaStream_t st);

}  // namespace pmmf
