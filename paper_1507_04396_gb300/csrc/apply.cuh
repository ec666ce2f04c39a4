// apply.cuh -- matrix-free arithmetic and PCG helpers (internal).
#pragma once

#include <vector>

#include "common.cuh"

namespace pmmf {

struct ApplyStage {
    int64_t m = 0, nrot = 0, cmax = 0, s = 0;
    const int64_t *coff = nullptr;
    const int32_t *members = nullptr;
    const int64_t *roff = nullptr;
    const int32_t *lvl_off = nullptr;
    const int32_t *nlev = nullptr;
    const Rot2 *lvlrot = nullptr;
};
using ApplyStages = std::vector<ApplyStage>;

struct HData {
    int64_t n = 0, m = 0;
    const double *hdiag = nullptr;
    const int32_t *core_pos = nullptr;   // n: position in the core or -1
    const int32_t *core_idx = nullptr;   // m
    const double *core = nullptr;        // m x m
    const double *core_inv = nullptr;    // m x m
};

struct DevCsr {
    int64_t n = 0;
    const int64_t *rp = nullptr;
    const int32_t *ci = nullptr;
    const double *v = nullptr;
};

pmmf_status apply_rotations(const ApplyStages &S, bool transpose, double *x, int64_t ld,
                            int64_t nrhs, cudaStream_t st);
pmmf_status copy_block(const double *x, int64_t ldx, double *y, int64_t ldy, int64_t n,
                       int64_t nrhs, cudaStream_t st);
pmmf_status apply_h(const HData &H, bool inverse, double *x, int64_t ld, int64_t nrhs,
                    cudaStream_t st);
pmmf_status apply_h_scratch(const HData &H, bool inverse, double *x, int64_t ld, int64_t nrhs,
                            double *zc, cudaStream_t st);
pmmf_status invert_core(const double *core, int64_t m, const double *hdiag, const int32_t *core_pos,
                        int64_t n, double *inv, unsigned *status, cudaStream_t st);
pmmf_status spmv(const DevCsr &A, const double *x, double *y, int nrhs, cudaStream_t st);
pmmf_status dots(const double *x, const double *y, int64_t n, int nrhs, double *out,
                 double *partial, cudaStream_t st);
int64_t dot_partial_size(int nrhs);
pmmf_status cg_update_xr(double *x, double *r, const double *p, const double *q, int64_t n,
                         int nrhs, const double *rz, const double *pq, const int32_t *done,
                         cudaStream_t st);
pmmf_status cg_update_p(double *p, const double *z, int64_t n, int nrhs, const double *rznew,
                        double *rz, const int32_t *done, cudaStream_t st);
pmmf_status vec_sub(const double *b, const double *q, double *r, int64_t cnt, cudaStream_t st);

}  // namespace pmmf
