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
    // k >= 3 (see StageRotations)
    int K = 2;
    const int32_t *kidx = nullptr, *kkv = nullptr, *lvlidx = nullptr;
    const double *kO = nullptr;
};
using ApplyStages = std::vector<ApplyStage>;

// H = diagonal on wavelet coordinates plus a block-diagonal core: nblk blocks
// of slot stride bs (one dense block of size m for a single factorization,
// one block per matrix for a batch).  Core slot a = blk * bs + l; block blk
// holds bdim[blk] <= bs coordinates (all bs when bdim is null) and its values
// at core[blk * bs * bs + l * bs + l'].
struct HData {
    int64_t n = 0, m = 0;                // m = nblk * bs core slots
    int64_t nblk = 1, bs = 0;
    const int32_t *bdim = nullptr;       // nblk (null: every block full)
    const double *hdiag = nullptr;
    const int32_t *core_pos = nullptr;   // n: core slot or -1
    const int32_t *core_idx = nullptr;   // m slots: global id (unused slots -1)
    const double *core = nullptr;        // nblk * bs * bs
    const double *core_inv = nullptr;    // nblk * bs * bs
    const double *core_isqrt = nullptr;  // bs * bs (single core): core^{-1/2}
    // n: 1 / h_i and 1 / sqrt(h_i) of the diagonal (formed with core_inv and
    // core_isqrt; NULL: the wavelet part divides instead of multiplying)
    const double *hrcp = nullptr;
    const double *hisr = nullptr;
};

// out[i] = 1 / h_i (root false) or 1 / sqrt(h_i) (root true), i < n.
pmmf_status h_reciprocals(const double *hdiag, int64_t n, bool root, double *out, cudaStream_t st);

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
// mode 0: H, 1: H^{-1}, 2: H^{-1/2} (the core's inverse square root formed
// by core_inverse_sqrt).
pmmf_status apply_h(const HData &H, int mode, double *x, int64_t ld, int64_t nrhs,
                    cudaStream_t st);
pmmf_status apply_h_scratch(const HData &H, int mode, double *x, int64_t ld, int64_t nrhs,
                            double *zc, cudaStream_t st);
// out = S^{-1/2} for each core block's symmetric S (lower triangle mirrored,
// the block's bdim x bdim part; bdim NULL: all bs), by the coupled
// Newton-Schulz iteration, 0 on the padding; status gets ST_NOT_SPD for a
// wavelet entry that is not positive; PMMF_ERR_NOT_SPD when the iteration
// diverges or stalls (an eigenvalue <= 0, or numerically so).  iterations
// (may be NULL) gets the number of Newton-Schulz steps taken.
pmmf_status core_inverse_sqrt(const double *core, int64_t nblk, int64_t bs, const int32_t *bdim,
                              const double *hdiag, const int32_t *core_pos, int64_t n,
                              double *out, unsigned *status, int *iterations, cudaStream_t st);
pmmf_status invert_core(const double *core, int64_t m, const double *hdiag, const int32_t *core_pos,
                        int64_t n, double *inv, unsigned *status, cudaStream_t st);
// Block cores (nblk > 1): every block inverted by the same Gauss-Jordan
// sweep as invert_core, one CTA per block in shared memory.
pmmf_status invert_core_blocks(const double *core, int64_t nblk, int64_t bs, const int32_t *bdim,
                               const double *hdiag, const int32_t *core_pos, int64_t n,
                               double *inv, unsigned *status, cudaStream_t st);
pmmf_status spmv(const DevCsr &A, const double *x, double *y, int nrhs, cudaStream_t st);
pmmf_status dots(const double *x, const double *y, int64_t n, int nrhs, double *out,
                 double *partial, cudaStream_t st);
int64_t dot_partial_size(int nrhs);
pmmf_status cg_update_xr(double *x, double *r, const double *p, const double *q, int64_t n,
                         int nrhs, const double *rz, const double *pq, const int32_t *done,
                         double *alpha, cudaStream_t st);
pmmf_status cg_update_p(double *p, const double *z, int64_t n, int nrhs, const double *rznew,
                        double *rz, const int32_t *done, double *beta, cudaStream_t st);
// done/iters per column after the iteration counter *itc is advanced.
pmmf_status cg_check(const double *rr, const double *bnorm, double rtol, int nrhs, int32_t *done,
                     int32_t *iters, int32_t *itc, cudaStream_t st);
pmmf_status vec_sub(const double *b, const double *q, double *r, int64_t cnt, cudaStream_t st);

}  // namespace pmmf
