// batch.cuh -- building blocks of the batched (block-diagonal) factorization
// (internal).
#pragma once

#include "stage.cuh"

namespace pmmf {

// lo[b], cnt[b]: first row and number of active coordinates of matrix b
// (coordinates moff[b] .. moff[b+1]-1) in the ascending active list.
pmmf_status batch_ranges(const int32_t *act, int64_t s, const int64_t *moff, int64_t nmat,
                         int64_t *lo, int64_t *cnt, cudaStream_t st);

// Core blocks of the nret retiring matrices rmat[] (rows rlo[] .. + rcnt[]).
pmmf_status batch_core(const Csr &A, const int32_t *act, const int32_t *pos, int64_t nret,
                       const int64_t *rmat, const int64_t *rlo, const int64_t *rcnt, int64_t bs,
                       double *core, int32_t *core_idx, int32_t *core_pos, int32_t *bdim,
                       double *hdiag, cudaStream_t st);

// Drop the rows of retired matrices (retired_mat[b] != 0) from A and act.
pmmf_status batch_drop_rows(Csr &A, DBuf<int32_t> &act, const int32_t *retired_mat,
                            const int64_t *moff, int64_t nmat, cudaStream_t st);

// One cluster per active matrix: members = act, cluster offsets coff (m + 1).
pmmf_status batch_clusters(const int32_t *act, int64_t s, const int64_t *coff, int64_t m,
                           StageClusters &out, int32_t *cl, int32_t *loc, cudaStream_t st);

// ST_BAD_CSR when an entry lies outside its row's diagonal block.
pmmf_status check_blocks(int64_t n, const int64_t *rp, const int32_t *ci, const int64_t *moff,
                         int64_t nmat, unsigned *status, cudaStream_t st);

// out[b] = squared Frobenius norm of diagonal block b.
pmmf_status block_sumsq(const int64_t *rp, const double *v, const int64_t *moff, int64_t nmat,
                        double *out, cudaStream_t st);

}  // namespace pmmf
