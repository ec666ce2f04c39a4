// batch.cu -- kernels of the batched factorization: many independent
// symmetric matrices stored as one block-diagonal matrix, each factored as
// its own pMMF with one cluster per stage (Algorithm 1 with the clustering
// step returning the whole active set of the matrix).  All matrices advance
// through the stages together, so every stage is one launch per kernel kind
// over every cluster of every matrix.  A matrix whose active set has reached
// the core size retires: its remaining rows become its dense core block of H
// and leave the active matrix.
#include "batch.cuh"

namespace pmmf {
namespace {

// Per matrix b: first row of its coordinates in the ascending active list and
// how many of them are active.
__global__ void k_batch_ranges(const int32_t *act, int64_t s, const int64_t *moff, int64_t nmat,
                               int64_t *lo, int64_t *cnt) {
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nmat;
         b += (int64_t)gridDim.x * blockDim.x) {
        int64_t l = 0, h = s;
        while (l < h) {
            int64_t mid = (l + h) >> 1;
            if (act[mid] < moff[b]) l = mid + 1; else h = mid;
        }
        int64_t l2 = l, h2 = s;
        while (l2 < h2) {
            int64_t mid = (l2 + h2) >> 1;
            if (act[mid] < moff[b + 1]) l2 = mid + 1; else h2 = mid;
        }
        lo[b] = l;
        cnt[b] = l2 - l;
    }
}

// One CTA per retiring matrix: its rows [lo, lo + cnt) of the active matrix
// become the dense core block at slot blk * bs (H on S_L, Sec. 2); the block's
// diagonal also goes to hdiag.
__global__ void k_batch_core(const int64_t *rp, const int32_t *ci, const double *v,
                             const int32_t *act, const int32_t *pos, const int64_t *rmat,
                             const int64_t *rlo, const int64_t *rcnt, int64_t bs, double *core,
                             int32_t *core_idx, int32_t *core_pos, int32_t *bdim, double *hdiag) {
    const int64_t b = rmat[blockIdx.x];
    const int64_t lo = rlo[blockIdx.x], cnt = rcnt[blockIdx.x];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double *cb = core + b * bs * bs;
    if (threadIdx.x == 0) bdim[b] = (int32_t)cnt;
    for (int64_t l = wid; l < cnt; l += nw) {
        const int64_t r = lo + l;
        const int32_t g = act[r];
        if (lane == 0) {
            core_idx[b * bs + l] = g;
            core_pos[g] = (int32_t)(b * bs + l);
        }
        for (int64_t q = rp[r] + lane; q < rp[r + 1]; q += 32) {
            const int64_t l2 = pos[ci[q]] - lo;
            cb[l * bs + l2] = v[q];
            if (l2 == l) hdiag[g] = v[q];
        }
    }
}

__global__ void k_row_keep(const int32_t *act, int64_t s, const int32_t *retired_mat,
                           const int64_t *moff, int64_t nmat, int32_t *keep, int64_t *len,
                           const int64_t *rp) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < s;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int32_t g = act[r];
        int64_t l = 0, h = nmat;   // matrix of g: last b with moff[b] <= g
        while (h - l > 1) {
            const int64_t mid = (l + h) >> 1;
            if (moff[mid] <= g) l = mid; else h = mid;
        }
        const int k = retired_mat[l] ? 0 : 1;
        keep[r] = k;
        len[r] = k ? rp[r + 1] - rp[r] : 0;
    }
}

// Warp per kept row: copy it to its new position.  start = exclusive scan of
// the kept rows' lengths (the new row pointers, by old row).
__global__ void k_compact_rows(const int64_t *rp, const int32_t *ci, const double *v,
                               const int32_t *act, int64_t s, const int32_t *keep,
                               const int64_t *newrow, const int64_t *start, int64_t *nrp,
                               int32_t *nci, double *nv, int32_t *nact) {
    const int lane = threadIdx.x & 31;
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = w; r < s; r += nw) {
        if (!keep[r]) continue;
        const int64_t nr = newrow[r];
        const int64_t d = start[r] - rp[r];
        for (int64_t q = rp[r] + lane; q < rp[r + 1]; q += 32) {
            nci[q + d] = ci[q];
            nv[q + d] = v[q];
        }
        if (lane == 0) {
            nact[nr] = act[r];
            nrp[nr] = start[r];
        }
    }
}

// Clusters = the active matrices in order; members = the active list itself.
__global__ void k_batch_clusters(const int32_t *act, int64_t s, const int64_t *coff, int64_t m,
                                 int32_t *members, int32_t *cl, int32_t *loc) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < s;
         r += (int64_t)gridDim.x * blockDim.x) {
        int64_t l = 0, h = m;   // cluster of row r: last u with coff[u] <= r
        while (h - l > 1) {
            const int64_t mid = (l + h) >> 1;
            if (coff[mid] <= r) l = mid; else h = mid;
        }
        const int32_t g = act[r];
        members[r] = g;
        cl[g] = (int32_t)l;
        loc[g] = (int32_t)(r - coff[l]);
    }
}

// Entries outside their row's diagonal block set the status (not block-diagonal).
__global__ void k_check_blocks(int64_t n, const int64_t *rp, const int32_t *ci,
                               const int64_t *moff, int64_t nmat, unsigned *status) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x) {
        int64_t l = 0, h = nmat;
        while (h - l > 1) {
            const int64_t mid = (l + h) >> 1;
            if (moff[mid] <= r) l = mid; else h = mid;
        }
        if (rp[r] < rp[r + 1] && (ci[rp[r]] < moff[l] || ci[rp[r + 1] - 1] >= moff[l + 1]))
            atomicOr(status, ST_BAD_CSR);
    }
}

// Squared Frobenius norm of every block (its rows are contiguous), one CTA per
// block, a fixed reduction order.
__global__ void k_block_sumsq(const int64_t *rp, const double *v, const int64_t *moff,
                              double *out) {
    __shared__ double red[256];
    const int64_t b = blockIdx.x;
    const int64_t e0 = rp[moff[b]], e1 = rp[moff[b + 1]];
    double acc = 0.0;
    for (int64_t q = e0 + threadIdx.x; q < e1; q += blockDim.x) acc = __fma_rn(v[q], v[q], acc);
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] = __dadd_rn(red[threadIdx.x], red[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) out[b] = red[0];
}

}  // namespace

pmmf_status batch_ranges(const int32_t *act, int64_t s, const int64_t *moff, int64_t nmat,
                         int64_t *lo, int64_t *cnt, cudaStream_t st) {
    k_batch_ranges<<<grid_for(nmat, 128), 128, 0, st>>>(act, s, moff, nmat, lo, cnt);
    return launched("batch_ranges");
}

pmmf_status batch_core(const Csr &A, const int32_t *act, const int32_t *pos, int64_t nret,
                       const int64_t *rmat, const int64_t *rlo, const int64_t *rcnt, int64_t bs,
                       double *core, int32_t *core_idx, int32_t *core_pos, int32_t *bdim,
                       double *hdiag, cudaStream_t st) {
    if (nret == 0) return PMMF_OK;
    k_batch_core<<<(unsigned)nret, 256, 0, st>>>(A.rowptr.p, A.col.p, A.val.p, act, pos, rmat, rlo,
                                                  rcnt, bs, core, core_idx, core_pos, bdim, hdiag);
    return launched("batch_core");
}

pmmf_status batch_drop_rows(Csr &A, DBuf<int32_t> &act, const int32_t *retired_mat,
                            const int64_t *moff, int64_t nmat, cudaStream_t st) {
    const int64_t s = A.rows;
    DBuf<int32_t> keep;
    DBuf<int64_t> len, newrow;
    PMMF_TRY(keep.alloc(s, st));
    PMMF_TRY(len.alloc(s + 1, st));
    PMMF_TRY(newrow.alloc(s + 1, st));
    k_row_keep<<<grid_for(s, 256), 256, 0, st>>>(act.p, s, retired_mat, moff, nmat, keep.p, len.p,
                                                  A.rowptr.p);
    PMMF_TRY(launched("row_keep"));
    PMMF_TRY(scan_i32_to_i64(keep.p, newrow.p, s, st));
    PMMF_TRY(scan_i64(len.p, len.p, s, st));
    int64_t hv[2] = {0, 0};
    PMMF_CUDA_TRY(cudaMemcpyAsync(&hv[0], newrow.p + s, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    PMMF_CUDA_TRY(cudaMemcpyAsync(&hv[1], len.p + s, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    PMMF_CUDA_TRY(cudaStreamSynchronize(st));
    Csr B;
    B.rows = hv[0];
    B.nnz = hv[1];
    PMMF_TRY(B.rowptr.alloc(B.rows + 1, st));
    PMMF_TRY(B.col.alloc(B.nnz, st));
    PMMF_TRY(B.val.alloc(B.nnz, st));
    DBuf<int32_t> nact;
    PMMF_TRY(nact.alloc(B.rows, st));
    k_compact_rows<<<grid_for(s * 32, 256), 256, 0, st>>>(A.rowptr.p, A.col.p, A.val.p, act.p, s,
                                                          keep.p, newrow.p, len.p, B.rowptr.p,
                                                          B.col.p, B.val.p, nact.p);
    PMMF_TRY(launched("compact_rows"));
    PMMF_CUDA_TRY(cudaMemcpyAsync(B.rowptr.p + B.rows, len.p + s, sizeof(int64_t),
                                  cudaMemcpyDeviceToDevice, st));
    A = std::move(B);
    act = std::move(nact);
    return PMMF_OK;
}

pmmf_status batch_clusters(const int32_t *act, int64_t s, const int64_t *coff, int64_t m,
                           StageClusters &out, int32_t *cl, int32_t *loc, cudaStream_t st) {
    PMMF_TRY(out.members.alloc(s, st));
    out.m = m;
    k_batch_clusters<<<grid_for(s, 256), 256, 0, st>>>(act, s, coff, m, out.members.p, cl, loc);
    return launched("batch_clusters");
}

pmmf_status check_blocks(int64_t n, const int64_t *rp, const int32_t *ci, const int64_t *moff,
                         int64_t nmat, unsigned *status, cudaStream_t st) {
    k_check_blocks<<<grid_for(n, 256), 256, 0, st>>>(n, rp, ci, moff, nmat, status);
    return launched("check_blocks");
}

pmmf_status block_sumsq(const int64_t *rp, const double *v, const int64_t *moff, int64_t nmat,
                        double *out, cudaStream_t st) {
    k_block_sumsq<<<(unsigned)nmat, 256, 0, st>>>(rp, v, moff, out);
    return launched("block_sumsq");
}

}  // namespace pmmf
