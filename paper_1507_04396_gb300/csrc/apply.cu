// apply.cu -- matrix-free arithmetic with the factorization (Sec. 2.4) and the
// preconditioned conjugate gradient solver of Sec. 4.
//
//   U x      stages 1..P in order; inside a stage every cluster's rotations
//            level by level (one CTA per cluster, the cluster's slice of x
//            staged in shared memory).
//   U^T x    stages P..1, levels in reverse, transposed rotations.
//   H x      diagonal on wavelet coordinates, dense core block on S_L.
//   H^-1 x   reciprocal diagonal; the core's inverse, formed once by in-place
//            Gauss-Jordan elimination (the core is symmetric positive
//            definite, so no pivoting is needed and a non-positive pivot means
//            "not SPD").
#include "apply.cuh"

#include <cooperative_groups.h>

#include <cmath>
#include <mutex>
#include <utility>
#include <vector>
#include "rotmath.cuh"

namespace pmmf {

namespace {

constexpr int AP_THREADS = 256;

// The rotation data of one stage as the apply kernels read it.
struct StageDesc {
    const int64_t *coff;
    const int32_t *members;
    const int64_t *roff;
    const int32_t *lvl_off, *nlev;
    const Rot2 *lvlrot;
    const int32_t *kidx, *kkv, *lvlidx;
    const double *kO;
    int64_t m;
    int K, pad;
};

// Shared memory of the apply kernels: the staged rotations of a cluster
// (rcap slots: its Givens rotations, fewer than its size, and its level
// offsets, at most its size + 1; rcap 0 reads both from global memory), then
// the slice of x (cluster size x right-hand sides).  Rotations are staged for
// clusters of up to APPLY_STAGE_MAX coordinates.
constexpr int64_t APPLY_STAGE_MAX = 1024;

__host__ __device__ constexpr size_t apply_smem_rot(int64_t rcap) {
    return (sizeof(Rot2) * (size_t)rcap + sizeof(int32_t) * (size_t)(rcap + 2) + 15) & ~(size_t)15;
}

// Cluster u of a stage: gather x[members][0..nr) into shared memory together
// with the cluster's level offsets and (k = 2) its rotations, apply the levels
// (in reverse, transposed, for U^T), scatter.  Staging the rotations turns
// the two dependent global loads of every level (its offsets, then each
// task's rotation) into shared-memory loads.  Ends with the scatter: a caller
// reusing the shared memory for another cluster syncs first.
template <bool TRANSPOSE, int NR>
__device__ __forceinline__ void apply_cluster(const StageDesc &a, int64_t u, unsigned char *smem,
                                              int64_t rcap, double *x, int64_t ld, int64_t r0, int nr) {
    const int64_t base = a.coff[u];
    const int c = (int)(a.coff[u + 1] - base);
    const int nl = a.nlev[u];
    if (nl == 0) return;
    Rot2 *srot = (Rot2 *)smem;
    int32_t *slo = (int32_t *)(srot + rcap);
    double *sx = (double *)(smem + apply_smem_rot(rcap));
    const int32_t *lo = a.lvl_off + a.roff[u] + u;
    const int rb = lo[0];
    const int nrot = lo[nl] - rb;
    const bool staged = nrot <= rcap;   // (the launch sets rcap >= any cluster's rotations, or 0)
    if (staged) {
        for (int L = threadIdx.x; L <= nl; L += AP_THREADS) slo[L] = lo[L] - rb;
        if (a.K == 2)
            for (int q = threadIdx.x; q < nrot; q += AP_THREADS) srot[q] = a.lvlrot[rb + q];
    }
    for (int64_t q = threadIdx.x; q < (int64_t)c * nr; q += AP_THREADS) {
        int64_t l = q / nr, r = q - l * nr;
        sx[q] = x[(int64_t)a.members[base + l] * ld + r0 + r];
    }
    __syncthreads();
    for (int Li = 0; Li < nl; ++Li) {
        const int L = TRANSPOSE ? nl - 1 - Li : Li;
        const int b0 = staged ? slo[L] : lo[L] - rb;
        const int cnt = (staged ? slo[L + 1] : lo[L + 1] - rb) - b0;
        for (int q = threadIdx.x; q < cnt * nr; q += AP_THREADS) {
            const int t = q / nr, r = q - t * nr;
            if (a.K == 2) {
                const Rot2 rt = staged ? srot[b0 + t] : a.lvlrot[rb + b0 + t];
                double va = sx[rt.li * nr + r], vb = sx[rt.lj * nr + r], na, nb;
                if (TRANSPOSE) rot_pair_t(rt.c, rt.s, va, vb, na, nb);
                else rot_pair(rt.c, rt.s, va, vb, na, nb);
                sx[rt.li * nr + r] = na;
                sx[rt.lj * nr + r] = nb;
            } else {
                // x_T' = O x_T, or x_T = O^T x_T' for the transpose (chains
                // over the block's rows of O^T, i.e. its columns)
                const int64_t tt = a.lvlidx[rb + b0 + t];
                const int kk = a.kkv[tt];
                const int32_t *T = a.kidx + tt * a.K;
                const double *O = a.kO + tt * a.K * a.K;
                double in[8], out[8], Ot[64];
                for (int k = 0; k < kk; ++k) in[k] = sx[T[k] * nr + r];
                if (TRANSPOSE) {
                    for (int k = 0; k < kk; ++k)
                        for (int l = 0; l < kk; ++l) Ot[k * kk + l] = O[l * kk + k];
                    for (int k = 0; k < kk; ++k) out[k] = rot_row(Ot, kk, k, in);
                } else {
                    for (int k = 0; k < kk; ++k) out[k] = rot_row(O, kk, k, in);
                }
                for (int k = 0; k < kk; ++k) sx[T[k] * nr + r] = out[k];
            }
        }
        __syncthreads();
    }
    for (int64_t q = threadIdx.x; q < (int64_t)c * nr; q += AP_THREADS) {
        int64_t l = q / nr, r = q - l * nr;
        x[(int64_t)a.members[base + l] * ld + r0 + r] = sx[q];
    }
}

// One CTA per cluster of one stage.
// NR > 0: nr is NR, known at compile time (the divisions by nr become shifts).
template <bool TRANSPOSE, int NR>
__global__ void __launch_bounds__(AP_THREADS)
k_apply_stage(const StageDesc a, int64_t rcap, double *x, int64_t ld, int64_t r0, int nr_rt) {
    extern __shared__ __align__(16) unsigned char smem[];
    apply_cluster<TRANSPOSE, NR>(a, blockIdx.x, smem, rcap, x, ld, r0, NR > 0 ? NR : nr_rt);
}

// Every stage of a pass in one cooperative launch: the CTAs take a stage's
// clusters in turn, and a grid barrier separates the stages (a stage reads
// what the previous one scattered), so a pass has no launch gaps.
constexpr int APPLY_MAXST = 40;
struct StagePass {
    StageDesc d[APPLY_MAXST];
    int n;
};

template <bool TRANSPOSE, int NR>
__global__ void __launch_bounds__(AP_THREADS, 6)
k_apply_all(const __grid_constant__ StagePass P, int64_t rcap, double *x, int64_t ld, int64_t r0,
            int nr_rt) {
    namespace cg = cooperative_groups;
    extern __shared__ __align__(16) unsigned char smem[];
    const int nr = NR > 0 ? NR : nr_rt;
    for (int pi = 0; pi < P.n; ++pi) {
        const StageDesc &a = P.d[TRANSPOSE ? P.n - 1 - pi : pi];
        for (int64_t u = blockIdx.x; u < a.m; u += gridDim.x) {
            apply_cluster<TRANSPOSE, NR>(a, u, smem, rcap, x, ld, r0, nr);
            __syncthreads();
        }
        if (pi + 1 < P.n) cg::this_grid().sync();
    }
}

// y = x (strided copy of an n x nrhs block)
__global__ void k_copy_block(const double *x, int64_t ldx, double *y, int64_t ldy, int64_t n,
                             int64_t nrhs) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n * nrhs;
         q += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = q / nrhs, r = q - i * nrhs;
        y[i * ldy + r] = x[i * ldx + r];
    }
}

// Wavelet part of H (MODE 0), H^-1 (1) or H^-1/2 (2) (core coordinates
// untouched here); gathers the core slice into zc.
// rc (may be NULL): the per-coordinate reciprocals of MODE 1 or 2, so the
// wavelet part is one multiply instead of an FP64 divide (and square root) per
// entry.  The product rounds twice (1/h, then v * 1/h; three times with the
// square root), so it can differ from the correctly rounded quotient by a few
// ulps, not only one; the inverse ops are therefore compared with the oracle
// to a tolerance.
// NRC > 0: nrhs is NRC, known at compile time.
template <int MODE, int NRC>
__global__ void k_h_diag(double *x, int64_t ld, int64_t n, int64_t nrhs_rt, const double *hdiag,
                         const int32_t *core_pos, double *zc, const double *rc) {
    const int64_t nrhs = NRC > 0 ? NRC : nrhs_rt;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n * nrhs;
         q += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = q / nrhs, r = q - i * nrhs;
        int32_t cp = core_pos[i];
        double v = x[i * ld + r];
        if (cp >= 0) zc[(int64_t)cp * nrhs + r] = v;
        else if (MODE != 0 && rc) x[i * ld + r] = __dmul_rn(rc[i], v);
        else x[i * ld + r] = MODE == 2 ? __ddiv_rn(v, __dsqrt_rn(hdiag[i]))
                           : MODE == 1 ? __ddiv_rn(v, hdiag[i]) : __dmul_rn(hdiag[i], v);
    }
}

template <bool ROOT>
__global__ void k_recip(const double *h, int64_t n, double *out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = ROOT ? __ddiv_rn(1.0, __dsqrt_rn(h[i])) : __ddiv_rn(1.0, h[i]);
}

// Core part: x[core_idx[a]] = sum_b C[a][b] zc[b] over the slots b of a's
// block, a sequential chain per output (a single core is one block).
__global__ void k_core_gemv(const double *C, int64_t nblk, int64_t bs, const int32_t *bdim,
                            const double *zc, int64_t nrhs, const int32_t *core_idx, double *x,
                            int64_t ld) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nblk * bs * nrhs;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = q / nrhs, r = q - a * nrhs;
        const int64_t blk = a / bs, l = a - blk * bs;
        const int64_t dim = bdim ? bdim[blk] : bs;
        if (l >= dim) continue;
        const double *row = C + blk * bs * bs + l * bs;
        const double *zb = zc + blk * bs * nrhs;
        double acc = 0.0;
        for (int64_t b = 0; b < dim; ++b) acc = __dadd_rn(acc, __dmul_rn(row[b], zb[b * nrhs + r]));
        x[(int64_t)core_idx[a] * ld + r] = acc;
    }
}

__global__ void k_wavelet_positive(const double *hdiag, const int32_t *core_pos, int64_t n,
                                   unsigned *status) {
    bool bad = false;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        if (core_pos[i] < 0 && !(hdiag[i] > 0.0)) bad = true;
    if (bad) atomicOr(status, ST_NOT_SPD);
}

// Symmetric copy of the core from its lower triangle (the part a Cholesky
// factorization would read).
__global__ void k_sym_lower(const double *C, int64_t m, double *S) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < m * m;
         q += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = q / m, j = q - i * m;
        S[q] = i >= j ? C[i * m + j] : C[j * m + i];
    }
}

__global__ void k_gj_save(const double *S, int64_t m, int64_t k, double *rowk, double *colk,
                          unsigned *status) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < m;
         q += (int64_t)gridDim.x * blockDim.x) {
        rowk[q] = S[k * m + q];
        colk[q] = S[q * m + k];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && !(S[k * m + k] > 0.0)) atomicOr(status, ST_NOT_SPD);
}

// In-place Gauss-Jordan step on pivot k: a_kk <- 1/p, a_kj <- a_kj/p,
// a_ik <- -a_ik/p, a_ij <- a_ij - a_ik a_kj / p.
__global__ void k_gj_step(double *S, int64_t m, int64_t k, const double *rowk, const double *colk) {
    const double p = rowk[k];
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < m * m;
         q += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = q / m, j = q - i * m;
        double v;
        if (i == k && j == k) v = __ddiv_rn(1.0, p);
        else if (i == k) v = __ddiv_rn(rowk[j], p);
        else if (j == k) v = -__ddiv_rn(colk[i], p);
        else v = __dsub_rn(S[q], __ddiv_rn(__dmul_rn(colk[i], rowk[j]), p));
        S[q] = v;
    }
}

// One block per CTA: symmetric copy from the lower triangle, then the same
// in-place Gauss-Jordan steps as k_gj_save / k_gj_step, in shared memory.
__global__ void k_gj_blocks(const double *C, int64_t bs, const int32_t *bdim, double *inv,
                            unsigned *status) {
    extern __shared__ double S[];
    const int64_t blk = blockIdx.x;
    const int m = bdim ? bdim[blk] : (int)bs;
    const double *Cb = C + blk * bs * bs;
    double *Ib = inv + blk * bs * bs;
    double *rowk = S + (int64_t)m * m;
    double *colk = rowk + m;
    for (int q = threadIdx.x; q < m * m; q += blockDim.x) {
        const int i = q / m, j = q - i * m;
        S[q] = i >= j ? Cb[i * bs + j] : Cb[j * bs + i];
    }
    __syncthreads();
    for (int k = 0; k < m; ++k) {
        for (int q = threadIdx.x; q < m; q += blockDim.x) {
            rowk[q] = S[k * m + q];
            colk[q] = S[q * m + k];
        }
        __syncthreads();
        const double p = rowk[k];
        if (threadIdx.x == 0 && !(p > 0.0)) atomicOr(status, ST_NOT_SPD);
        for (int q = threadIdx.x; q < m * m; q += blockDim.x) {
            const int i = q / m, j = q - i * m;
            double v;
            if (i == k && j == k) v = __ddiv_rn(1.0, p);
            else if (i == k) v = __ddiv_rn(rowk[j], p);
            else if (j == k) v = -__ddiv_rn(colk[i], p);
            else v = __dsub_rn(S[q], __ddiv_rn(__dmul_rn(colk[i], rowk[j]), p));
            S[q] = v;
        }
        __syncthreads();
    }
    for (int q = threadIdx.x; q < m * m; q += blockDim.x) {
        const int i = q / m, j = q - i * m;
        Ib[i * bs + j] = S[q];
    }
}

// ---- PCG helpers (n x nrhs row-major, ld = nrhs) ----

// y = A x for n x nrhs blocks (nrhs <= 8): a group of 8 lanes per row, lane
// r < nrhs owns right-hand side r and walks the row in order (the row's
// entries are read once per group; x rows are 8 contiguous doubles).
__global__ void k_spmv(int64_t n, const int64_t *rp, const int32_t *ci, const double *v,
                       const double *x, double *y, int nrhs) {
    const int r = threadIdx.x & 7;
    const int64_t g = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 3;
    const int64_t ng = ((int64_t)gridDim.x * blockDim.x) >> 3;
    for (int64_t i = g; i < n; i += ng) {
        if (r >= nrhs) continue;
        double acc = 0.0;
        for (int64_t q = rp[i]; q < rp[i + 1]; ++q)
            acc = __fma_rn(v[q], x[(int64_t)ci[q] * nrhs + r], acc);
        y[i * nrhs + r] = acc;
    }
}

constexpr int DOT_BLOCKS = 304;

// partial[b * nrhs + r] = sum over this block's rows of x[:, r] * y[:, r]
__global__ void k_dot_partial(const double *x, const double *y, int64_t n, int nrhs,
                              double *partial) {
    __shared__ double ws[8][8];
    double acc[8];
    for (int r = 0; r < 8; ++r) acc[r] = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        for (int r = 0; r < nrhs; ++r) acc[r] = __fma_rn(x[i * nrhs + r], y[i * nrhs + r], acc[r]);
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int r = 0; r < nrhs; ++r) {
        double s = warp_sum(acc[r]);
        if (lane == 0) ws[w][r] = s;
    }
    __syncthreads();
    if (threadIdx.x < (unsigned)nrhs) {
        double s = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += ws[q][threadIdx.x];
        partial[blockIdx.x * nrhs + threadIdx.x] = s;
    }
}

__global__ void k_dot_final(const double *partial, int nb, int nrhs, double *out) {
    int r = threadIdx.x;
    if (r < nrhs) {
        double s = 0.0;
        for (int b = 0; b < nb; ++b) s += partial[b * nrhs + r];
        out[r] = s;
    }
}

// ratio[c] = num[c] / den[c] (one divide per column, not per entry)
__global__ void k_ratio(const double *num, const double *den, int nrhs, double *ratio) {
    const int r = threadIdx.x;
    if (r < nrhs) ratio[r] = __ddiv_rn(num[r], den[r]);
}

// alpha = rz / pq on active columns; x += alpha p; r -= alpha q
__global__ void k_cg_xr(double *x, double *r, const double *p, const double *q, int64_t n,
                        int nrhs, const double *alpha, const int32_t *done) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n * nrhs;
         t += (int64_t)gridDim.x * blockDim.x) {
        int c = (int)(t % nrhs);
        if (done[c]) continue;
        const double a = alpha[c];
        x[t] = __fma_rn(a, p[t], x[t]);
        r[t] = __fma_rn(-a, q[t], r[t]);
    }
}

// beta = rz_new / rz; p = z + beta p; rz <- rz_new  (active columns)
__global__ void k_cg_p(double *p, const double *z, int64_t n, int nrhs, const double *beta,
                       const int32_t *done) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n * nrhs;
         t += (int64_t)gridDim.x * blockDim.x) {
        int c = (int)(t % nrhs);
        if (done[c]) continue;
        p[t] = __fma_rn(beta[c], p[t], z[t]);
    }
}

// Convergence of every column after iteration ++*itc: ||r|| / ||b|| <= rtol
// (same arithmetic as the host test: sqrt, then divide).
__global__ void k_cg_check(const double *rr, const double *bnorm, double rtol, int nrhs,
                           int32_t *done, int32_t *iters, int32_t *itc) {
    if (threadIdx.x != 0) return;
    const int it = ++*itc;
    for (int c = 0; c < nrhs; ++c) {
        if (done[c]) continue;
        iters[c] = it;
        if (__ddiv_rn(__dsqrt_rn(rr[c]), bnorm[c]) <= rtol) done[c] = 1;
    }
}

__global__ void k_copy_scalars(const double *src, double *dst, const int32_t *done, int nrhs) {
    int r = threadIdx.x;
    if (r < nrhs && !done[r]) dst[r] = src[r];
}

__global__ void k_sub(const double *b, const double *q, double *r, int64_t cnt) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < cnt;
         t += (int64_t)gridDim.x * blockDim.x)
        r[t] = __dsub_rn(b[t], q[t]);
}

}  // namespace

namespace {

StageDesc desc_of(const ApplyStage &a) {
    StageDesc d;
    d.coff = a.coff;
    d.members = a.members;
    d.roff = a.roff;
    d.lvl_off = a.lvl_off;
    d.nlev = a.nlev;
    d.lvlrot = a.lvlrot;
    d.kidx = a.kidx;
    d.kkv = a.kkv;
    d.lvlidx = a.lvlidx;
    d.kO = a.kO;
    d.m = a.m;
    d.K = a.K;
    d.pad = 0;
    return d;
}

// Algorithmic bytes of one stage's rotation pass: the stage's coordinates read
// and written once per right-hand side, their ids, and the rotations (24 B
// each) with their level offsets.
double stage_bytes(const ApplyStage &a, int64_t nr) {
    return 16.0 * (double)a.s * nr + 4.0 * (double)a.s + 24.0 * (double)a.nrot + 4.0 * (double)(a.nrot + a.m);
}

// Blocks of `kern` resident per SM with `sh` bytes of shared memory (asked
// once per kernel, size and device); 0 when cooperative launches are
// unavailable.
int coop_per_sm(const void *kern, size_t sh, int *nsm) {
    static std::mutex mu;
    struct Entry {
        int dev;
        const void *k;
        size_t sh;
        int per_sm, nsm;
    };
    static std::vector<Entry> seen;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    std::lock_guard<std::mutex> g(mu);
    for (const Entry &e : seen)
        if (e.dev == dev && e.k == kern && e.sh == sh) {
            *nsm = e.nsm;
            return e.per_sm;
        }
    int coop = 0, per_sm = 0, n = 0;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess) coop = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) n = 0;
    if (coop && n > 0 &&
        allow_smem(kern, sh) == cudaSuccess &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, AP_THREADS, sh) != cudaSuccess)
        per_sm = 0;
    if (!coop) per_sm = 0;
    cudaGetLastError();
    seen.push_back({dev, kern, sh, per_sm, n});
    *nsm = n;
    return per_sm;
}

// The whole pass in one cooperative launch; *done false when it cannot run.
pmmf_status apply_fused(const ApplyStages &S, bool transpose, double *x, int64_t ld, int64_t nrhs,
                        int64_t cmax, cudaStream_t st, bool *done) {
    *done = false;
    StagePass P;
    P.n = 0;
    int64_t mmax = 0;
    double bytes = 0.0;
    for (const ApplyStage &a : S) {
        if (a.nrot == 0) continue;
        if (P.n == APPLY_MAXST) return PMMF_OK;
        P.d[P.n++] = desc_of(a);
        mmax = std::max(mmax, a.m);
        bytes += stage_bytes(a, nrhs);
    }
    if (P.n == 0) {
        *done = true;
        return PMMF_OK;
    }
    int64_t rcap = cmax <= APPLY_STAGE_MAX ? cmax : 0;
    const size_t sh = apply_smem_rot(rcap) + sizeof(double) * (size_t)cmax * (size_t)nrhs;
    const void *kern = transpose ? (nrhs == 8 ? (const void *)k_apply_all<true, 8>
                                              : nrhs == 1 ? (const void *)k_apply_all<true, 1>
                                                          : (const void *)k_apply_all<true, 0>)
                                 : (nrhs == 8 ? (const void *)k_apply_all<false, 8>
                                              : nrhs == 1 ? (const void *)k_apply_all<false, 1>
                                                          : (const void *)k_apply_all<false, 0>);
    int nsm = 0;
    const int per_sm = coop_per_sm(kern, sh, &nsm);
    if (per_sm <= 0) return PMMF_OK;
    const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>(mmax, (int64_t)per_sm * nsm));
    int64_t r0 = 0;
    int nr_rt = (int)nrhs;
    void *args[] = {&P, &rcap, &x, &ld, &r0, &nr_rt};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(g);
    cfg.blockDim = dim3(AP_THREADS);
    cfg.dynamicSmemBytes = sh;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    prof_begin(KF_APPLY, st);
    PMMF_CUDA_TRY(cudaLaunchKernelExC(&cfg, kern, args));
    prof_end(KF_APPLY, st, bytes, 0.0);
    PMMF_TRY(launched("apply_all"));
    *done = true;
    return PMMF_OK;
}

}  // namespace

pmmf_status apply_rotations(const ApplyStages &S, bool transpose, double *x, int64_t ld,
                            int64_t nrhs, cudaStream_t st) {
    int64_t cmax = 0;
    for (const ApplyStage &a : S)
        if (a.nrot > 0) cmax = std::max(cmax, a.cmax);
    if (cmax == 0) return PMMF_OK;
    // one pass per launch (PMMF_TUNE_APPLY_FUSED = 2) when every right-hand
    // side fits the shared-memory slice (24 KB per cluster keeps several CTAs
    // per SM).  Measured on GB300 it is not faster than a launch per stage
    // (kNN n = 65,536, U^T H U x on 8 columns: 0.234 against 0.232 ms; 128^3
    // Poisson A~^-1 x: 1.09 against 1.00 ms): a late stage's time is its
    // clusters' chains of dependency levels, not the launch, so it runs only
    // when asked for.
    if (tuned(TUNE_APPLY_FUSED, cmax, 1) == 2 && (int64_t)(24 * 1024) / cmax >= nrhs) {
        bool done = false;
        PMMF_TRY(apply_fused(S, transpose, x, ld, nrhs, cmax, st, &done));
        if (done) return PMMF_OK;
    }
    for (size_t pi = 0; pi < S.size(); ++pi) {
        const ApplyStage &a = transpose ? S[S.size() - 1 - pi] : S[pi];
        if (a.nrot == 0) continue;
        int64_t chunk = (int64_t)(24 * 1024) / (a.cmax > 0 ? a.cmax : 1);
        if (chunk < 1) {
            set_error("apply: cluster too large for shared memory");
            return PMMF_ERR_UNSUPPORTED;
        }
        if (chunk > nrhs) chunk = nrhs;
        const StageDesc d = desc_of(a);
        for (int64_t r0 = 0; r0 < nrhs; r0 += chunk) {
            int nr = (int)(nrhs - r0 < chunk ? nrhs - r0 : chunk);
            const int64_t rcap = a.cmax <= APPLY_STAGE_MAX ? a.cmax : 0;
            size_t sh = apply_smem_rot(rcap) + sizeof(double) * (size_t)a.cmax * (size_t)nr;
            // one right-hand side and blocks of 8 (PCG's usual widths) get
            // instantiations with the width fixed
            auto kern = transpose ? (nr == 8 ? k_apply_stage<true, 8> : nr == 1 ? k_apply_stage<true, 1>
                                                                      : k_apply_stage<true, 0>)
                                  : (nr == 8 ? k_apply_stage<false, 8> : nr == 1 ? k_apply_stage<false, 1>
                                                                       : k_apply_stage<false, 0>);
            prof_begin(KF_APPLY, st);
            PMMF_CUDA_TRY(allow_smem(kern, sh));
            kern<<<(unsigned)a.m, AP_THREADS, sh, st>>>(d, rcap, x, ld, r0, nr);
            prof_end(KF_APPLY, st, stage_bytes(a, nr), 0.0);
            PMMF_TRY(launched("apply_stage"));
        }
    }
    return PMMF_OK;
}

pmmf_status copy_block(const double *x, int64_t ldx, double *y, int64_t ldy, int64_t n,
                       int64_t nrhs, cudaStream_t st) {
    if (ldx == nrhs && ldy == nrhs) {
        // contiguous: one device copy, no per-entry index arithmetic
        if (n * nrhs > 0)
            PMMF_CUDA_TRY(cudaMemcpyAsync(y, x, sizeof(double) * (size_t)(n * nrhs),
                                          cudaMemcpyDeviceToDevice, st));
        return PMMF_OK;
    }
    k_copy_block<<<grid_for(n * nrhs, 256), 256, 0, st>>>(x, ldx, y, ldy, n, nrhs);
    return launched("copy_block");
}

pmmf_status h_reciprocals(const double *hdiag, int64_t n, bool root, double *out, cudaStream_t st) {
    if (n <= 0) return PMMF_OK;
    if (root) k_recip<true><<<grid_for(n, 256), 256, 0, st>>>(hdiag, n, out);
    else k_recip<false><<<grid_for(n, 256), 256, 0, st>>>(hdiag, n, out);
    return launched("h_reciprocals");
}

pmmf_status apply_h_scratch(const HData &H, int mode, double *x, int64_t ld, int64_t nrhs,
                            double *zc, cudaStream_t st) {
    const unsigned g = grid_for(H.n * nrhs, 256);
    // blocks of 8 right-hand sides (PCG's usual width) with the width fixed
    if (nrhs == 8) {
        if (mode == 2) k_h_diag<2, 8><<<g, 256, 0, st>>>(x, ld, H.n, nrhs, H.hdiag, H.core_pos, zc, H.hisr);
        else if (mode == 1) k_h_diag<1, 8><<<g, 256, 0, st>>>(x, ld, H.n, nrhs, H.hdiag, H.core_pos, zc, H.hrcp);
        else k_h_diag<0, 8><<<g, 256, 0, st>>>(x, ld, H.n, nrhs, H.hdiag, H.core_pos, zc, nullptr);
    } else {
        if (mode == 2) k_h_diag<2, 0><<<g, 256, 0, st>>>(x, ld, H.n, nrhs, H.hdiag, H.core_pos, zc, H.hisr);
        else if (mode == 1) k_h_diag<1, 0><<<g, 256, 0, st>>>(x, ld, H.n, nrhs, H.hdiag, H.core_pos, zc, H.hrcp);
        else k_h_diag<0, 0><<<g, 256, 0, st>>>(x, ld, H.n, nrhs, H.hdiag, H.core_pos, zc, nullptr);
    }
    PMMF_TRY(launched("h_diag"));
    const double *C = mode == 2 ? H.core_isqrt : mode == 1 ? H.core_inv : H.core;
    k_core_gemv<<<grid_for(H.m * nrhs, 64), 64, 0, st>>>(C, H.nblk, H.bs, H.bdim, zc, nrhs,
                                                         H.core_idx, x, ld);
    return launched("core_gemv");
}

pmmf_status apply_h_scratch(const HData &H, bool inverse, double *x, int64_t ld, int64_t nrhs,
                            double *zc, cudaStream_t st) {
    return apply_h_scratch(H, inverse ? 1 : 0, x, ld, nrhs, zc, st);
}

pmmf_status apply_h(const HData &H, int mode, double *x, int64_t ld, int64_t nrhs,
                    cudaStream_t st) {
    DBuf<double> zc;
    PMMF_TRY(zc.alloc(H.m * nrhs, st));
    return apply_h_scratch(H, mode, x, ld, nrhs, zc.p, st);
}

pmmf_status apply_h(const HData &H, bool inverse, double *x, int64_t ld, int64_t nrhs,
                    cudaStream_t st) {
    return apply_h(H, inverse ? 1 : 0, x, ld, nrhs, st);
}

pmmf_status invert_core_blocks(const double *core, int64_t nblk, int64_t bs, const int32_t *bdim,
                               const double *hdiag, const int32_t *core_pos, int64_t n,
                               double *inv, unsigned *status, cudaStream_t st) {
    k_wavelet_positive<<<grid_for(n, 256), 256, 0, st>>>(hdiag, core_pos, n, status);
    PMMF_TRY(launched("wavelet_positive"));
    if (nblk == 0 || bs == 0) return PMMF_OK;
    const size_t sh = sizeof(double) * (size_t)(bs * bs + 2 * bs);
    if (sh > 220 * 1024) {
        set_error("core blocks too large to invert in shared memory");
        return PMMF_ERR_UNSUPPORTED;
    }
    PMMF_CUDA_TRY(allow_smem(k_gj_blocks, sh));
    k_gj_blocks<<<(unsigned)nblk, 256, sh, st>>>(core, bs, bdim, inv, status);
    return launched("gj_blocks");
}

pmmf_status invert_core(const double *core, int64_t m, const double *hdiag, const int32_t *core_pos,
                        int64_t n, double *inv, unsigned *status, cudaStream_t st) {
    k_wavelet_positive<<<grid_for(n, 256), 256, 0, st>>>(hdiag, core_pos, n, status);
    PMMF_TRY(launched("wavelet_positive"));
    k_sym_lower<<<grid_for(m * m, 256), 256, 0, st>>>(core, m, inv);
    PMMF_TRY(launched("sym_lower"));
    DBuf<double> rowk, colk;
    PMMF_TRY(rowk.alloc(m, st));
    PMMF_TRY(colk.alloc(m, st));
    for (int64_t k = 0; k < m; ++k) {
        k_gj_save<<<grid_for(m, 256), 256, 0, st>>>(inv, m, k, rowk.p, colk.p, status);
        PMMF_TRY(launched("gj_save"));
        k_gj_step<<<grid_for(m * m, 256), 256, 0, st>>>(inv, m, k, rowk.p, colk.p);
        PMMF_TRY(launched("gj_step"));
    }
    return PMMF_OK;
}

// ---- core inverse square root (Sec. 4, xi = 1/2) --------------------------
// The coupled Newton-Schulz iteration for S^{1/2} and S^{-1/2} of a symmetric
// positive definite S scaled into the unit ball (Higham, Functions of
// Matrices, Sec. 6.3): Y_0 = S / alpha, Z_0 = I,
//   T = (3 I - Z Y) / 2,  Y <- Y T,  Z <- T Z,
// with Z -> (S / alpha)^{-1/2} quadratically once Z Y is near I.  Every step
// is a dense product, which is what a GPU does well; the eigendecomposition
// the definition suggests is a long chain of dependent rotations.
constexpr int NS_TILE = 64, NS_KT = 16, NS_THREADS = 256, NS_MAXIT = 100;

// Per core block: alpha = ||S||_F of the block's d x d symmetric core (lower
// triangle mirrored); Y = S / alpha with the identity on the padding, Z = I.
__global__ void __launch_bounds__(NS_THREADS) k_ns_init(const double *C, int64_t bs,
                                                        const int32_t *bdim, double *Y, double *Z,
                                                        double *alpha, unsigned *status) {
    __shared__ double red[NS_THREADS];
    const int64_t blk = blockIdx.x;
    const int64_t d = bdim ? bdim[blk] : bs;
    const double *Cb = C + blk * bs * bs;
    double acc = 0.0;
    for (int64_t q = threadIdx.x; q < d * d; q += NS_THREADS) {
        const int64_t i = q / d, j = q - i * d;
        const double v = i >= j ? Cb[i * bs + j] : Cb[j * bs + i];
        acc = __fma_rn(v, v, acc);
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = NS_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] = __dadd_rn(red[threadIdx.x], red[threadIdx.x + w]);
        __syncthreads();
    }
    double a = d > 0 ? __dsqrt_rn(red[0]) : 1.0;
    if (!(a > 0.0 && a < INFINITY)) {
        if (threadIdx.x == 0) atomicOr(status, ST_NOT_SPD);
        a = 1.0;
    }
    if (threadIdx.x == 0) alpha[blk] = a;
    double *Yb = Y + blk * bs * bs, *Zb = Z + blk * bs * bs;
    for (int64_t q = threadIdx.x; q < bs * bs; q += NS_THREADS) {
        const int64_t i = q / bs, j = q - i * bs;
        Yb[q] = i < d && j < d ? __ddiv_rn(i >= j ? Cb[i * bs + j] : Cb[j * bs + i], a)
                               : (i == j ? 1.0 : 0.0);
        Zb[q] = i == j ? 1.0 : 0.0;
    }
}

// C_b = A_b B_b for every bs x bs block b = blockIdx.z; 64 x 64 output tile
// per CTA, 4 x 4 outputs per thread, k staged 16 at a time in shared memory.
// EPI: C <- (3 I - A B) / 2, and the tile's sum of (A B - I)^2 over the
// block's d x d part goes to part[b * tiles + tile].
template <bool EPI>
__global__ void __launch_bounds__(NS_THREADS) k_ns_gemm(const double *A, const double *B,
                                                        double *C, int64_t bs,
                                                        const int32_t *bdim, double *part) {
    __shared__ double As[NS_KT][NS_TILE + 1];
    __shared__ double Bs[NS_KT][NS_TILE];
    __shared__ double red[NS_THREADS];
    const int64_t blk = blockIdx.z;
    const double *Ab = A + blk * bs * bs, *Bb = B + blk * bs * bs;
    double *Cb = C + blk * bs * bs;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int64_t r0 = (int64_t)blockIdx.y * NS_TILE, c0 = (int64_t)blockIdx.x * NS_TILE;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    for (int64_t k0 = 0; k0 < bs; k0 += NS_KT) {
        for (int e = threadIdx.x; e < NS_TILE * NS_KT; e += NS_THREADS) {
            const int ra = e / NS_KT, ka = e - ra * NS_KT;
            const int64_t gr = r0 + ra, gk = k0 + ka;
            As[ka][ra] = gr < bs && gk < bs ? Ab[gr * bs + gk] : 0.0;
            const int kb = e / NS_TILE, cb = e - kb * NS_TILE;
            const int64_t gk2 = k0 + kb, gc = c0 + cb;
            Bs[kb][cb] = gk2 < bs && gc < bs ? Bb[gk2 * bs + gc] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < NS_KT; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = __fma_rn(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
    const int64_t d = bdim ? bdim[blk] : bs;
    double ssq = 0.0;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t gr = r0 + ty + 16 * i, gc = c0 + tx + 16 * j;
            if (gr >= bs || gc >= bs) continue;
            double v = acc[i][j];
            if (EPI) {
                const double e = gr == gc ? __dsub_rn(v, 1.0) : v;
                if (gr < d && gc < d) ssq = __fma_rn(e, e, ssq);
                v = __dsub_rn(gr == gc ? 1.5 : 0.0, __dmul_rn(0.5, v));
            }
            Cb[gr * bs + gc] = v;
        }
    if (EPI) {
        red[threadIdx.x] = ssq;
        __syncthreads();
        for (int w = NS_THREADS / 2; w > 0; w >>= 1) {
            if (threadIdx.x < w) red[threadIdx.x] = __dadd_rn(red[threadIdx.x], red[threadIdx.x + w]);
            __syncthreads();
        }
        if (threadIdx.x == 0)
            part[blk * (int64_t)(gridDim.x * gridDim.y) + blockIdx.y * gridDim.x + blockIdx.x] = red[0];
    }
}

// out[0] = max over blocks of ||Z Y - I||_F (tile partials summed in a fixed
// order); a NaN anywhere gives NaN.
__global__ void __launch_bounds__(NS_THREADS) k_ns_resid(const double *part, int64_t nblk,
                                                         int tiles, double *out) {
    __shared__ double red[NS_THREADS];
    double mx = 0.0;
    for (int64_t b = threadIdx.x; b < nblk; b += NS_THREADS) {
        double sum = 0.0;
        for (int t = 0; t < tiles; ++t) sum = __dadd_rn(sum, part[b * tiles + t]);
        if (!(sum <= mx)) mx = sum;
    }
    red[threadIdx.x] = mx;
    __syncthreads();
    for (int w = NS_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w && !(red[threadIdx.x + w] <= red[threadIdx.x]))
            red[threadIdx.x] = red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = __dsqrt_rn(red[0]);
}

// out = (Z + Z^T) / (2 sqrt(alpha)) on each block's d x d part, 0 on the padding.
__global__ void k_ns_finish(const double *Z, int64_t nblk, int64_t bs, const int32_t *bdim,
                            const double *alpha, double *out) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nblk * bs * bs;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t blk = q / (bs * bs), l = q - blk * bs * bs;
        const int64_t i = l / bs, j = l - i * bs;
        const int64_t d = bdim ? bdim[blk] : bs;
        const double *Zb = Z + blk * bs * bs;
        out[q] = i < d && j < d
                     ? __ddiv_rn(__dmul_rn(0.5, __dadd_rn(Zb[i * bs + j], Zb[j * bs + i])),
                                 __dsqrt_rn(alpha[blk]))
                     : 0.0;
    }
}

pmmf_status core_inverse_sqrt(const double *core, int64_t nblk, int64_t bs, const int32_t *bdim,
                              const double *hdiag, const int32_t *core_pos, int64_t n,
                              double *out, unsigned *status, int *iterations, cudaStream_t st) {
    k_wavelet_positive<<<grid_for(n, 256), 256, 0, st>>>(hdiag, core_pos, n, status);
    PMMF_TRY(launched("wavelet_positive"));
    if (iterations) *iterations = 0;
    if (nblk == 0 || bs == 0) return PMMF_OK;
    const int64_t bb = nblk * bs * bs;
    const int tx = (int)((bs + NS_TILE - 1) / NS_TILE);
    if (nblk > 65535) {
        set_error("too many core blocks for the inverse square root");
        return PMMF_ERR_UNSUPPORTED;
    }
    DBuf<double> Y, Z, Y2, Z2, T, alpha, part, res;
    PMMF_TRY(Y.alloc(bb, st));
    PMMF_TRY(Z.alloc(bb, st));
    PMMF_TRY(Y2.alloc(bb, st));
    PMMF_TRY(Z2.alloc(bb, st));
    PMMF_TRY(T.alloc(bb, st));
    PMMF_TRY(alpha.alloc(nblk, st));
    PMMF_TRY(part.alloc(nblk * tx * tx, st));
    PMMF_TRY(res.alloc(1, st));
    k_ns_init<<<(unsigned)nblk, NS_THREADS, 0, st>>>(core, bs, bdim, Y.p, Z.p, alpha.p, status);
    PMMF_TRY(launched("ns_init"));
    const dim3 grid((unsigned)tx, (unsigned)tx, (unsigned)nblk);
    double *y = Y.p, *z = Z.p, *y2 = Y2.p, *z2 = Z2.p;
    double prev = INFINITY, r = INFINITY;
    bool conv = false;
    int it = 0;
    for (; it < NS_MAXIT; ++it) {
        k_ns_gemm<true><<<grid, NS_THREADS, 0, st>>>(z, y, T.p, bs, bdim, part.p);
        PMMF_TRY(launched("ns_gemm"));
        k_ns_resid<<<1, NS_THREADS, 0, st>>>(part.p, nblk, tx * tx, res.p);
        PMMF_TRY(launched("ns_resid"));
        PMMF_CUDA_TRY(cudaMemcpyAsync(&r, res.p, sizeof(double), cudaMemcpyDeviceToHost, st));
        PMMF_CUDA_TRY(cudaStreamSynchronize(st));
        // converged: at the rounding floor, or no longer contracting once
        // quadratic convergence has brought the residual near it
        if (r <= 1e-15 * (double)bs || (r <= 1e-6 && r > 0.25 * prev)) {
            conv = true;
            break;
        }
        if (!(r < 1e12)) break;     // diverging (an eigenvalue <= 0) or NaN
        k_ns_gemm<false><<<grid, NS_THREADS, 0, st>>>(y, T.p, y2, bs, bdim, nullptr);
        PMMF_TRY(launched("ns_gemm"));
        k_ns_gemm<false><<<grid, NS_THREADS, 0, st>>>(T.p, z, z2, bs, bdim, nullptr);
        PMMF_TRY(launched("ns_gemm"));
        std::swap(y, y2);
        std::swap(z, z2);
        prev = r;
    }
    if (iterations) *iterations = it;
    if (!conv && !(r <= 1e-6)) {
        set_error("core is not positive definite (its inverse square root did not converge)");
        return PMMF_ERR_NOT_SPD;
    }
    k_ns_finish<<<grid_for(bb, 256), 256, 0, st>>>(z, nblk, bs, bdim, alpha.p, out);
    return launched("ns_finish");
}

pmmf_status spmv(const DevCsr &A, const double *x, double *y, int nrhs, cudaStream_t st) {
    k_spmv<<<grid_for(A.n * 8, 256), 256, 0, st>>>(A.n, A.rp, A.ci, A.v, x, y, nrhs);
    return launched("spmv");
}

pmmf_status dots(const double *x, const double *y, int64_t n, int nrhs, double *out,
                 double *partial, cudaStream_t st) {
    k_dot_partial<<<DOT_BLOCKS, 256, 0, st>>>(x, y, n, nrhs, partial);
    PMMF_TRY(launched("dot_partial"));
    k_dot_final<<<1, 32, 0, st>>>(partial, DOT_BLOCKS, nrhs, out);
    return launched("dot_final");
}

int64_t dot_partial_size(int nrhs) { return (int64_t)DOT_BLOCKS * nrhs; }

pmmf_status cg_update_xr(double *x, double *r, const double *p, const double *q, int64_t n,
                         int nrhs, const double *rz, const double *pq, const int32_t *done,
                         double *alpha, cudaStream_t st) {
    k_ratio<<<1, 32, 0, st>>>(rz, pq, nrhs, alpha);
    PMMF_TRY(launched("ratio"));
    k_cg_xr<<<grid_for(n * nrhs, 256), 256, 0, st>>>(x, r, p, q, n, nrhs, alpha, done);
    return launched("cg_xr");
}

pmmf_status cg_update_p(double *p, const double *z, int64_t n, int nrhs, const double *rznew,
                        double *rz, const int32_t *done, double *beta, cudaStream_t st) {
    k_ratio<<<1, 32, 0, st>>>(rznew, rz, nrhs, beta);
    PMMF_TRY(launched("ratio"));
    k_cg_p<<<grid_for(n * nrhs, 256), 256, 0, st>>>(p, z, n, nrhs, beta, done);
    PMMF_TRY(launched("cg_p"));
    k_copy_scalars<<<1, 32, 0, st>>>(rznew, rz, done, nrhs);
    return launched("copy_scalars");
}

pmmf_status cg_check(const double *rr, const double *bnorm, double rtol, int nrhs, int32_t *done,
                     int32_t *iters, int32_t *itc, cudaStream_t st) {
    k_cg_check<<<1, 32, 0, st>>>(rr, bnorm, rtol, nrhs, done, iters, itc);
    return launched("cg_check");
}

pmmf_status vec_sub(const double *b, const double *q, double *r, int64_t cnt, cudaStream_t st) {
    k_sub<<<grid_for(cnt, 256), 256, 0, st>>>(b, q, r, cnt);
    return launched("sub");
}

}  // namespace pmmf

namespace pmmf {

// H or H^-1 with caller-provided scratch for the core slice (H.m * nrhs
// doubles); used by the allocation-free entry point.

}  // namespace pmmf
