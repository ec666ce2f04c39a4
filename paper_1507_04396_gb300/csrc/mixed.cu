// mixed.cu -- the rotation search with a low-precision Gram shortlist.
//
// The cluster's Gram matrix is formed on the tensor cores from a TF32 or BF16
// split of its rows, x = hi + lo with hi = round(x), lo = round(x - hi), as
// hi hi^T + hi lo^T + lo hi^T with FP32 accumulation over chunks of 128 terms
// and FP64 accumulation of the chunks.  That matrix only screens partners:
// for the pivot row i every candidate j gets a score interval
//   |G~_ij| w_j -/+ B_ij w_j,
// where B bounds |G~ - G| entry by entry (initially eps sqrt(G_ii G_jj) with
// eps from the input rounding and the FP32 accumulation over s terms, then
// carried through every rotation of G~ with the rotation's own rounding
// added), and w_j = 1/sqrt(G_jj) with G_jj kept in FP64.  Every candidate
// whose interval reaches the (k-1)-th largest lower end is re-scored in FP64
// from the FP64 rows, and the partners are the best FP64 scores (ties to the
// smaller index), as in FP64 mode.  The angle uses FP64 Gram entries (dot
// products of the current rows), the rows themselves are rotated in FP64, and
// the FP64 diagonal follows the FP64 k x k block.  Only the Gram matrix, its
// error bound and their rotation are in reduced precision.
#include <climits>
#include <cmath>

#include <cooperative_groups.h>
#include <cuda_bf16.h>

#include <vector>

#include "dense.cuh"
#include "mixed.cuh"

namespace pmmf {
namespace {

namespace cg = cooperative_groups;

constexpr int MX_THREADS = 512;
constexpr int PAIRS = 28;            // tuple pairs (k <= 8)
constexpr int MX_WARPS = MX_THREADS / 32;
constexpr int SL_MAX = 64;           // shortlists above this are counted as long
constexpr int DOT_BATCH = 8;

__device__ __forceinline__ uint64_t mixm(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t drawm(uint64_t seed, uint64_t p, uint64_t u, uint64_t t) {
    uint64_t h = mixm(seed);
    h = mixm(h ^ p);
    h = mixm(h ^ u);
    return mixm(h ^ t);
}

__device__ int nth_set(const uint32_t *mask, int nwords, int64_t pos) {
    int rem = (int)pos;
    for (int wi = 0; wi < nwords; ++wi) {
        const uint32_t m = mask[wi];
        const int pc = __popc(m);
        if (rem < pc) {
            for (int b = 0; b < 32; ++b)
                if ((m >> b) & 1u) {
                    if (rem == 0) return wi * 32 + b;
                    --rem;
                }
        }
        rem -= pc;
    }
    return -1;
}

__device__ __forceinline__ bool on(const uint32_t *mask, int y) { return (mask[y >> 5] >> (y & 31)) & 1u; }

// ---------------------------------------------------------------- slab

// Row q of the slab = row pos[members[q]] of D (cluster order), in FP64 and in
// the reduced precision (TF32: round to nearest, ties away, kept in a float;
// BF16: round to nearest even).
// The reduced-precision rows have stride sp (s rounded up to even for BF16,
// the padding zero): XH = round(x), XL = round(x - XH) (TF32: round to nearest,
// ties away, kept in a float; BF16: round to nearest even).
template <int PREC>
__global__ void k_build_slab(const double *D, int64_t s, int64_t sp, const int32_t *pos,
                             const int32_t *members, double *X, void *XH, void *XL) {
    const int64_t q = blockIdx.x;
    const double *src = D + (int64_t)pos[members[q]] * s;
    for (int64_t r = threadIdx.x; r < sp; r += blockDim.x) {
        const double v = r < s ? src[r] : 0.0;
        if (r < s) X[q * s + r] = v;
        if (PREC == PMMF_PREC_TF32) {
            const float f = __double2float_rn(v);
            uint32_t h, l;
            asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(f));
            const float rest = __double2float_rn(v - (double)__uint_as_float(h));
            asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l) : "f"(rest));
            ((uint32_t *)XH)[q * sp + r] = h;
            ((uint32_t *)XL)[q * sp + r] = l;
        } else {
            const __nv_bfloat16 h = __float2bfloat16_rn(__double2float_rn(v));
            const __nv_bfloat16 l = __float2bfloat16_rn(__double2float_rn(v - (double)__bfloat162float(h)));
            ((__nv_bfloat16 *)XH)[q * sp + r] = h;
            ((__nv_bfloat16 *)XL)[q * sp + r] = l;
        }
    }
}

// FP64 squared norms of the slab rows (warp per row, fixed order).
__global__ void k_row_norms(const double *X, int64_t rows, int64_t s, double *out) {
    const int lane = threadIdx.x & 31;
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t q = w; q < rows; q += nw) {
        double acc = 0.0;
        for (int64_t r = lane; r < s; r += 32) acc = __fma_rn(X[q * s + r], X[q * s + r], acc);
        acc = warp_sum(acc);
        if (lane == 0) out[q] = acc;
    }
}

// Local symmetric blocks M^u_ab = D[x_min][x_max] (one CTA per cluster).
__global__ void k_local_block(const double *D, int64_t s, const int32_t *pos, const int64_t *coff,
                              const int32_t *members, const int64_t *goff, double *M) {
    const int64_t u = blockIdx.x;
    const int64_t base = coff[u];
    const int64_t c = coff[u + 1] - base;
    double *Mu = M + goff[u];
    for (int64_t q = threadIdx.x; q < c * c; q += blockDim.x) {
        const int64_t a = q / c, b = q - a * c;
        const int64_t pa = pos[members[base + (a < b ? a : b)]];
        const int64_t pb = pos[members[base + (a < b ? b : a)]];
        Mu[q] = D[pa * s + pb];
    }
}

// ---------------------------------------------------------------- tensor-core Gram

// mma.sync fragments (PTX ISA, warp-level MMA):
//   m16n8k16 BF16: A a0..a3 = rows (g, g+8), k pairs (2t, 2t+1) and (2t+8, 2t+9);
//                  B b0, b1 = k pairs (2t, 2t+1), (2t+8, 2t+9) of column g;
//   m16n8k8 TF32:  A a0..a3 = (g, t), (g+8, t), (g, t+4), (g+8, t+4);
//                  B b0, b1 = (t, g), (t+4, g);
//   C c0..c3 = (g, 2t), (g, 2t+1), (g+8, 2t), (g+8, 2t+1);  g = lane / 4, t = lane % 4.
constexpr int TG = 64;      // output tile
constexpr int TKB = 32;     // k chunk staged in shared memory (elements)
constexpr int KFLUSH = 16;  // FP32 accumulation length before the chunk sum is
                            // added into the compensated sum (a multiple of the
                            // MMA's k step): the FP32 part of the certified bound
                            // grows with it, the additions shrink

__device__ __forceinline__ void mma_bf16(float *d, const uint32_t *a, const uint32_t *b) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ void mma_tf32(float *d, const uint32_t *a, const uint32_t *b) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// One CTA (4 warps, each a 32 x 32 patch) per 64 x 64 tile (ta <= tb) of one
// cluster's Gram block: hi hi^T + hi lo^T + lo hi^T on the tensor cores.
template <int PREC>
__global__ void __launch_bounds__(128)
k_tc_gram(const void *XH, const void *XL, int64_t sp /* padded row length */,
          const int64_t *coff, const int64_t *goff, const int32_t *tu, const int32_t *ta,
          const int32_t *tb, float *G) {
    // operand tiles as 32-bit words: BF16 pairs or TF32 values
    constexpr int WPR = PREC == PMMF_PREC_BF16 ? TKB / 2 : TKB;   // words per row per chunk
    __shared__ uint32_t Ah[TG][WPR + 4], Al[TG][WPR + 4], Bh[TG][WPR + 4], Bl[TG][WPR + 4];
    const int64_t u = tu[blockIdx.x];
    const int64_t base = coff[u];
    const int c = (int)(coff[u + 1] - base);
    const int a0 = ta[blockIdx.x] * TG, b0 = tb[blockIdx.x] * TG;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    float acc[2][4][4];
    float shi[2][4][4], slo[2][4][4];   // compensated sums of the chunk sums
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 4; ++j)
            for (int q = 0; q < 4; ++q) {
                acc[i][j][q] = 0.0f;
                shi[i][j][q] = 0.0f;
                slo[i][j][q] = 0.0f;
            }
    const uint32_t *WH = (const uint32_t *)XH, *WL = (const uint32_t *)XL;
    const int64_t wrow = PREC == PMMF_PREC_BF16 ? sp / 2 : sp;   // words per row
    for (int64_t k0 = 0; k0 < sp; k0 += TKB) {
        const int64_t kw0 = PREC == PMMF_PREC_BF16 ? k0 / 2 : k0;
        const int64_t kwl = wrow - kw0;                            // words left in the row
        for (int q = tid; q < TG * WPR; q += 128) {
            const int r = q / WPR, kw = q - r * WPR;
            const bool okk = kw < kwl;
            const bool oa = a0 + r < c && okk, ob = b0 + r < c && okk;
            const int64_t ia = (base + a0 + r) * wrow + kw0 + kw, ib = (base + b0 + r) * wrow + kw0 + kw;
            Ah[r][kw] = oa ? WH[ia] : 0u;
            Al[r][kw] = oa ? WL[ia] : 0u;
            Bh[r][kw] = ob ? WH[ib] : 0u;
            Bl[r][kw] = ob ? WL[ib] : 0u;
        }
        __syncthreads();
        constexpr int KSTEP = PREC == PMMF_PREC_BF16 ? 16 : 8;
        for (int kk = 0; kk < TKB / KSTEP; ++kk) {
            const int kb = kk * 8;   // word offset of this k step (8 words either way)
            uint32_t ah[2][4], al[2][4], bh[4][2], bl[4][2];
            for (int i = 0; i < 2; ++i) {
                const int r = wm + i * 16;
                ah[i][0] = Ah[r + g][kb + t];
                ah[i][1] = Ah[r + g + 8][kb + t];
                ah[i][2] = Ah[r + g][kb + t + 4];
                ah[i][3] = Ah[r + g + 8][kb + t + 4];
                al[i][0] = Al[r + g][kb + t];
                al[i][1] = Al[r + g + 8][kb + t];
                al[i][2] = Al[r + g][kb + t + 4];
                al[i][3] = Al[r + g + 8][kb + t + 4];
            }
            for (int j = 0; j < 4; ++j) {
                const int n = wn + j * 8 + g;
                bh[j][0] = Bh[n][kb + t];
                bh[j][1] = Bh[n][kb + t + 4];
                bl[j][0] = Bl[n][kb + t];
                bl[j][1] = Bl[n][kb + t + 4];
            }
            for (int i = 0; i < 2; ++i)
                for (int j = 0; j < 4; ++j) {
                    if (PREC == PMMF_PREC_BF16) {
                        mma_bf16(acc[i][j], al[i], bh[j]);
                        mma_bf16(acc[i][j], ah[i], bl[j]);
                        mma_bf16(acc[i][j], ah[i], bh[j]);
                    } else {
                        mma_tf32(acc[i][j], al[i], bh[j]);
                        mma_tf32(acc[i][j], ah[i], bl[j]);
                        mma_tf32(acc[i][j], ah[i], bh[j]);
                    }
                }
            // every KFLUSH terms the chunk sums move into the compensated sums
            if (((kk + 1) * KSTEP) % KFLUSH == 0) {
                for (int i = 0; i < 2; ++i)
                    for (int j = 0; j < 4; ++j)
                        for (int q = 0; q < 4; ++q) {
                            two_sum_acc(shi[i][j][q], slo[i][j][q], acc[i][j][q]);
                            acc[i][j][q] = 0.0f;
                        }
            }
        }
        __syncthreads();
    }
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 4; ++j)
            for (int q = 0; q < 4; ++q) two_sum_acc(shi[i][j][q], slo[i][j][q], acc[i][j][q]);
    float *Gu = G + goff[u];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 4; ++j)
            for (int q = 0; q < 4; ++q) {
                const int a = a0 + wm + i * 16 + g + (q >= 2 ? 8 : 0);
                const int b = b0 + wn + j * 8 + 2 * t + (q & 1);
                // on a diagonal tile only a <= b is taken (both positions):
                // (a, b) and (b, a) are separate sums there, and one of them
                // must fill both places
                if (a < c && b < c && (a0 != b0 || a <= b)) {
                    // hi + lo once, in FP64, then rounded to the stored FP32
                    const float f = __double2float_rn(__dadd_rn((double)shi[i][j][q], (double)slo[i][j][q]));
                    Gu[(int64_t)a * c + b] = f;
                    Gu[(int64_t)b * c + a] = f;
                }
            }
}

// ---------------------------------------------------------------- search

__device__ __forceinline__ double block_max(double v, double *red) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    // the MX_WARPS maxima by shuffles (max is exact, so any order gives the
    // same value) rather than a serial loop in every thread: each FP64
    // instruction a warp issues holds the SM's FP64 pipe
    double r = red[lane % MX_WARPS];
    for (int o = MX_WARPS / 2; o > 0; o >>= 1) r = fmax(r, __shfl_xor_sync(0xffffffffu, r, o));
    return r;
}

// Partial dot products of row xi with the rows xs[0..nb) over the columns
// [r0, r1) (this CTA's slice), reduced over the CTA in a fixed order; thread b
// < nb returns the b-th sum (others 0).  Ends with a barrier.  Each thread
// adds its columns in ascending order; the loops over the batch are unrolled
// (sums and row pointers in registers) and two columns' loads are issued
// together.
__device__ double slice_dots(const double *xi, const double *const *xs, int nb, int64_t r0,
                             int64_t r1, double *red) {
    double acc[DOT_BATCH];
    const double *p[DOT_BATCH];
#pragma unroll
    for (int b = 0; b < DOT_BATCH; ++b) {
        acc[b] = 0.0;
        p[b] = xs[b];
    }
    int64_t r = r0 + threadIdx.x;
    for (; r + MX_THREADS < r1; r += 2 * MX_THREADS) {
        const double a0 = xi[r], a1 = xi[r + MX_THREADS];
        double v0[DOT_BATCH], v1[DOT_BATCH];
#pragma unroll
        for (int b = 0; b < DOT_BATCH; ++b) {
            v0[b] = b < nb ? p[b][r] : 0.0;
            v1[b] = b < nb ? p[b][r + MX_THREADS] : 0.0;
        }
#pragma unroll
        for (int b = 0; b < DOT_BATCH; ++b)
            if (b < nb) {
                acc[b] = __fma_rn(a0, v0[b], acc[b]);
                acc[b] = __fma_rn(a1, v1[b], acc[b]);
            }
    }
    if (r < r1) {
        const double a0 = xi[r];
#pragma unroll
        for (int b = 0; b < DOT_BATCH; ++b)
            if (b < nb) acc[b] = __fma_rn(a0, p[b][r], acc[b]);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    // the warp's 8 sums by a halving butterfly: at lane distance 16, 8, 4
    // each lane keeps half of its sums (added to the partner's) and sends the
    // other half, so lane L ends with the sum b = bits 4, 3, 2 of L over the
    // lanes that share bits 0-1, completed at distances 2 and 1 (9 FP64 adds
    // per lane instead of 8 full warp sums of 5)
    static_assert(DOT_BATCH == 8, "the butterfly below halves 8 sums three times");
    {
        const bool h4 = lane & 16, h3 = lane & 8, h2 = lane & 4;
        double k4[4], k3[2];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const double snd = h4 ? acc[j] : acc[4 + j];
            k4[j] = __dadd_rn(h4 ? acc[4 + j] : acc[j], __shfl_xor_sync(0xffffffffu, snd, 16));
        }
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const double snd = h3 ? k4[j] : k4[2 + j];
            k3[j] = __dadd_rn(h3 ? k4[2 + j] : k4[j], __shfl_xor_sync(0xffffffffu, snd, 8));
        }
        double k2 = __dadd_rn(h2 ? k3[1] : k3[0], __shfl_xor_sync(0xffffffffu, h2 ? k3[0] : k3[1], 4));
        k2 = __dadd_rn(k2, __shfl_xor_sync(0xffffffffu, k2, 2));
        k2 = __dadd_rn(k2, __shfl_xor_sync(0xffffffffu, k2, 1));
        const int b = (h4 ? 4 : 0) + (h3 ? 2 : 0) + (h2 ? 1 : 0);
        if ((lane & 3) == 0 && b < nb) red[b * MX_WARPS + w] = k2;
    }
    __syncthreads();
    double v = 0.0;
    if (threadIdx.x < (unsigned)nb)
        for (int q = 0; q < MX_WARPS; ++q) v = __dadd_rn(v, red[threadIdx.x * MX_WARPS + q]);
    __syncthreads();
    return v;
}

// The search of one cluster by CL CTAs (a thread-block cluster for CL > 1):
// every CTA runs the step's decisions (scores, shortlist, angles, bookkeeping)
// on its own copy of G~, B and M, with identical inputs and so identical
// results, while the long FP64 work is split by columns of the FP64 rows:
// CTA r computes the shortlist's dot products over its slice of the s columns
// (the partial sums go to every CTA's shared memory, double-buffered by step
// parity, and are added in rank order after one cluster barrier) and rotates
// its slice of the rows.  Only CTA 0 writes the results.
// KM: the largest tuple (3 for k <= 3, 8 otherwise); the tuple's arrays are
// sized by it and their loops unrolled, so they stay in registers.
template <int CL, int KM>
__global__ void __launch_bounds__(MX_THREADS)
k_select_mixed(int64_t s, const int64_t *coff, const int32_t *members, const int64_t *goff,
               int64_t gcopy, double *Xs, float *Gt, float *Bd, double *Mall,
               const double *gdiag0, const int64_t *roff, uint64_t seed, int64_t stage, int K,
               double eps, int32_t *kidx, int32_t *kkv, int32_t *kel, int32_t *klvl, double *kO,
               int32_t *lvlidx, int32_t *lvl_off, int32_t *nlev, int32_t *elimflag,
               unsigned long long *stats, unsigned *status) {
    extern __shared__ double sh[];
    const int64_t u = blockIdx.x / CL;
    int rank = 0;
    if constexpr (CL > 1) rank = (int)cg::this_cluster().block_rank();
    const bool lead = rank == 0;
    const int64_t base = coff[u];
    const int c = (int)(coff[u + 1] - base);
    const int64_t r0 = roff[u];
    const int e = (int)(roff[u + 1] - r0);
    // this CTA's columns of the FP64 rows
    const int64_t cs0 = s * rank / CL, cs1 = s * (rank + 1) / CL;
    double *X = Xs + base * s;
    float *G = Gt + gcopy * rank + goff[u];
    float *B = Bd + gcopy * rank + goff[u];
    double *M = Mall + gcopy * rank + goff[u];
    double *gd = sh;
    double *md = gd + c;
    double *w = md + c;
    double *hi = w + c;
    double *lo = hi + c;
    double *red = lo + c;                       // MX_WARPS * DOT_BATCH
    const int nwords = (c + 31) / 32;
    uint32_t *mask = (uint32_t *)(red + MX_WARPS * DOT_BATCH);
    int32_t *lvl = (int32_t *)(mask + nwords);
    int32_t *lcnt = lvl + c;                    // e + 2
    int32_t *sl = lcnt + e + 2;                 // shortlist, c
    // partial dot sums from every CTA: [parity][rank][candidate] (c slots),
    // then the pairs of the tuple [parity][rank][pair] (PAIRS slots)
    double *pd = (double *)(((uintptr_t)(sl + c) + 15) & ~(uintptr_t)15);
    double *pd2 = pd + 2 * CL * c;
    __shared__ int s_T[8], s_kk, s_maxlev, s_nsl, s_fall;
    __shared__ double s_O[64], s_GT[64], s_es[SL_MAX + 8];
    __shared__ double s_gw[64], s_J[4], s_R[4];   // the warp's Jacobi
    __shared__ int s_Tt[8];                          // this step's tuple
    __shared__ double s_R2[2][64];                   // the tuple blocks' R = O X_TT
    __shared__ int s_wcnt[MX_WARPS];
    __shared__ double s_bs[8], s_bg[8];              // the partners found by warp 0
    __shared__ int s_by[8];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    // the CTAs of the cluster meet (one CTA: the block barrier)
    auto csync = [&]() {
        if constexpr (CL > 1) cg::this_cluster().sync();
        else __syncthreads();
    };

    for (int a = tid; a < c; a += MX_THREADS) {
        gd[a] = gdiag0[base + a];
        md[a] = M[(int64_t)a * c + a];
        w[a] = gd[a] > 0.0 ? __ddiv_rn(1.0, __dsqrt_rn(gd[a])) : 0.0;
        lvl[a] = 0;
    }
    for (int wi = tid; wi < nwords; wi += MX_THREADS) {
        const int rem = c - wi * 32;
        mask[wi] = rem >= 32 ? 0xffffffffu : ((1u << rem) - 1u);
    }
    for (int q = tid; q < e + 2; q += MX_THREADS) lcnt[q] = 0;
    if (tid == 0) s_maxlev = 0;
    __syncthreads();
    // initial bound eps sqrt(G_aa G_bb), rounded up
    for (int64_t q = tid; q < (int64_t)c * c; q += MX_THREADS) {
        const int a = (int)(q / c), b = (int)(q - (int64_t)a * c);
        const double v = __dmul_ru(__dmul_ru(eps, __dsqrt_ru(gd[a])), __dsqrt_ru(gd[b]));
        B[q] = __double2float_ru(v);
    }
    __syncthreads();

    int na = c;
    unsigned long long n_rescored = 0, n_fall = 0, sl_max = 0;
    for (int t = 0; t < e; ++t, --na) {
        if (tid == 0) {
            const uint64_t r = drawm(seed, (uint64_t)stage, (uint64_t)u, (uint64_t)t);
            s_T[0] = nth_set(mask, nwords, (int64_t)__umul64hi(r, (uint64_t)na));
            s_kk = K < na ? K : na;
        }
        __syncthreads();
        const int i = s_T[0], kk = s_kk;
        // score intervals from the reduced-precision row
        for (int y = tid; y < c; y += MX_THREADS) {
            double h = -1.0, l = -1.0;
            if (y != i && on(mask, y)) {
                const double sc = f64_from_bits(f64_bits(__dmul_rn((double)G[(int64_t)i * c + y], w[y])) & F64_ABS);
                const double d = __dmul_ru((double)B[(int64_t)i * c + y], __dmul_ru(w[y], 1.0 + 0x1p-40));
                h = __dadd_ru(sc, __dadd_ru(d, __dmul_ru(sc, 0x1p-50)));
                l = __dsub_rd(sc, __dadd_ru(d, __dmul_ru(sc, 0x1p-50)));
            }
            hi[y] = h;
            lo[y] = l;
        }
        __syncthreads();
        // threshold: the (kk-1)-th largest lower end (one occurrence of the
        // maximum is removed between rounds)
        double tau = -1.0;
        for (int a = 1; a < kk; ++a) {
            double mv = -1.0;
            for (int y = tid; y < c; y += MX_THREADS) mv = fmax(mv, lo[y]);
            mv = block_max(mv, red);
            tau = mv;
            if (a + 1 < kk) {
                // the lowest index holding the maximum, found by all threads
                int first = INT_MAX;
                for (int y = tid; y < c; y += MX_THREADS)
                    if (lo[y] == mv) {
                        first = y;
                        break;
                    }
                for (int o = 16; o > 0; o >>= 1) first = min(first, __shfl_xor_sync(0xffffffffu, first, o));
                __syncthreads();
                if (lane == 0) s_wcnt[wid] = first;
                __syncthreads();
                if (tid == 0) {
                    int f = s_wcnt[0];
                    for (int q = 1; q < MX_WARPS; ++q) f = min(f, s_wcnt[q]);
                    if (f < c) lo[f] = -1.0;
                }
                __syncthreads();
            }
        }
        // shortlist: candidates whose upper end reaches tau (ascending index)
        {
            int cnt = 0;
            for (int y0 = 0; y0 < c; y0 += MX_THREADS) {
                const int y = y0 + tid;
                const bool in = y < c && hi[y] >= tau && hi[y] >= 0.0;
                const unsigned bal = __ballot_sync(0xffffffffu, in);
                if (lane == 0) s_wcnt[wid] = __popc(bal);
                __syncthreads();
                int off = cnt;
                for (int q = 0; q < wid; ++q) off += s_wcnt[q];
                int tot = 0;
                for (int q = 0; q < MX_WARPS; ++q) tot += s_wcnt[q];
                if (in) sl[off + __popc(bal & ((1u << lane) - 1u))] = y;
                cnt += tot;
                __syncthreads();
            }
            if (tid == 0) {
                s_nsl = cnt;
                s_fall = cnt > SL_MAX;
            }
            __syncthreads();
        }
        const int nsl = s_nsl;
        if (s_fall) ++n_fall;
        n_rescored += (unsigned long long)nsl;
        sl_max = max(sl_max, (unsigned long long)nsl);
        // FP64 re-score: G_iy = <X_i, X_y>; partners by FP64 score
        double best_s[KM];
        int best_y[KM];
        double best_g[KM];
#pragma unroll
        for (int a = 0; a < KM; ++a) {
            best_s[a] = -1.0;
            best_y[a] = 0x7fffffff;
            best_g[a] = 0.0;
        }
        // this CTA's partial sums (its columns) of every shortlisted dot
        // product, into every CTA's buffer of this step's parity
        const int par = t & 1;
        for (int q0 = 0; q0 < nsl; q0 += DOT_BATCH) {
            const int nb = min(DOT_BATCH, nsl - q0);
            const double *xs[DOT_BATCH];
            for (int b = 0; b < DOT_BATCH; ++b) xs[b] = X + (int64_t)sl[q0 + (b < nb ? b : 0)] * s;
            const double v = slice_dots(X + (int64_t)i * s, xs, nb, cs0, cs1, red);
            if (tid < nb) {
                const int64_t slot = (int64_t)(par * CL + rank) * c + q0 + tid;
                if constexpr (CL > 1) {
                    for (int d = 0; d < CL; ++d) cg::this_cluster().map_shared_rank(pd, d)[slot] = v;
                } else {
                    pd[slot] = v;
                }
            }
        }
        csync();
        if (wid == 0) {
            // warp 0 alone: lane l scores the candidates l, l + 32, ... (the
            // FP64 dot product: the CTAs' partial sums in rank order) into its
            // own sorted top kk-1 (score descending, ties to the smaller
            // index: a candidate takes the first place it beats, the entries
            // below move down); then kk-1 rounds of a warp argmax over the
            // lanes' heads, the winner's lane dropping its head, give the
            // same list as one insertion pass over all candidates
            for (int q = lane; q < nsl; q += 32) {
                const int y = sl[q];
                double gv = pd[(int64_t)(par * CL) * c + q];
                for (int r = 1; r < CL; ++r) gv = __dadd_rn(gv, pd[(int64_t)(par * CL + r) * c + q]);
                const double sc = f64_from_bits(f64_bits(__dmul_rn(gv, w[y])) & F64_ABS);
                double cs = sc, cg = gv;
                int cy = y;
#pragma unroll
                for (int a = 0; a < KM - 1; ++a) {
                    if (a < kk - 1 && (cs > best_s[a] || (cs == best_s[a] && cy < best_y[a]))) {
                        const double ts = best_s[a], tg = best_g[a];
                        const int ty = best_y[a];
                        best_s[a] = cs;
                        best_y[a] = cy;
                        best_g[a] = cg;
                        cs = ts;
                        cy = ty;
                        cg = tg;
                    }
                }
            }
#pragma unroll
            for (int a = 0; a < KM - 1; ++a) {
                if (a >= kk - 1) break;
                double hs = best_s[0];
                int hy = best_y[0];
                for (int o = 16; o > 0; o >>= 1) {
                    const double os = __shfl_xor_sync(0xffffffffu, hs, o);
                    const int oy = __shfl_xor_sync(0xffffffffu, hy, o);
                    if (os > hs || (os == hs && oy < hy)) {
                        hs = os;
                        hy = oy;
                    }
                }
                const unsigned own = __ballot_sync(0xffffffffu, best_y[0] == hy && best_s[0] == hs);
                const int src = own ? __ffs(own) - 1 : 0;
                const double hg = __shfl_sync(0xffffffffu, best_g[0], src);
                if (lane == 0) {
                    s_bs[a] = hs;
                    s_by[a] = hy;
                    s_bg[a] = hg;
                }
                if (own && lane == src) {
#pragma unroll
                    for (int b = 0; b < KM - 2; ++b) {
                        best_s[b] = best_s[b + 1];
                        best_y[b] = best_y[b + 1];
                        best_g[b] = best_g[b + 1];
                    }
                    best_s[KM - 2] = -1.0;
                    best_y[KM - 2] = 0x7fffffff;
                    best_g[KM - 2] = 0.0;
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int a = 0; a < KM - 1; ++a)
            if (a < kk - 1) {
                best_s[a] = s_bs[a];
                best_y[a] = s_by[a];
                best_g[a] = s_bg[a];
            }
        int T[KM];
        T[0] = i;
#pragma unroll
        for (int a = 1; a < KM; ++a) {
            int y = a < kk ? best_y[a - 1] : -1;
            if (a < kk && (y < 0 || y >= c)) {
                // never taken (the shortlist holds at least kk - 1 candidates);
                // keeps every index in range: the first active index not used
                if (tid == 0) atomicOr(status, ST_NOT_CONVERGED);
                for (y = 0; y < c; ++y) {
                    bool used = !on(mask, y);
#pragma unroll
                    for (int b = 0; b < a; ++b) used |= T[b] == y;
                    if (!used) break;
                }
            }
            T[a] = y;
        }
        // the tuple in shared memory too, for the uses with run-time positions
        if (tid == 0) {
#pragma unroll
            for (int a = 0; a < KM; ++a)
                if (a < kk) s_Tt[a] = T[a];
        }
        __syncthreads();
        // FP64 k x k block: diagonal kept, (i, partner) from the re-score, the
        // partner pairs by further dot products
        if (tid == 0) {
            for (int a = 0; a < kk; ++a) s_GT[a * kk + a] = gd[s_Tt[a]];
#pragma unroll
            for (int a = 1; a < KM; ++a)
                if (a < kk) {
                    s_GT[a] = best_g[a - 1];
                    s_GT[a * kk] = best_g[a - 1];
                }
        }
        if (kk >= 3) {
            // the partners' pairs (a < b, both >= 1): partial sums as above
            int pi = 0;
            for (int a = 1; a < kk; ++a) {
                const int nb = kk - 1 - a;
                if (nb <= 0) continue;
                const double *xs[DOT_BATCH];
                for (int b = 0; b < DOT_BATCH; ++b) xs[b] = X + (int64_t)s_Tt[a + 1 + (b < nb ? b : 0)] * s;
                const double v = slice_dots(X + (int64_t)s_Tt[a] * s, xs, nb, cs0, cs1, red);
                if (tid < nb) {
                    const int64_t slot = (int64_t)(par * CL + rank) * PAIRS + pi + tid;
                    if constexpr (CL > 1) {
                        for (int d = 0; d < CL; ++d) cg::this_cluster().map_shared_rank(pd2, d)[slot] = v;
                    } else {
                        pd2[slot] = v;
                    }
                }
                pi += nb;
            }
            csync();
            if (tid == 0) {
                int q = 0;
                for (int a = 1; a < kk; ++a)
                    for (int b = a + 1; b < kk; ++b, ++q) {
                        double v = pd2[(int64_t)(par * CL) * PAIRS + q];
                        for (int r = 1; r < CL; ++r) v = __dadd_rn(v, pd2[(int64_t)(par * CL + r) * PAIRS + q]);
                        s_GT[a * kk + b] = v;
                        s_GT[b * kk + a] = v;
                    }
            }
        }
        if (wid == 0) {
            if (kk == 2) {
                if (lane == 0) {
                    double cc, ss;
                    jacobi2(s_GT[0], s_GT[1], s_GT[3], cc, ss);
                    s_O[0] = cc;
                    s_O[1] = -ss;
                    s_O[2] = ss;
                    s_O[3] = cc;
                }
            } else {
                // the k x k block diagonalised by the warp
                for (int a = lane; a < kk * kk; a += 32) s_gw[a] = s_GT[a];
                __syncwarp();
                if (!jacobi_k_warp(kk, s_gw, s_O, s_J, s_R) && lane == 0) atomicOr(status, ST_NOT_CONVERGED);
            }
        }
        __syncthreads();
        // FP64 rows X_T <- O X_T (this CTA's columns); two columns per round,
        // both loaded before either is stored
        for (int64_t r = cs0 + tid; r < cs1; r += 2 * MX_THREADS) {
            const bool two = r + MX_THREADS < cs1;
            double in0[KM], in1[KM];
#pragma unroll
            for (int a = 0; a < KM; ++a) {
                in0[a] = a < kk ? X[(int64_t)T[a] * s + r] : 0.0;
                in1[a] = a < kk && two ? X[(int64_t)T[a] * s + r + MX_THREADS] : 0.0;
            }
            double out0[KM], out1[KM];
#pragma unroll
            for (int a = 0; a < KM; ++a) {
                out0[a] = a < kk ? rot_row_u<KM>(s_O, kk, a, in0) : 0.0;
                out1[a] = a < kk && two ? rot_row_u<KM>(s_O, kk, a, in1) : 0.0;
            }
#pragma unroll
            for (int a = 0; a < KM; ++a)
                if (a < kk) {
                    X[(int64_t)T[a] * s + r] = out0[a];
                    if (two) X[(int64_t)T[a] * s + r + MX_THREADS] = out1[a];
                }
        }
        // tuple blocks: G_TT' = O G_TT O^T in FP64 (from the FP64 block),
        // M_TT' likewise, by warp 0 one entry per lane (R = O X_TT, then
        // R O^T for a <= b, mirrored); their inputs are not among the entries
        // the rows below rotate, so warp 0 joins the rows afterwards
        if (wid == 0) {
            const int nR = 2 * kk * kk;
            for (int q = lane; q < nR; q += 32) {
                const int mat = q / (kk * kk), t = q - mat * kk * kk;
                const int a = t / kk, cc = t - a * kk;
                double in[KM];
#pragma unroll
                for (int b = 0; b < KM; ++b)
                    in[b] = b < kk ? (mat ? M[(int64_t)s_Tt[b] * c + s_Tt[cc]] : s_GT[b * kk + cc]) : 0.0;
                s_R2[mat][a * kk + cc] = rot_row_u<KM>(s_O, kk, a, in);
            }
            __syncwarp();
            const int nup = kk * (kk + 1) / 2;
            for (int q = lane; q < 2 * nup; q += 32) {
                const int mat = q / nup;
                int t = q - mat * nup, a = 0;
                while (t >= kk - a) {   // (a, b), a <= b, in row order
                    t -= kk - a;
                    ++a;
                }
                const int b = a + t;
                const double *R = s_R2[mat];
                double acc = __dmul_rn(R[a * kk + kk - 1], s_O[b * kk + kk - 1]);
                for (int cc = kk - 2; cc >= 0; --cc) acc = __fma_rn(R[a * kk + cc], s_O[b * kk + cc], acc);
                const int ta = s_Tt[a], tb = s_Tt[b];
                if (mat == 0) {
                    const float f = __double2float_rn(acc);
                    const float bf = __fadd_ru(__fmul_ru(fabsf(f), 0x1p-22f), 1e-30f);
                    G[(int64_t)ta * c + tb] = f;
                    G[(int64_t)tb * c + ta] = f;
                    B[(int64_t)ta * c + tb] = bf;
                    B[(int64_t)tb * c + ta] = bf;
                    if (a == b) gd[ta] = acc;
                } else {
                    M[(int64_t)ta * c + tb] = acc;
                    M[(int64_t)tb * c + ta] = acc;
                    if (a == b) md[ta] = acc;
                }
            }
        }
        // reduced-precision Gram rows and their bound; FP64 local block M
        {
            float Of[KM * KM], Oa[KM * KM];   // O in FP32 and |O|, stride KM
#pragma unroll
            for (int a = 0; a < KM; ++a)
#pragma unroll
                for (int b = 0; b < KM; ++b) {
                    Of[a * KM + b] = a < kk && b < kk ? __double2float_rn(s_O[a * kk + b]) : 0.0f;
                    Oa[a * KM + b] = fabsf(Of[a * KM + b]);
                }
            // rounding of one rotated entry: kk products and sums in FP32 plus
            // the FP32 rounding of O itself
            const float gam = (float)(kk + 3) * 0x1p-24f;
            for (int y = tid; y < c; y += MX_THREADS) {
                bool inT = false;
#pragma unroll
                for (int a = 0; a < KM; ++a) inT |= a < kk && T[a] == y;
                if (inT || !on(mask, y)) continue;
                float gin[KM], bin[KM];
                double min_[KM];
#pragma unroll
                for (int a = 0; a < KM; ++a) {
                    gin[a] = a < kk ? G[(int64_t)T[a] * c + y] : 0.0f;
                    bin[a] = a < kk ? B[(int64_t)T[a] * c + y] : 0.0f;
                    min_[a] = a < kk ? M[(int64_t)T[a] * c + y] : 0.0;
                }
#pragma unroll
                for (int a = 0; a < KM; ++a) {
                    if (a >= kk) continue;
                    float gv = 0.0f, bv = 0.0f, mag = 0.0f;
#pragma unroll
                    for (int b = 0; b < KM; ++b) {
                        if (b >= kk) continue;
                        gv = __fmaf_rn(Of[a * KM + b], gin[b], gv);
                        bv = __fmaf_ru(Oa[a * KM + b], bin[b], bv);
                        mag = __fmaf_ru(Oa[a * KM + b], fabsf(gin[b]), mag);
                    }
                    bv = __fmaf_ru(gam, mag, bv);
                    G[(int64_t)T[a] * c + y] = gv;
                    G[(int64_t)y * c + T[a]] = gv;
                    B[(int64_t)T[a] * c + y] = bv;
                    B[(int64_t)y * c + T[a]] = bv;
                    const double mv = rot_row_u<KM>(s_O, kk, a, min_);
                    M[(int64_t)T[a] * c + y] = mv;
                    M[(int64_t)y * c + T[a]] = mv;
                }
            }
        }
        __syncthreads();
        if (tid < kk) {
            const int x = s_Tt[tid];
            const double gv = gd[x];
            w[x] = gv > 0.0 ? __ddiv_rn(1.0, __dsqrt_rn(gv)) : 0.0;
        }
        if (tid == 0) {
            int bi = 0;
            double dbest = __dsub_rn(gd[s_Tt[0]], __dmul_rn(md[s_Tt[0]], md[s_Tt[0]]));
            for (int a = 1; a < kk; ++a) {
                const int x = s_Tt[a];
                const double d = __dsub_rn(gd[x], __dmul_rn(md[x], md[x]));
                if (d <= dbest) {
                    dbest = d;
                    bi = a;
                }
            }
            const int le = s_Tt[bi];
            int L = 0;
            for (int a = 0; a < kk; ++a) L = max(L, lvl[s_Tt[a]]);
            ++L;
            for (int a = 0; a < kk; ++a) lvl[s_Tt[a]] = L;
            s_maxlev = max(s_maxlev, L);
            mask[le >> 5] &= ~(1u << (le & 31));
            if (lead) {
                const int64_t rr = r0 + t;
                for (int a = 0; a < K; ++a) kidx[rr * K + a] = a < kk ? s_Tt[a] : -1;
                for (int a = 0; a < K * K; ++a) kO[rr * K * K + a] = a < kk * kk ? s_O[a] : 0.0;
                kkv[rr] = kk;
                kel[rr] = le;
                klvl[rr] = L;
            }
        }
        __syncthreads();
    }
    // no CTA leaves while another may still write into its shared memory;
    // the records are CTA 0's to finish
    if constexpr (CL > 1) cg::this_cluster().sync();
    if (!lead) return;
    if (tid == 0) {
        atomicAdd(&stats[0], n_rescored);
        atomicAdd(&stats[1], n_fall);
        atomicAdd(&stats[2], (unsigned long long)e);
        atomicMax(&stats[3], sl_max);
    }
    const int nl = s_maxlev;
    for (int t = tid; t < e; t += MX_THREADS) {
        atomicAdd(&lcnt[klvl[r0 + t]], 1);
        elimflag[members[base + kel[r0 + t]]] = (int32_t)stage;
    }
    __syncthreads();
    if (tid == 0) {
        int acc = 0;
        for (int L = 1; L <= nl; ++L) {
            const int cnt = lcnt[L];
            lcnt[L] = acc;
            lvl_off[r0 + u + L - 1] = (int32_t)(r0 + acc);
            acc += cnt;
        }
        lvl_off[r0 + u + nl] = (int32_t)(r0 + acc);
        nlev[u] = nl;
    }
    __syncthreads();
    for (int t = tid; t < e; t += MX_THREADS) {
        const int slot = atomicAdd(&lcnt[klvl[r0 + t]], 1);
        lvlidx[r0 + slot] = (int32_t)(r0 + t);
    }
}

// k = 2 rotations found by the k-point search, in the Givens records the
// update and apply kernels use for k = 2.
__global__ void k_to_givens(const int32_t *kidx, const int32_t *kel, const int32_t *klvl,
                            const double *kO, const int32_t *lvlidx, int64_t nrot, RotRec *rec,
                            Rot2 *lvlrot) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nrot;
         t += (int64_t)gridDim.x * blockDim.x) {
        rec[t] = RotRec{kidx[2 * t], kidx[2 * t + 1], kel[t], klvl[t], kO[4 * t], kO[4 * t + 2]};
        const int64_t q = lvlidx[t];
        lvlrot[t] = Rot2{kidx[2 * q], kidx[2 * q + 1], kO[4 * q], kO[4 * q + 2]};
    }
}

}  // namespace

// G~ of every cluster by the tcgen05 kernel (the default) or by the
// warp-level mma.sync kernel (PMMF_TUNE_TC_GRAM = 1); the same chunking and
// compensated sums, so the same certified bound.
pmmf_status tc_gram(int precision, const void *XH, const void *XL, int64_t rows, int64_t sp,
                    const int64_t *coff, const std::vector<int64_t> &hcoff, const int64_t *goff,
                    float *G, unsigned *status, cudaStream_t st) {
    int64_t cmax = 0;
    for (size_t u = 0; u + 1 < hcoff.size(); ++u) cmax = std::max(cmax, hcoff[u + 1] - hcoff[u]);
    if (tuned(TUNE_TC_GRAM, cmax, 2) == 2)
        return tc_gram_tcgen05(precision, XH, XL, rows, sp, coff, hcoff, goff, G, status, st);
    const int64_t m = (int64_t)hcoff.size() - 1;
    std::vector<int32_t> tu, ta, tb;
    for (int64_t u = 0; u < m; ++u) {
        const int64_t c = hcoff[u + 1] - hcoff[u];
        const int T = (int)((c + TG - 1) / TG);
        for (int a = 0; a < T; ++a)
            for (int b = a; b < T; ++b) {
                tu.push_back((int32_t)u);
                ta.push_back(a);
                tb.push_back(b);
            }
    }
    if (tu.empty()) return PMMF_OK;
    DBuf<int32_t> dtu, dta, dtb;
    PMMF_TRY(dtu.alloc((int64_t)tu.size(), st));
    PMMF_TRY(dta.alloc((int64_t)tu.size(), st));
    PMMF_TRY(dtb.alloc((int64_t)tu.size(), st));
    PMMF_CUDA_TRY(cudaMemcpyAsync(dtu.p, tu.data(), sizeof(int32_t) * tu.size(), cudaMemcpyHostToDevice, st));
    PMMF_CUDA_TRY(cudaMemcpyAsync(dta.p, ta.data(), sizeof(int32_t) * ta.size(), cudaMemcpyHostToDevice, st));
    PMMF_CUDA_TRY(cudaMemcpyAsync(dtb.p, tb.data(), sizeof(int32_t) * tb.size(), cudaMemcpyHostToDevice, st));
    if (precision == PMMF_PREC_BF16)
        k_tc_gram<PMMF_PREC_BF16><<<(unsigned)tu.size(), 128, 0, st>>>(XH, XL, sp, coff, goff, dtu.p,
                                                                      dta.p, dtb.p, G);
    else
        k_tc_gram<PMMF_PREC_TF32><<<(unsigned)tu.size(), 128, 0, st>>>(XH, XL, sp, coff, goff, dtu.p,
                                                                      dta.p, dtb.p, G);
    return launched("tc_gram");
}

pmmf_status mixed_stage_select(const DBuf<double> &D, int64_t s, const int32_t *pos,
                               const StageClusters &cls, const std::vector<int64_t> &hcoff,
                               int64_t cmax, int precision, uint64_t seed, int64_t stage,
                               StageRotations &rot, int32_t *elimflag, unsigned long long *stats,
                               unsigned *status, cudaStream_t st) {
    const int64_t m = cls.m;
    GramBlocks gb;   // goff and the FP64 local blocks M (G is not used here)
    PMMF_TRY(gram_blocks(cls, gb, st));
    DBuf<double> X;
    DBuf<uint32_t> XH, XL;
    DBuf<double> gd0;
    DBuf<float> Gt, Bd;
    PMMF_TRY(X.alloc(s * s, st));
    // padded row length: a multiple of 8 elements keeps every row of the split
    // slab on a 16-byte boundary (the TMA row stride)
    const int64_t sp = (s + 7) / 8 * 8;
    PMMF_TRY(XH.alloc(precision == PMMF_PREC_BF16 ? s * sp / 2 : s * sp, st));
    PMMF_TRY(XL.alloc(precision == PMMF_PREC_BF16 ? s * sp / 2 : s * sp, st));
    PMMF_TRY(gd0.alloc(s, st));
    // CTAs per cluster: as many as the SMs allow (up to the portable 8), so
    // stages with few clusters still spread their FP64 work over the GPU;
    // every CTA has its own copy of G~, B and M
    int nsm = 152;
    {
        int dev = 0;
        if (cudaGetDevice(&dev) == cudaSuccess)
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    }
    int CLn = 1;
    while (CLn < 8 && m * (int64_t)CLn * 2 <= (int64_t)nsm) CLn *= 2;
    PMMF_TRY(Gt.alloc(gb.total * CLn, st));
    PMMF_TRY(Bd.alloc(gb.total * CLn, st));
    DBuf<double> Mc;
    PMMF_TRY(Mc.alloc(gb.total * CLn, st));
    if (precision == PMMF_PREC_BF16)
        k_build_slab<PMMF_PREC_BF16><<<(unsigned)s, 256, 0, st>>>(D.p, s, sp, pos, cls.members.p, X.p,
                                                                  XH.p, XL.p);
    else
        k_build_slab<PMMF_PREC_TF32><<<(unsigned)s, 256, 0, st>>>(D.p, s, sp, pos, cls.members.p, X.p,
                                                                  XH.p, XL.p);
    PMMF_TRY(launched("build_slab"));
    k_row_norms<<<grid_for(s * 32, 256), 256, 0, st>>>(X.p, s, s, gd0.p);
    PMMF_TRY(launched("row_norms"));
    k_local_block<<<(unsigned)m, 256, 0, st>>>(D.p, s, pos, cls.coff.p, cls.members.p, gb.goff.p, gb.M.p);
    PMMF_TRY(launched("local_block"));
    double flops = 0.0;
    for (int64_t u = 0; u < m; ++u) {
        const double c = (double)(hcoff[u + 1] - hcoff[u]);
        flops += c * (c + 1.0) * (double)s;
    }
    prof_begin(KF_GRAM, st);
    PMMF_TRY(tc_gram(precision, XH.p, XL.p, s, sp, cls.coff.p, hcoff, gb.goff.p, Gt.p, status, st));
    prof_end(KF_GRAM, st, (precision == PMMF_PREC_BF16 ? 4.0 : 8.0) * (double)s * (double)sp +
                              4.0 * (double)gb.total, 3.0 * flops);

    // eps, relative to |x||y| per term: the split leaves |x - hi - lo| <= u^2 |x|
    // (u = 2^-11 TF32, 2^-8 BF16), the dropped lo lo^T term is <= u^2 |x||y|,
    // so the three products miss x y by <= 3 u^2 (1 + u) |x||y|; FP32
    // accumulation of 3 KFLUSH products per chunk of KFLUSH terms (taken at
    // twice the round-to-nearest bound); the compensated sum of the N chunk
    // sums (Sum2: |hi + lo - sum| <= gamma_{N-1}^2 sum |chunk|, gamma_n =
    // n 2^-24 / (1 - n 2^-24), the chunk sums bounded by the terms' |x||y| to
    // within (1 + 2^-10)), hi + lo taken in FP64 (2^-52 with margin) and the
    // final FP32 rounding add the rest; Cauchy-Schwarz turns sum |x||y| into
    // sqrt(G_ii G_jj).  10% margin.
    const double uin = precision == PMMF_PREC_BF16 ? 0x1p-8 : 0x1p-11;
    const double nch = std::ceil((double)sp / KFLUSH) + 1.0;
    const double gam = nch * 0x1p-24 / (1.0 - nch * 0x1p-24);
    const double eps = 1.1 * (3.0 * uin * uin * (1.0 + uin) + 6.0 * (double)KFLUSH * 0x1p-24 +
                              gam * gam * (1.0 + 0x1p-10) + 0x1p-52 + 0x1p-24);
    const int K = rot.K;
    const int64_t nr = std::max<int64_t>(rot.nrot, 1);
    PMMF_TRY(rot.kidx.alloc(nr * K, st));
    PMMF_TRY(rot.kO.alloc(nr * K * K, st));
    PMMF_TRY(rot.kk.alloc(nr, st));
    PMMF_TRY(rot.kel.alloc(nr, st));
    PMMF_TRY(rot.klvl.alloc(nr, st));
    PMMF_TRY(rot.lvlidx.alloc(nr, st));
    PMMF_TRY(rot.lvl_off.alloc(rot.nrot + m + 1, st));
    PMMF_TRY(rot.nlev.zeros(m, st));
    // the copies of G~ and M for the cluster's other CTAs
    for (int r = 0; r < CLn; ++r) {
        if (r > 0 && gb.total > 0)
            PMMF_CUDA_TRY(cudaMemcpyAsync(Gt.p + r * gb.total, Gt.p, sizeof(float) * (size_t)gb.total,
                                          cudaMemcpyDeviceToDevice, st));
        if (gb.total > 0)
            PMMF_CUDA_TRY(cudaMemcpyAsync(Mc.p + r * gb.total, gb.M.p, sizeof(double) * (size_t)gb.total,
                                          cudaMemcpyDeviceToDevice, st));
    }
    size_t sh = sizeof(double) * (5 * (size_t)cmax + MX_WARPS * DOT_BATCH) +
                sizeof(uint32_t) * (size_t)((cmax + 31) / 32) +
                sizeof(int32_t) * (size_t)(3 * cmax + 4) + 16;
    sh += sizeof(double) * 2 * (size_t)CLn * ((size_t)cmax + PAIRS);   // partial dot sums
    if (sh > 200 * 1024) {
        set_error("cluster too large for the shortlist search");
        return PMMF_ERR_UNSUPPORTED;
    }
    auto launch = [&](auto kern, int cl) -> pmmf_status {
        PMMF_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh));
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(m * cl), 1, 1);
        cfg.blockDim = dim3(MX_THREADS, 1, 1);
        cfg.dynamicSmemBytes = sh;
        cfg.stream = st;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = (unsigned)cl;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = cl > 1 ? 1 : 0;
        PMMF_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, s, (const int64_t *)cls.coff.p,
                                         (const int32_t *)cls.members.p, (const int64_t *)gb.goff.p,
                                         gb.total, X.p, Gt.p, Bd.p, Mc.p, (const double *)gd0.p,
                                         (const int64_t *)rot.roff.p, seed, stage, K, eps, rot.kidx.p,
                                         rot.kk.p, rot.kel.p, rot.klvl.p, rot.kO.p, rot.lvlidx.p,
                                         rot.lvl_off.p, rot.nlev.p, elimflag, stats, status));
        return PMMF_OK;
    };
    prof_begin(KF_SELECT, st);
    if (K <= 3) {
        if (CLn == 8) PMMF_TRY(launch(k_select_mixed<8, 3>, 8));
        else if (CLn == 4) PMMF_TRY(launch(k_select_mixed<4, 3>, 4));
        else if (CLn == 2) PMMF_TRY(launch(k_select_mixed<2, 3>, 2));
        else PMMF_TRY(launch(k_select_mixed<1, 3>, 1));
    } else {
        if (CLn == 8) PMMF_TRY(launch(k_select_mixed<8, 8>, 8));
        else if (CLn == 4) PMMF_TRY(launch(k_select_mixed<4, 8>, 4));
        else if (CLn == 2) PMMF_TRY(launch(k_select_mixed<2, 8>, 2));
        else PMMF_TRY(launch(k_select_mixed<1, 8>, 1));
    }
    prof_end(KF_SELECT, st, 0.0, 0.0);
    PMMF_TRY(launched("select_mixed"));
    if (K == 2) {
        PMMF_TRY(rot.rec.alloc(nr, st));
        PMMF_TRY(rot.lvl.alloc(nr, st));
        k_to_givens<<<grid_for(rot.nrot, 256), 256, 0, st>>>(rot.kidx.p, rot.kel.p, rot.klvl.p,
                                                             rot.kO.p, rot.lvlidx.p, rot.nrot,
                                                             rot.rec.p, rot.lvl.p);
        PMMF_TRY(launched("to_givens"));
    }
    return PMMF_OK;
}

}  // namespace pmmf

using namespace pmmf;

extern "C" pmmf_status pmmf_gram_reduced(const double *X, int64_t rows, int64_t s, int precision,
                                         float *G, void *stream) {
    set_error("");
    if (!X || !G || rows < 1 || rows > 4096 || s < 1 || s > ((int64_t)1 << 24) ||
        (precision != PMMF_PREC_TF32 && precision != PMMF_PREC_BF16)) {
        set_error("pmmf_gram_reduced: NULL buffer, size out of range or not a reduced precision");
        return PMMF_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t sp = (s + 7) / 8 * 8;
    DBuf<double> D, Xs;
    DBuf<uint32_t> XH, XL;
    DBuf<int32_t> iota;
    DBuf<int64_t> coff, goff;
    DBuf<float> Gd;
    DBuf<unsigned> status;
    PMMF_TRY(D.alloc(rows * s, st));
    PMMF_TRY(Xs.alloc(rows * s, st));
    PMMF_TRY(XH.zeros(precision == PMMF_PREC_BF16 ? rows * sp / 2 : rows * sp, st));
    PMMF_TRY(XL.zeros(precision == PMMF_PREC_BF16 ? rows * sp / 2 : rows * sp, st));
    PMMF_TRY(iota.alloc(rows, st));
    PMMF_TRY(coff.alloc(2, st));
    PMMF_TRY(goff.alloc(1, st));
    PMMF_TRY(Gd.zeros(rows * rows, st));
    PMMF_TRY(status.zeros(1, st));
    std::vector<int32_t> hi((size_t)rows);
    for (int64_t q = 0; q < rows; ++q) hi[(size_t)q] = (int32_t)q;
    const int64_t hcoff_a[2] = {0, rows}, hgoff = 0;
    PMMF_CUDA_TRY(cudaMemcpyAsync(D.p, X, sizeof(double) * (size_t)(rows * s), cudaMemcpyHostToDevice, st));
    PMMF_CUDA_TRY(cudaMemcpyAsync(iota.p, hi.data(), sizeof(int32_t) * hi.size(), cudaMemcpyHostToDevice, st));
    PMMF_CUDA_TRY(cudaMemcpyAsync(coff.p, hcoff_a, sizeof(hcoff_a), cudaMemcpyHostToDevice, st));
    PMMF_CUDA_TRY(cudaMemcpyAsync(goff.p, &hgoff, sizeof(hgoff), cudaMemcpyHostToDevice, st));
    if (precision == PMMF_PREC_BF16)
        k_build_slab<PMMF_PREC_BF16><<<(unsigned)rows, 256, 0, st>>>(D.p, s, sp, iota.p, iota.p, Xs.p,
                                                                     XH.p, XL.p);
    else
        k_build_slab<PMMF_PREC_TF32><<<(unsigned)rows, 256, 0, st>>>(D.p, s, sp, iota.p, iota.p, Xs.p,
                                                                     XH.p, XL.p);
    PMMF_TRY(launched("build_slab"));
    const std::vector<int64_t> hcoff = {0, rows};
    PMMF_TRY(tc_gram(precision, XH.p, XL.p, rows, sp, coff.p, hcoff, goff.p, Gd.p, status.p, st));
    unsigned hs = 0;
    PMMF_CUDA_TRY(cudaMemcpyAsync(G, Gd.p, sizeof(float) * (size_t)(rows * rows), cudaMemcpyDeviceToHost, st));
    PMMF_CUDA_TRY(cudaMemcpyAsync(&hs, status.p, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    PMMF_CUDA_TRY(cudaStreamSynchronize(st));
    if (hs & ST_TIMEOUT) {
        set_error("pmmf_gram_reduced: a bounded wait in the tensor-core pipeline ran out");
        return PMMF_ERR_TIMEOUT;
    }
    return PMMF_OK;
}
