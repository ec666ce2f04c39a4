// dense.cu -- the stage of Algorithm 1 on a dense active matrix D (s x s,
// row-major, rows and columns in ascending global id).  Same readings and
// arithmetic as the sparse path, so the results are the same bits:
//   Gram      G^u_ab = sum over r ascending of D[x_a][r] D[x_b][r], one fma
//             chain per entry (a tiled FP64 product of the cluster's rows with
//             themselves; zero entries leave a chain unchanged, so this equals
//             the sparse merge), M^u_ab = D[x_min][x_max]
//   update    A_p = (A Q^T)^T Q^T: every row has the stage's rotations applied
//             (all clusters at once, one dependency level after another, a
//             rotation with two zero inputs skipped), a transpose, and again
//   account   residual of the eliminated coordinates, H diagonal, compaction
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>

#include "dense.cuh"

namespace pmmf {
namespace {

constexpr int GT = 64;        // Gram tile (outputs per side)
constexpr int GK = 16;        // k chunk

// Copy the caller's n x ld matrix into a contiguous n x n block, checking
// finiteness and exact symmetry; -0 is stored as +0.
__global__ void k_dense_load(const double *A, int64_t n, int64_t ld, double *D, unsigned *status) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n * n;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = q / n, j = q - i * n;
        const double v = A[i * ld + j];
        const double t = A[j * ld + i];
        if (!isfinite(v)) atomicOr(status, ST_NONFINITE);
        if (__double_as_longlong(v) != __double_as_longlong(t) && !(v == 0.0 && t == 0.0))
            atomicOr(status, ST_NOT_SYMMETRIC);
        D[q] = v == 0.0 ? 0.0 : v;
    }
}

// One CTA per 64 x 64 tile (ta <= tb) of one cluster's Gram block; 256
// threads, each a 4 x 4 patch, accumulated as fma chains over r ascending.
__global__ void __launch_bounds__(256)
k_dense_gram(const double *D, int64_t s, const int32_t *pos, const int64_t *coff,
             const int32_t *members, const int64_t *goff, const int32_t *tu, const int32_t *ta,
             const int32_t *tb, double *G, double *M) {
    __shared__ double As[GK][GT + 1], Bs[GK][GT + 1];
    __shared__ int64_t rowA[GT], rowB[GT];
    const int64_t u = tu[blockIdx.x];
    const int64_t base = coff[u];
    const int c = (int)(coff[u + 1] - base);
    const int a0 = ta[blockIdx.x] * GT, b0 = tb[blockIdx.x] * GT;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    if (tid < GT) {
        rowA[tid] = a0 + tid < c ? (int64_t)pos[members[base + a0 + tid]] : -1;
    } else if (tid < 2 * GT) {
        const int l = tid - GT;
        rowB[l] = b0 + l < c ? (int64_t)pos[members[base + b0 + l]] : -1;
    }
    __syncthreads();
    double acc[4][4];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    for (int64_t k0 = 0; k0 < s; k0 += GK) {
        // 64 rows x 16 columns of each operand: thread loads column tid % 16 of
        // rows tid / 16 + 16 q (coalesced along the row)
        const int kc = tid & 15;
        for (int q = 0; q < 4; ++q) {
            const int rr = (tid >> 4) + 16 * q;
            const int64_t k = k0 + kc;
            const int64_t ra = rowA[rr], rb = rowB[rr];
            As[kc][rr] = (ra >= 0 && k < s) ? D[ra * s + k] : 0.0;
            Bs[kc][rr] = (rb >= 0 && k < s) ? D[rb * s + k] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
            double av[4], bv[4];
            for (int i = 0; i < 4; ++i) av[i] = As[kk][ty * 4 + i];
            for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx * 4 + j];
            for (int i = 0; i < 4; ++i)
                for (int j = 0; j < 4; ++j) acc[i][j] = __fma_rn(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }
    double *Gu = G + goff[u];
    double *Mu = M + goff[u];
    for (int i = 0; i < 4; ++i) {
        const int a = a0 + ty * 4 + i;
        if (a >= c) continue;
        for (int j = 0; j < 4; ++j) {
            const int b = b0 + tx * 4 + j;
            if (b >= c) continue;
            Gu[(int64_t)a * c + b] = acc[i][j];
            Gu[(int64_t)b * c + a] = acc[i][j];
            const int64_t pa = rowA[ty * 4 + i], pb = rowB[tx * 4 + j];
            const double mv = a <= b ? D[pa * s + pb] : D[pb * s + pa];
            Mu[(int64_t)a * c + b] = mv;
            Mu[(int64_t)b * c + a] = mv;
        }
    }
}

// Stage-wide level lists: per level L (1-based) the number of rotations of
// every cluster at that level.
__global__ void k_level_count(const int64_t *roff, const int32_t *lvl_off, const int32_t *nlev,
                              int64_t m, int32_t *gcnt) {
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < m;
         u += (int64_t)gridDim.x * blockDim.x) {
        const int32_t *lo = lvl_off + roff[u] + u;
        for (int L = 1; L <= nlev[u]; ++L) atomicAdd(&gcnt[L], lo[L] - lo[L - 1]);
    }
}

// Scatter every cluster's level-grouped rotations into the stage-wide list,
// with row positions in place of cluster-local indices.
__global__ void k_level_scatter(const int64_t *coff, const int32_t *members, const int32_t *pos,
                                const int64_t *roff, const int32_t *lvl_off, const int32_t *nlev,
                                int64_t m, const int64_t *goffL, int32_t *gcur, DenseRotList L) {
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < m;
         u += (int64_t)gridDim.x * blockDim.x) {
        const int64_t base = coff[u];
        const int32_t *lo = lvl_off + roff[u] + u;
        for (int lv = 1; lv <= nlev[u]; ++lv) {
            for (int32_t q = lo[lv - 1]; q < lo[lv]; ++q) {
                const int64_t slot = goffL[lv - 1] + atomicAdd(&gcur[lv], 1);
                if (L.K == 2) {
                    const Rot2 r = L.lvlrot[q];
                    L.g2[slot] = Rot2{pos[members[base + r.li]], pos[members[base + r.lj]], r.c, r.s};
                } else {
                    const int64_t t = L.lvlidx[q];
                    const int kk = L.kkv[t];
                    L.gt[slot] = t;
                    for (int a = 0; a < L.K; ++a)
                        L.gpos[slot * L.K + a] = a < kk ? pos[members[base + L.kidx[t * L.K + a]]] : -1;
                    if (L.gO3) {
                        // k = 3: the record in slot order (no load through t)
                        L.gkk[slot] = kk;
                        for (int a = 0; a < 3; ++a)
                            for (int b = 0; b < 3; ++b)
                                L.gO3[slot * 9 + a * 3 + b] = a < kk && b < kk ? L.kO[t * 9 + a * kk + b] : 0.0;
                    }
                }
            }
        }
    }
}

// A k = 3 slot's record in registers (scalars, so it never needs an address).
struct Rec3 {
    int kk, p0, p1, p2;
    double o0, o1, o2, o3, o4, o5, o6, o7, o8;
};

__device__ __forceinline__ Rec3 rec3_load(const int32_t *gkk, const int32_t *gpos, const double *gO3,
                                          int64_t q) {
    const double *O = gO3 + q * 9;
    const int32_t *P = gpos + q * 3;
    return Rec3{gkk[q], P[0], P[1], P[2], O[0], O[1], O[2], O[3], O[4], O[5], O[6], O[7], O[8]};
}

// Row a of x_T' = O x_T for a tuple of kk <= 3 (O's row a is oa0..oa2): the
// chain of rot_row_u<3>, the last column's product, then fmas down to column 0.
__device__ __forceinline__ double rec3_row(double oa0, double oa1, double oa2, int kk, double i0,
                                           double i1, double i2) {
    if (kk == 3) return __fma_rn(oa0, i0, __fma_rn(oa1, i1, __dmul_rn(oa2, i2)));
    if (kk == 2) return __fma_rn(oa0, i0, __dmul_rn(oa1, i1));
    return __dmul_rn(oa0, i0);
}

// x_T' = O x_T on the row held in shared memory; a tuple whose inputs are all
// zero is skipped.
__device__ __forceinline__ void rec3_apply(double *row, const Rec3 x) {
    const double i0 = row[x.p0];
    const double i1 = x.kk > 1 ? row[x.p1] : 0.0;
    const double i2 = x.kk > 2 ? row[x.p2] : 0.0;
    if (!(nonzero_bits(i0) || (x.kk > 1 && nonzero_bits(i1)) || (x.kk > 2 && nonzero_bits(i2)))) return;
    const double n0 = rec3_row(x.o0, x.o1, x.o2, x.kk, i0, i1, i2);
    const double n1 = rec3_row(x.o3, x.o4, x.o5, x.kk, i0, i1, i2);
    const double n2 = rec3_row(x.o6, x.o7, x.o8, x.kk, i0, i1, i2);
    row[x.p0] = n0;
    if (x.kk > 1) row[x.p1] = n1;
    if (x.kk > 2) row[x.p2] = n2;
}

// One CTA per row: the row in shared memory, every level's rotations applied
// in turn (rotations of one level touch disjoint positions).
// KM: the largest tuple (3 for k <= 3, 8 otherwise); a k-point rotation's
// inputs and outputs are register arrays of that size.
template <int KM>
__global__ void __launch_bounds__(256)
k_dense_rows(double *D, int64_t s, const int64_t *goffL, int nlv, DenseRotList L) {
    extern __shared__ double row[];
    const int64_t r = blockIdx.x;
    double *Dr = D + r * s;
    for (int64_t q = threadIdx.x; q < s; q += blockDim.x) row[q] = Dr[q];
    __syncthreads();
    if constexpr (KM == 3) {
        if (L.K == 3 && L.gO3) {
            // k = 3 with slot-ordered records: the thread's first slot of the
            // next level (positions, tuple size, block O) is loaded into
            // registers while this level runs; the same chain per output as
            // rot_row_u<3>, so the same bits
            const int32_t *gkk = L.gkk, *gpos = L.gpos;
            const double *gO3 = L.gO3;
            if (nlv > 0) {
                int64_t b0 = goffL[0], b1 = goffL[1];
                const int64_t q0 = b0 + threadIdx.x;
                Rec3 cur{};
                if (q0 < b1) cur = rec3_load(gkk, gpos, gO3, q0);
                for (int lv = 0; lv < nlv; ++lv) {
                    const int64_t b2 = lv + 2 <= nlv ? goffL[lv + 2] : b1;
                    const int64_t qn = b1 + threadIdx.x;
                    Rec3 nxt{};
                    if (lv + 1 < nlv && qn < b2) nxt = rec3_load(gkk, gpos, gO3, qn);
                    if (b0 + threadIdx.x < b1) rec3_apply(row, cur);
                    for (int64_t q = b0 + threadIdx.x + blockDim.x; q < b1; q += blockDim.x)
                        rec3_apply(row, rec3_load(gkk, gpos, gO3, q));
                    __syncthreads();
                    cur = nxt;
                    b0 = b1;
                    b1 = b2;
                }
            }
            for (int64_t q = threadIdx.x; q < s; q += blockDim.x) Dr[q] = row[q];
            return;
        }
    }
    for (int lv = 0; lv < nlv; ++lv) {
        for (int64_t q = goffL[lv] + threadIdx.x; q < goffL[lv + 1]; q += blockDim.x) {
            if (L.K == 2) {
                const Rot2 t = L.g2[q];
                const double a = row[t.li], b = row[t.lj];
                if (nonzero_bits(a) || nonzero_bits(b)) {
                    double na, nb;
                    rot_pair(t.c, t.s, a, b, na, nb);
                    row[t.li] = na;
                    row[t.lj] = nb;
                }
            } else {
                const int64_t t = L.gt[q];
                const int kk = L.kkv[t];
                const int32_t *P = L.gpos + q * L.K;
                double in[KM];
                int pa[KM];
                bool nz = false;
#pragma unroll
                for (int a = 0; a < KM; ++a) {
                    pa[a] = a < kk ? P[a] : 0;
                    in[a] = a < kk ? row[pa[a]] : 0.0;
                    nz |= a < kk && nonzero_bits(in[a]);
                }
                if (nz) {
                    const double *O = L.kO + t * L.K * L.K;
                    double out[KM];
#pragma unroll
                    for (int a = 0; a < KM; ++a) out[a] = a < kk ? rot_row_u<KM>(O, kk, a, in) : 0.0;
#pragma unroll
                    for (int a = 0; a < KM; ++a)
                        if (a < kk) row[pa[a]] = out[a];
                }
            }
        }
        __syncthreads();
    }
    for (int64_t q = threadIdx.x; q < s; q += blockDim.x) Dr[q] = row[q];
}

__global__ void k_dense_transpose(const double *in, int64_t s, double *out) {
    __shared__ double t[32][33];
    const int64_t bx = blockIdx.x * 32, by = blockIdx.y * 32;
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
        const int64_t r = by + j, c = bx + threadIdx.x;
        if (r < s && c < s) t[j][threadIdx.x] = in[r * s + c];
    }
    __syncthreads();
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
        const int64_t r = bx + j, c = by + threadIdx.x;
        if (r < s && c < s) out[r * s + c] = t[threadIdx.x][j];
    }
}

// Per position: eliminated in this stage?
__global__ void k_dense_flags(const int32_t *act, int64_t s, const int32_t *elimflag,
                              int32_t stage, int32_t *el, int32_t *keep) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < s;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int e = elimflag[act[r]] == stage;
        el[r] = e;
        keep[r] = !e;
    }
}

// One CTA per row x: H_xx for an eliminated x, and the residual terms
// A_p[x][y]^2, y != x, with x or y eliminated (R4).
__global__ void __launch_bounds__(256)
k_dense_account(const double *D, int64_t s, const int32_t *el, const int32_t *act, double *hdiag,
                double *contrib) {
    __shared__ double red[256];
    const int64_t x = blockIdx.x;
    const double *Dx = D + x * s;
    const int ex = el[x];
    double acc = 0.0;
    for (int64_t y = threadIdx.x; y < s; y += blockDim.x) {
        if (y == x) continue;
        if (ex || el[y]) acc = __fma_rn(Dx[y], Dx[y], acc);
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] = __dadd_rn(red[threadIdx.x], red[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (red[0] != 0.0) atomicAdd(contrib, red[0]);
        if (ex) hdiag[act[x]] = Dx[x];
    }
}

__global__ void k_dense_survivors(const int32_t *act, int64_t s, const int32_t *keep,
                                  const int64_t *newpos, int32_t *sidx, int32_t *nact) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < s;
         r += (int64_t)gridDim.x * blockDim.x)
        if (keep[r]) {
            sidx[newpos[r]] = (int32_t)r;
            nact[newpos[r]] = act[r];
        }
}

__global__ void k_dense_compact(const double *D, int64_t s, const int32_t *sidx, int64_t s2,
                                double *out) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < s2 * s2;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = q / s2, j = q - i * s2;
        out[q] = D[(int64_t)sidx[i] * s + sidx[j]];
    }
}

__global__ void k_dense_core(const double *D, int64_t s, const int32_t *act, double *core,
                             double *hdiag) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < s * s;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = q / s, j = q - i * s;
        core[q] = D[q];
        if (i == j) hdiag[act[i]] = D[q];
    }
}

__global__ void k_count_nonzeros(const double *D, int64_t cnt, unsigned long long *out) {
    unsigned long long c = 0;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < cnt;
         q += (int64_t)gridDim.x * blockDim.x)
        c += nonzero_bits(D[q]) ? 1ull : 0ull;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

__global__ void k_map_cols(int32_t *col, int64_t nnz, const int32_t *act) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nnz;
         q += (int64_t)gridDim.x * blockDim.x)
        col[q] = act[col[q]];
}

// ---------------------------------------------------------------- cluster-ordered tiles

// The blocked update in the layout of the stage's clusters: the columns of
// the active block (and, after a transpose that also reorders, its rows) are
// permuted so that every cluster's coordinates are contiguous, each cluster's
// run padded to a multiple of TILE_W columns (128 bytes).  A cluster's
// rotations then act on one contiguous run of every row, so a CTA takes one
// cluster and a group of rows: it stages the cluster's level-ordered
// rotations in shared memory once, and moves RB-row tiles of the run in and
// out with TMA tensor copies (boxes of RB rows x TILE_W columns) on a
// double-buffered mbarrier pipeline, applying the rotations level by level
// (one task per (row, rotation) pair of a level).  Per row the rotations of
// a cluster are applied in level order, as in k_dense_rows, so the bits are
// the same.
constexpr int TILE_W = 16;

// padded cluster-ordered position of every active position (cp), and the
// active position of every padded position (rowof, -1 for padding; set to -1
// beforehand).  One CTA per cluster.
__global__ void k_cluster_positions(const int64_t *coff, const int32_t *members, const int32_t *pos,
                                    const int64_t *poff, int32_t *cp, int32_t *rowof) {
    const int64_t u = blockIdx.x;
    for (int64_t j = coff[u] + threadIdx.x; j < coff[u + 1]; j += blockDim.x) {
        const int32_t r = pos[members[j]];
        const int64_t a = poff[u] + (j - coff[u]);
        cp[r] = (int32_t)a;
        rowof[a] = r;
    }
}

// Dc[r][a] = D[r][rowof[a]] (0 on padding), r < s, a < S.
__global__ void k_gather_cols(const double *D, int64_t s, const int32_t *rowof, int64_t S, double *Dc) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < s * S;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = q / S, a = q - r * S;
        const int32_t j = rowof[a];
        Dc[q] = j >= 0 ? D[r * s + j] : 0.0;
    }
}

// T[a][b] = Dc[rowof[b]][a] (0 where b is padding): the transpose with the
// rows taken in cluster order; T is S x S.
__global__ void k_transpose_perm(const double *Dc, int64_t S, const int32_t *rowof, double *T) {
    __shared__ double t[32][33];
    const int64_t a0 = blockIdx.x * 32, b0 = blockIdx.y * 32;
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
        const int64_t b = b0 + j, a = a0 + threadIdx.x;
        double v = 0.0;
        if (b < S && a < S) {
            const int32_t r = rowof[b];
            if (r >= 0) v = Dc[(int64_t)r * S + a];
        }
        t[j][threadIdx.x] = v;
    }
    __syncthreads();
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
        const int64_t a = a0 + j, b = b0 + threadIdx.x;
        if (a < S && b < S) T[a * S + b] = t[threadIdx.x][j];
    }
}

struct TileRot {
    int K;
    const int64_t *roff;
    const int32_t *lvl_off, *nlev;
    const Rot2 *lvlrot;
    const int32_t *lvlidx, *kkv, *kidx;
    const double *kO;
};

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Bounded wait for phase `parity` of an mbarrier; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    const uint32_t a = smem_addr(bar);
    for (int it = 0; it < (1 << 24); ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Element (row i, column c) of a tile: boxes of RB x TILE_W, box-major.
template <int RB>
__device__ __forceinline__ double &tile_at(double *buf, int i, int c) {
    return buf[(c / TILE_W) * (RB * TILE_W) + i * TILE_W + (c % TILE_W)];
}

// One CTA per (cluster, row group); see above.  rows: the rows of the tensor
// (s for the column-permuted block, S for the transposed one).
constexpr int TILE_WARPS = 8;   // 256 threads

template <int RB>
__global__ void __launch_bounds__(TILE_WARPS * 32)
k_dense_tiles(const __grid_constant__ CUtensorMap tmap, int64_t rows, const int64_t *coff,
              const int64_t *poff, TileRot R, int64_t rows_per_group, unsigned *status) {
    extern __shared__ __align__(1024) unsigned char tsm[];
    const int64_t u = blockIdx.x;
    const int tid = threadIdx.x;
    const int64_t r_begin = blockIdx.y * rows_per_group;
    const int64_t r_end = min(rows, r_begin + rows_per_group);
    if (r_begin >= r_end) return;
    const int nblk = (int)((r_end - r_begin + RB - 1) / RB);
    const int nch = (int)((poff[u + 1] - poff[u]) / TILE_W);
    const int64_t x0 = poff[u];
    const int64_t rr0 = R.roff[u];
    const int32_t *lo = R.lvl_off + rr0 + u;
    const int nl = R.nlev[u];
    const int64_t q0 = lo[0];
    const int ne = (int)(lo[nl] - q0);
    const int K = R.K;
    // layout: two tile buffers, the level offsets, the rotations, two mbarriers
    const size_t tbytes = (size_t)nch * RB * TILE_W * sizeof(double);
    double *buf0 = (double *)tsm;
    double *buf1 = (double *)(tsm + tbytes);
    int32_t *lvo = (int32_t *)(tsm + 2 * tbytes);
    unsigned char *rt = (unsigned char *)(lvo + ((nl + 2) & ~1));
    // k = 2: Rot2 per slot; k >= 3: kk, K local indices and K*K block per slot
    Rot2 *r2 = (Rot2 *)rt;
    // bytes per k-point slot: kk and the K indices, rounded up to 8, then
    // the K*K block (so every slot's doubles are 8-aligned)
    const int kstride = ((4 + 4 * K + 7) & ~7) + 8 * K * K;
    uint64_t *bar = (uint64_t *)(rt + (size_t)ne * (K <= 2 ? sizeof(Rot2) : (size_t)kstride));
    for (int L = tid; L <= nl; L += blockDim.x) lvo[L] = (int32_t)(lo[L] - q0);
    if (K <= 2) {
        for (int q = tid; q < ne; q += blockDim.x) r2[q] = R.lvlrot[q0 + q];
    } else {
        for (int q = tid; q < ne; q += blockDim.x) {
            const int64_t t = R.lvlidx[q0 + q];
            unsigned char *d = rt + (size_t)q * kstride;
            *(int32_t *)d = R.kkv[t];
            for (int a = 0; a < K; ++a) ((int32_t *)(d + 4))[a] = R.kidx[t * K + a];
            double *O = (double *)(d + ((4 + 4 * K + 7) & ~7));
            for (int a = 0; a < K * K; ++a) O[a] = R.kO[t * K * K + a];
        }
    }
    if (tid == 0) {
        for (int i = 0; i < 2; ++i)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar[i])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const uint32_t txb = (uint32_t)tbytes;
    auto issue_load = [&](int b, double *dst, uint64_t *mb) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(mb)),
                     "r"(txb) : "memory");
        const int y = (int)(r_begin + (int64_t)b * RB);
        for (int k = 0; k < nch; ++k) {
            const int x = (int)(x0 + (int64_t)k * TILE_W);
            asm volatile(
                "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes "
                "[%0], [%1, {%2, %3}], [%4];" ::"r"(smem_addr(dst + (size_t)k * RB * TILE_W)),
                "l"(&tmap), "r"(x), "r"(y), "r"(smem_addr(mb))
                : "memory");
        }
    };
    auto issue_store = [&](int b, double *src) {
        const int y = (int)(r_begin + (int64_t)b * RB);
        for (int k = 0; k < nch; ++k) {
            const int x = (int)(x0 + (int64_t)k * TILE_W);
            asm volatile(
                "cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(&tmap),
                "r"(x), "r"(y), "r"(smem_addr(src + (size_t)k * RB * TILE_W))
                : "memory");
        }
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    };
    if (tid == 0) issue_load(0, buf0, &bar[0]);
    bool ok = true;
    for (int b = 0; b < nblk && ok; ++b) {
        double *cur = (b & 1) ? buf1 : buf0;
        if (tid == 0 && b + 1 < nblk) {
            // the other buffer's last store has read its data
            asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
            issue_load(b + 1, (b & 1) ? buf0 : buf1, &bar[(b + 1) & 1]);
        }
        if (!mbar_wait(&bar[b & 1], (uint32_t)((b >> 1) & 1))) {
            if (tid == 0) atomicOr(status, ST_TIMEOUT);
            ok = false;
        }
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                // the loads of blocks b and b + 1 may still be in flight: give
                // them time to land (bounded) before the CTA's shared memory
                // is released
                mbar_wait(&bar[b & 1], (uint32_t)((b >> 1) & 1));
                if (b + 1 < nblk) mbar_wait(&bar[(b + 1) & 1], (uint32_t)(((b + 1) >> 1) & 1));
            }
            ok = false;
            break;
        }
        const int64_t left = r_end - (r_begin + (int64_t)b * RB);
        const int nrows = (int)(left < RB ? left : RB);
        // warp w owns the tile's rows w, w + 8, ...: the rows are independent
        // and the rotations of one level are disjoint, so a level ends with a
        // warp barrier, not a block barrier
        const int lane = tid & 31, wid = tid >> 5;
        const int rw = nrows > wid ? (nrows - wid + TILE_WARPS - 1) / TILE_WARPS : 0;
        for (int L = 0; L < nl; ++L) {
            const int s0 = lvo[L], ns = lvo[L + 1] - s0;
            const int tasks = rw * ns;
            for (int q = lane; q < tasks; q += 32) {
                const int ir = q / ns, slot = s0 + (q - ir * ns);
                const int i = wid + ir * TILE_WARPS;
                if (K <= 2) {
                    const Rot2 t = r2[slot];
                    double &ra = tile_at<RB>(cur, i, t.li);
                    double &rb = tile_at<RB>(cur, i, t.lj);
                    const double a = ra, bb = rb;
                    if (nonzero_bits(a) || nonzero_bits(bb)) {
                        double na, nb;
                        rot_pair(t.c, t.s, a, bb, na, nb);
                        ra = na;
                        rb = nb;
                    }
                } else {
                    const unsigned char *d = rt + (size_t)slot * kstride;
                    const int kk = *(const int32_t *)d;
                    const int32_t *P = (const int32_t *)(d + 4);
                    const double *O = (const double *)(d + ((4 + 4 * K + 7) & ~7));
                    double in[8];
                    bool nz = false;
                    for (int a = 0; a < kk; ++a) {
                        in[a] = tile_at<RB>(cur, i, P[a]);
                        nz |= nonzero_bits(in[a]);
                    }
                    if (nz) {
                        double out[8];
                        for (int a = 0; a < kk; ++a) out[a] = rot_row(O, kk, a, in);
                        for (int a = 0; a < kk; ++a) tile_at<RB>(cur, i, P[a]) = out[a];
                    }
                }
            }
            __syncwarp();
        }
        // the threads' writes before the TMA store reads the tile
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) issue_store(b, cur);
    }
    if (tid == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    __syncthreads();
}

// Per padded position: eliminated in this stage (from the flags of the active
// positions; 0 on padding), and its global id (0 on padding).
__global__ void k_pad_flags(const int32_t *cp, const int32_t *act, int64_t s, const int32_t *el,
                            int32_t *elp, int32_t *actp) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < s;
         r += (int64_t)gridDim.x * blockDim.x) {
        elp[cp[r]] = el[r];
        actp[cp[r]] = act[r];
    }
}

// Survivors in active order: their padded positions and global ids.
__global__ void k_pad_survivors(const int32_t *act, int64_t s, const int32_t *keep,
                                const int64_t *newpos, const int32_t *cp, int32_t *sidx,
                                int32_t *nact) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < s;
         r += (int64_t)gridDim.x * blockDim.x)
        if (keep[r]) {
            sidx[newpos[r]] = cp[r];
            nact[newpos[r]] = act[r];
        }
}

}  // namespace

pmmf_status dense_load(const double *A, int64_t n, int64_t ld, DBuf<double> &D, unsigned *status,
                       cudaStream_t st) {
    PMMF_TRY(D.alloc(n * n, st));
    k_dense_load<<<grid_for(n * n, 256), 256, 0, st>>>(A, n, ld, D.p, status);
    return launched("dense_load");
}

pmmf_status dense_gram(const DBuf<double> &D, int64_t s, const int32_t *pos,
                       const StageClusters &cls, const std::vector<int64_t> &hcoff,
                       GramBlocks &gb, cudaStream_t st) {
    std::vector<int32_t> tu, ta, tb;
    for (int64_t u = 0; u < cls.m; ++u) {
        const int64_t c = hcoff[u + 1] - hcoff[u];
        const int T = (int)((c + GT - 1) / GT);
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
    double flops = 0.0;
    for (int64_t u = 0; u < cls.m; ++u) {
        const double c = (double)(hcoff[u + 1] - hcoff[u]);
        flops += c * (c + 1.0) * (double)s;   // upper triangle, 2 flops per term
    }
    prof_begin(KF_GRAM, st);
    k_dense_gram<<<(unsigned)tu.size(), 256, 0, st>>>(D.p, s, pos, cls.coff.p, cls.members.p,
                                                      gb.goff.p, dtu.p, dta.p, dtb.p, gb.G.p, gb.M.p);
    prof_end(KF_GRAM, st, 8.0 * (double)s * (double)s + 16.0 * (double)gb.total, flops);
    PMMF_TRY(launched("dense_gram"));
    // the tile lists are freed stream-ordered after the launch
    return PMMF_OK;
}

pmmf_status dense_levels(const StageClusters &cls, const StageRotations &rot, const int32_t *pos,
                         int nlv, DenseLevels &out, cudaStream_t st) {
    const int64_t m = cls.m, nr = std::max<int64_t>(rot.nrot, 1);
    out.nlv = nlv;
    DBuf<int32_t> gcnt, gcur;
    PMMF_TRY(gcnt.zeros(nlv + 2, st));
    PMMF_TRY(gcur.zeros(nlv + 2, st));
    PMMF_TRY(out.goffL.alloc(nlv + 2, st));
    k_level_count<<<grid_for(m, 128), 128, 0, st>>>(rot.roff.p, rot.lvl_off.p, rot.nlev.p, m, gcnt.p);
    PMMF_TRY(launched("level_count"));
    // goffL[L - 1] = rotations at levels < L
    PMMF_TRY(scan_i32_to_i64(gcnt.p + 1, out.goffL.p, nlv, st));
    out.L.K = rot.K;
    out.L.lvlrot = rot.lvl.p;
    out.L.lvlidx = rot.lvlidx.p;
    out.L.kkv = rot.kk.p;
    out.L.kidx = rot.kidx.p;
    out.L.kO = rot.kO.p;
    if (rot.K == 2) {
        PMMF_TRY(out.g2.alloc(nr, st));
        out.L.g2 = out.g2.p;
    } else {
        PMMF_TRY(out.gt.alloc(nr, st));
        PMMF_TRY(out.gpos.alloc(nr * rot.K, st));
        out.L.gt = out.gt.p;
        out.L.gpos = out.gpos.p;
        if (rot.K == 3) {
            PMMF_TRY(out.gkk.alloc(nr, st));
            PMMF_TRY(out.gO3.alloc(nr * 9, st));
            out.L.gkk = out.gkk.p;
            out.L.gO3 = out.gO3.p;
        }
    }
    k_level_scatter<<<grid_for(m, 128), 128, 0, st>>>(cls.coff.p, cls.members.p, pos, rot.roff.p,
                                                      rot.lvl_off.p, rot.nlev.p, m, out.goffL.p,
                                                      gcur.p, out.L);
    return launched("level_scatter");
}

pmmf_status dense_update(DBuf<double> &D, int64_t s, const DenseLevels &lv, const int32_t *act,
                         const int32_t *elimflag, int64_t stage, double *hdiag, double *contrib,
                         DBuf<double> &Dnext, DBuf<int32_t> &nact, int64_t &s2, cudaStream_t st) {
    const size_t sh = sizeof(double) * (size_t)s;
    if (sh > 220 * 1024) {
        set_error("dense update: rows too long for shared memory");
        return PMMF_ERR_UNSUPPORTED;
    }
    auto rows_kern = lv.L.K <= 3 ? k_dense_rows<3> : k_dense_rows<8>;
    PMMF_CUDA_TRY(allow_smem(rows_kern, sh));
    DBuf<double> T;
    PMMF_TRY(T.alloc(s * s, st));
    // every pass reads and writes the s x s block once
    prof_begin(KF_ROWS, st);
    rows_kern<<<(unsigned)s, 256, sh, st>>>(D.p, s, lv.goffL.p, lv.nlv, lv.L);
    prof_end(KF_ROWS, st, 16.0 * (double)s * (double)s, 0.0);
    PMMF_TRY(launched("dense_rows"));
    dim3 tg((unsigned)((s + 31) / 32), (unsigned)((s + 31) / 32)), tb(32, 8);
    k_dense_transpose<<<tg, tb, 0, st>>>(D.p, s, T.p);
    PMMF_TRY(launched("dense_transpose"));
    prof_begin(KF_ROWS, st);
    rows_kern<<<(unsigned)s, 256, sh, st>>>(T.p, s, lv.goffL.p, lv.nlv, lv.L);
    prof_end(KF_ROWS, st, 16.0 * (double)s * (double)s, 0.0);
    PMMF_TRY(launched("dense_rows"));
    DBuf<int32_t> el, keep, sidx;
    DBuf<int64_t> newpos;
    PMMF_TRY(el.alloc(s, st));
    PMMF_TRY(keep.alloc(s, st));
    PMMF_TRY(newpos.alloc(s + 1, st));
    k_dense_flags<<<grid_for(s, 256), 256, 0, st>>>(act, s, elimflag, (int32_t)stage, el.p, keep.p);
    PMMF_TRY(launched("dense_flags"));
    k_dense_account<<<(unsigned)s, 256, 0, st>>>(T.p, s, el.p, act, hdiag, contrib);
    PMMF_TRY(launched("dense_account"));
    PMMF_TRY(scan_i32_to_i64(keep.p, newpos.p, s, st));
    PMMF_CUDA_TRY(cudaMemcpyAsync(&s2, newpos.p + s, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    PMMF_CUDA_TRY(cudaStreamSynchronize(st));
    PMMF_TRY(sidx.alloc(std::max<int64_t>(s2, 1), st));
    PMMF_TRY(nact.alloc(std::max<int64_t>(s2, 1), st));
    k_dense_survivors<<<grid_for(s, 256), 256, 0, st>>>(act, s, keep.p, newpos.p, sidx.p, nact.p);
    PMMF_TRY(launched("dense_survivors"));
    PMMF_TRY(Dnext.alloc(std::max<int64_t>(s2 * s2, 1), st));
    k_dense_compact<<<grid_for(s2 * s2, 256), 256, 0, st>>>(T.p, s, sidx.p, s2, Dnext.p);
    return launched("dense_compact");
}

// cuTensorMapEncodeTiled from the driver (looked up once).
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
        else
            cudaGetLastError();
    }
    return fn;
}

namespace {

// A rows x cols FP64 row-major block as a tensor map with RB x TILE_W boxes.
pmmf_status tile_map(CUtensorMap *m, double *base, int64_t rows, int64_t cols, int rb) {
    auto fn = encode_fn();
    if (!fn) {
        set_error("cuTensorMapEncodeTiled is not available");
        return PMMF_ERR_CUDA;
    }
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols * sizeof(double)};
    cuuint32_t box[2] = {(cuuint32_t)TILE_W, (cuuint32_t)rb};
    cuuint32_t es[2] = {1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, base, dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed");
        return PMMF_ERR_CUDA;
    }
    return PMMF_OK;
}

template <int RB>
pmmf_status launch_tiles(const CUtensorMap &map, int64_t rows, int64_t m, const int64_t *coff,
                         const int64_t *poff, const TileRot &R, size_t smem, unsigned *status,
                         cudaStream_t st) {
    int dev = 0, nsm = 152;
    if (cudaGetDevice(&dev) == cudaSuccess)
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int64_t groups = std::max<int64_t>(1, (2 * (int64_t)nsm + m - 1) / m);
    int64_t rpg = (rows + groups - 1) / groups;
    rpg = (rpg + RB - 1) / RB * RB;
    const int64_t gy = (rows + rpg - 1) / rpg;
    PMMF_CUDA_TRY(cudaFuncSetAttribute(k_dense_tiles<RB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem));
    k_dense_tiles<RB><<<dim3((unsigned)m, (unsigned)gy), TILE_WARPS * 32, smem, st>>>(map, rows, coff, poff, R, rpg,
                                                                       status);
    return launched("dense_tiles");
}

}  // namespace

pmmf_status dense_update_tiles(DBuf<double> &D, int64_t s, const StageClusters &cls,
                               const std::vector<int64_t> &hc, const StageRotations &rot,
                               const int32_t *pos, const int32_t *act, const int32_t *elimflag,
                               int64_t stage, double *hdiag, double *contrib, DBuf<double> &Dnext,
                               DBuf<int32_t> &nact, int64_t &s2, unsigned *status, cudaStream_t st,
                               bool *used) {
    *used = false;
    const int64_t m = cls.m;
    const int K = rot.K;
    std::vector<int64_t> poff((size_t)m + 1, 0), roff;
    std::vector<int32_t> nlev;
    roff.resize((size_t)m + 1);
    nlev.resize((size_t)m);
    PMMF_CUDA_TRY(cudaMemcpyAsync(roff.data(), rot.roff.p, sizeof(int64_t) * (size_t)(m + 1), cudaMemcpyDeviceToHost, st));
    PMMF_CUDA_TRY(cudaMemcpyAsync(nlev.data(), rot.nlev.p, sizeof(int32_t) * (size_t)m, cudaMemcpyDeviceToHost, st));
    PMMF_CUDA_TRY(cudaStreamSynchronize(st));
    int64_t cpad_max = 0, e_max = 0;
    int nl_max = 0;
    for (int64_t u = 0; u < m; ++u) {
        const int64_t c = hc[u + 1] - hc[u];
        const int64_t cp = (c + TILE_W - 1) / TILE_W * TILE_W;
        poff[u + 1] = poff[u] + cp;
        cpad_max = std::max(cpad_max, cp);
        e_max = std::max(e_max, roff[u + 1] - roff[u]);
        nl_max = std::max(nl_max, nlev[u]);
    }
    const int64_t S = poff[m];
    const size_t kstride = (size_t)((4 + 4 * K + 7) & ~7) + 8 * (size_t)K * K;
    const size_t rbytes = (size_t)e_max * (K <= 2 ? sizeof(Rot2) : kstride);
    const size_t fixed = 4 * (size_t)((nl_max + 2) & ~1) + rbytes + 64;
    int rb = 0;
    for (int cand : {16, 8, 4}) {
        const size_t need = 2 * (size_t)cpad_max * cand * sizeof(double) + fixed;
        if (need <= 224 * 1024) {
            rb = cand;
            break;
        }
    }
    if (rb == 0 || S >= INT32_MAX || s >= INT32_MAX || !encode_fn()) return PMMF_OK;   // caller falls back
    const size_t smem = 2 * (size_t)cpad_max * rb * sizeof(double) + fixed;
    DBuf<int64_t> dpoff;
    PMMF_TRY(dpoff.alloc(m + 1, st));
    PMMF_CUDA_TRY(cudaMemcpyAsync(dpoff.p, poff.data(), sizeof(int64_t) * poff.size(), cudaMemcpyHostToDevice, st));
    DBuf<int32_t> cp, rowof;
    PMMF_TRY(cp.alloc(std::max<int64_t>(s, 1), st));
    PMMF_TRY(rowof.alloc(S, st));
    PMMF_CUDA_TRY(cudaMemsetAsync(rowof.p, 0xFF, sizeof(int32_t) * (size_t)S, st));
    k_cluster_positions<<<(unsigned)m, 128, 0, st>>>(cls.coff.p, cls.members.p, pos, dpoff.p, cp.p,
                                                     rowof.p);
    PMMF_TRY(launched("cluster_positions"));
    // the columns in cluster order
    DBuf<double> Dc;
    PMMF_TRY(Dc.alloc(s * S, st));
    k_gather_cols<<<grid_for(s * S, 256), 256, 0, st>>>(D.p, s, rowof.p, S, Dc.p);
    PMMF_TRY(launched("gather_cols"));
    TileRot R;
    R.K = K;
    R.roff = rot.roff.p;
    R.lvl_off = rot.lvl_off.p;
    R.nlev = rot.nlev.p;
    R.lvlrot = rot.lvl.p;
    R.lvlidx = rot.lvlidx.p;
    R.kkv = rot.kk.p;
    R.kidx = rot.kidx.p;
    R.kO = rot.kO.p;
    auto tiles = [&](const CUtensorMap &map, int64_t rows) -> pmmf_status {
        if (rb == 16) return launch_tiles<16>(map, rows, m, cls.coff.p, dpoff.p, R, smem, status, st);
        if (rb == 8) return launch_tiles<8>(map, rows, m, cls.coff.p, dpoff.p, R, smem, status, st);
        return launch_tiles<4>(map, rows, m, cls.coff.p, dpoff.p, R, smem, status, st);
    };
    CUtensorMap m1, m2;
    PMMF_TRY(tile_map(&m1, Dc.p, s, S, rb));
    // pass 1: every row of A Q^T
    prof_begin(KF_ROWS, st);
    PMMF_TRY(tiles(m1, s));
    prof_end(KF_ROWS, st, 16.0 * (double)s * (double)S, 0.0);
    DBuf<double> T;
    PMMF_TRY(T.alloc(S * S, st));
    dim3 tg((unsigned)((S + 31) / 32), (unsigned)((S + 31) / 32)), tb(32, 8);
    k_transpose_perm<<<tg, tb, 0, st>>>(Dc.p, S, rowof.p, T.p);
    PMMF_TRY(launched("transpose_perm"));
    Dc.reset();
    PMMF_TRY(tile_map(&m2, T.p, S, S, rb));
    // pass 2: every row of the transpose
    prof_begin(KF_ROWS, st);
    PMMF_TRY(tiles(m2, S));
    prof_end(KF_ROWS, st, 16.0 * (double)S * (double)S, 0.0);
    // accounting on the padded layout, survivors in active order
    DBuf<int32_t> el, keep, elp, actp, sidx;
    DBuf<int64_t> newpos;
    PMMF_TRY(el.alloc(s, st));
    PMMF_TRY(keep.alloc(s, st));
    PMMF_TRY(elp.zeros(S, st));
    PMMF_TRY(actp.zeros(S, st));
    PMMF_TRY(newpos.alloc(s + 1, st));
    k_dense_flags<<<grid_for(s, 256), 256, 0, st>>>(act, s, elimflag, (int32_t)stage, el.p, keep.p);
    PMMF_TRY(launched("dense_flags"));
    k_pad_flags<<<grid_for(s, 256), 256, 0, st>>>(cp.p, act, s, el.p, elp.p, actp.p);
    PMMF_TRY(launched("pad_flags"));
    k_dense_account<<<(unsigned)S, 256, 0, st>>>(T.p, S, elp.p, actp.p, hdiag, contrib);
    PMMF_TRY(launched("dense_account"));
    PMMF_TRY(scan_i32_to_i64(keep.p, newpos.p, s, st));
    PMMF_CUDA_TRY(cudaMemcpyAsync(&s2, newpos.p + s, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    PMMF_CUDA_TRY(cudaStreamSynchronize(st));
    PMMF_TRY(sidx.alloc(std::max<int64_t>(s2, 1), st));
    PMMF_TRY(nact.alloc(std::max<int64_t>(s2, 1), st));
    k_pad_survivors<<<grid_for(s, 256), 256, 0, st>>>(act, s, keep.p, newpos.p, cp.p, sidx.p, nact.p);
    PMMF_TRY(launched("pad_survivors"));
    PMMF_TRY(Dnext.alloc(std::max<int64_t>(s2 * s2, 1), st));
    k_dense_compact<<<grid_for(s2 * s2, 256), 256, 0, st>>>(T.p, S, sidx.p, s2, Dnext.p);
    PMMF_TRY(launched("dense_compact"));
    *used = true;
    return PMMF_OK;
}

pmmf_status dense_nonzeros(const double *D, int64_t cnt, int64_t *out, cudaStream_t st) {
    DBuf<unsigned long long> c;
    PMMF_TRY(c.zeros(1, st));
    k_count_nonzeros<<<grid_for(cnt, 256), 256, 0, st>>>(D, cnt, c.p);
    PMMF_TRY(launched("count_nonzeros"));
    unsigned long long h = 0;
    PMMF_CUDA_TRY(cudaMemcpyAsync(&h, c.p, sizeof(h), cudaMemcpyDeviceToHost, st));
    PMMF_CUDA_TRY(cudaStreamSynchronize(st));
    *out = (int64_t)h;
    return PMMF_OK;
}

pmmf_status dense_core(const double *D, int64_t s, const int32_t *act, double *core, double *hdiag,
                       cudaStream_t st) {
    if (s <= 0) return PMMF_OK;
    k_dense_core<<<grid_for(s * s, 256), 256, 0, st>>>(D, s, act, core, hdiag);
    return launched("dense_core");
}

pmmf_status dense_record(const double *D, int64_t s, const int32_t *act, Csr &out,
                         cudaStream_t st) {
    PMMF_TRY(dense_to_csr(D, s, s, out.rowptr, out.col, out.val, st));
    out.rows = s;
    PMMF_CUDA_TRY(cudaMemcpyAsync(&out.nnz, out.rowptr.p + s, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    PMMF_CUDA_TRY(cudaStreamSynchronize(st));
    if (out.nnz > 0) {
        k_map_cols<<<grid_for(out.nnz, 256), 256, 0, st>>>(out.col.p, out.nnz, act);
        PMMF_TRY(launched("map_cols"));
    }
    return PMMF_OK;
}

}  // namespace pmmf
