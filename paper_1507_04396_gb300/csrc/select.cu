// select.cu -- per-cluster Gram matrices and the randomized greedy rotation
// search of Algorithm 2 (k = 2, Givens rotations), one CTA per cluster.
//
// Arithmetic follows a fixed operation order so that the rotations equal, bit
// for bit, those of a sequential FP64 reference using the same readings:
//   Gram      G_ab = sum over r ascending of A[x_a][r] * A[x_b][r], one fma
//             chain per entry (Sec. 2: G = A^T A for the cluster's columns,
//             using the rows of the stored matrix).
//   M         the cluster's diagonal block, symmetric: M_ab = A[min][max].
//   pick      i = the r * |I| / 2^64-th active index, r from splitmix64.
//   partner   j = argmax_{active j != i} |G_ij| * w_j, w_j = 1 / sqrt(G_jj)
//             (0 if G_jj <= 0), ties to the smaller index (Sec. 2.2).
//   angle     smaller-angle Jacobi rotation of [[G_ii, G_ij], [G_ij, G_jj]].
//   update    G <- q G q^T and M <- q M q^T, rows recomputed then mirrored.
//   eliminate i if G_ii - M_ii^2 < G_jj - M_jj^2, else j (Alg. 2).
//
// On GB300 a dependent FP64 operation costs ~64 cycles and a divide or square
// root ~600, so the per-step critical path is arranged around FP64 latency:
// scores are compared through their (order-preserving) bit patterns, and the
// angle takes two square roots and two independent divides.
#include <cooperative_groups.h>

#include <vector>

#include "common.cuh"
#include "rotmath.cuh"
#include "stage.cuh"

namespace pmmf {

namespace {

__device__ __forceinline__ uint64_t mix1(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t draw(uint64_t seed, uint64_t p, uint64_t u, uint64_t t) {
    uint64_t h = mix1(seed);
    h = mix1(h ^ p);
    h = mix1(h ^ u);
    return mix1(h ^ t);
}

// New 2x2 block of q X q^T for symmetric X with X_ii = a, X_ij = X_ji = b,
// X_jj = d: row step R = q X_TT, then column step R q^T (upper half, mirrored).
__device__ __forceinline__ void rot_block(double c, double s, double a, double b, double d,
                                          double &na, double &nb, double &nd) {
    double rii, rij, rji, rjj;
    rot_pair(c, s, a, b, rii, rji);   // column i of X_TT
    rot_pair(c, s, b, d, rij, rjj);   // column j of X_TT
    na = __fma_rn(rii, c, __dmul_rn(rij, -s));
    nb = __fma_rn(rii, s, __dmul_rn(rij, c));
    nd = __fma_rn(rji, s, __dmul_rn(rjj, c));
}

__global__ void k_square_sizes(const int64_t *coff, int64_t m, int64_t *sz) {
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < m;
         u += (int64_t)gridDim.x * blockDim.x) {
        int64_t c = coff[u + 1] - coff[u];
        sz[u] = c * c;
    }
}

// Transpose of the active matrix (rows by position, entries = (row's global
// id, value)): count, scan, scatter.  The order inside a transposed row is
// arbitrary; the Gram kernel below does not depend on it.
__global__ void k_tcount(const int64_t *rp, const int32_t *ci, int64_t s, const int32_t *pos,
                         int64_t *tcnt) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < rp[s];
         q += (int64_t)gridDim.x * blockDim.x)
        atomicAdd((unsigned long long *)&tcnt[pos[ci[q]]], 1ull);
}

// Each transposed entry keeps its row's cluster and local index, packed as
// (cluster << 32) | local index, so the Gram kernel tests and places it with
// one load instead of a dependent id -> cluster, local index chain.
__global__ void k_tscatter(const int64_t *rp, const int32_t *ci, const double *v, int64_t s,
                           const int32_t *pos, const int32_t *act, const int32_t *cl,
                           const int32_t *loc, int64_t *tcur, int64_t *tul, double *tv) {
    const int lane = threadIdx.x & 31;
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = w; r < s; r += nw) {
        const int32_t g = act[r];
        const int64_t ul = ((int64_t)cl[g] << 32) | (int64_t)(uint32_t)loc[g];
        for (int64_t q = rp[r] + lane; q < rp[r + 1]; q += 32) {
            const int64_t slot = (int64_t)atomicAdd((unsigned long long *)&tcur[pos[ci[q]]], 1ull);
            tul[slot] = ul;
            tv[slot] = v[q];
        }
    }
}

// Gram rows by the row-by-row (Gustavson) product, one warp per Gram row a of
// cluster u: row x_a's entries r are taken in ascending order and, for each,
// the stored entries of column r in cluster u update a dense accumulator, so
// every G_ab is one fma chain over the common columns in ascending order (the
// same bits as the merge in k_gram; the product is commutative, so G_ab and
// G_ba agree).  Whole rows are written, coalesced.  M row a: A[x_a][x_b] for
// b >= a from row x_a, A[x_b][x_a] for b < a from column x_a.
__global__ void k_gram_rows(const int64_t *rp, const int32_t *ci, const double *v,
                            const int64_t *trp, const int64_t *tul, const double *tv,
                            const int32_t *pos, const int32_t *cl, const int32_t *loc,
                            const int64_t *coff, const int32_t *members, int64_t s, int64_t cmax,
                            const int64_t *goff, double *G, double *M) {
    extern __shared__ double gacc[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    double *acc = gacc + (int64_t)wib * cmax;
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t j = w; j < s; j += nw) {
        const int32_t xa = members[j];
        const int32_t u = cl[xa];
        const int64_t base = coff[u];
        const int c = (int)(coff[u + 1] - base);
        const int a = (int)(j - base);
        const int64_t ra = pos[xa];
        for (int b = lane; b < c; b += 32) acc[b] = 0.0;
        __syncwarp();
        // row x_a's entries 32 at a time: lane t loads entry t's value and
        // its transposed column's range (one load chain for all of them),
        // then the entries are taken in ascending order from the registers
        const int64_t q0 = rp[ra], q1 = rp[ra + 1];
        for (int64_t qb = q0; qb < q1; qb += 32) {
            double va_l = 0.0;
            int64_t e0_l = 0, e1_l = 0;
            if (qb + lane < q1) {
                va_l = v[qb + lane];
                const int64_t rr = pos[ci[qb + lane]];
                e0_l = trp[rr];
                e1_l = trp[rr + 1];
            }
            const int nq = (int)(q1 - qb < 32 ? q1 - qb : 32);
            // the first 32 entries of the next column are loaded while the
            // current one is accumulated
            int64_t ul_n = -1;
            double tv_n = 0.0;
            {
                const int64_t e0 = __shfl_sync(0xffffffffu, e0_l, 0);
                const int64_t e1 = __shfl_sync(0xffffffffu, e1_l, 0);
                if (e0 + lane < e1) {
                    ul_n = tul[e0 + lane];
                    tv_n = tv[e0 + lane];
                }
            }
            for (int t = 0; t < nq; ++t) {
                const double va = __shfl_sync(0xffffffffu, va_l, t);
                const int64_t e0 = __shfl_sync(0xffffffffu, e0_l, t);
                const int64_t e1 = __shfl_sync(0xffffffffu, e1_l, t);
                const int64_t ul0 = ul_n;
                const double tv0 = tv_n;
                if (t + 1 < nq) {
                    const int64_t f0 = __shfl_sync(0xffffffffu, e0_l, t + 1);
                    const int64_t f1 = __shfl_sync(0xffffffffu, e1_l, t + 1);
                    ul_n = -1;
                    if (f0 + lane < f1) {
                        ul_n = tul[f0 + lane];
                        tv_n = tv[f0 + lane];
                    }
                }
                if (e0 + lane < e1 && (int32_t)(ul0 >> 32) == u) {
                    const int lb = (int)(uint32_t)ul0;
                    acc[lb] = __fma_rn(va, tv0, acc[lb]);
                }
                for (int64_t e = e0 + 32 + lane; e < e1; e += 32) {
                    const int64_t ul = tul[e];
                    if ((int32_t)(ul >> 32) == u) {
                        const int lb = (int)(uint32_t)ul;
                        acc[lb] = __fma_rn(va, tv[e], acc[lb]);
                    }
                }
                __syncwarp();
            }
        }
        double *Gr = G + goff[u] + (int64_t)a * c;
        for (int b = lane; b < c; b += 32) Gr[b] = acc[b];
        __syncwarp();
        for (int b = lane; b < c; b += 32) acc[b] = 0.0;
        __syncwarp();
        for (int64_t q = rp[ra] + lane; q < rp[ra + 1]; q += 32) {
            const int32_t xb = ci[q];
            if (cl[xb] == u && loc[xb] >= a) acc[loc[xb]] = v[q];
        }
        for (int64_t e = trp[ra] + lane; e < trp[ra + 1]; e += 32) {
            const int64_t ul = tul[e];
            const int lb = (int)(uint32_t)ul;
            if ((int32_t)(ul >> 32) == u && lb < a) acc[lb] = tv[e];
        }
        __syncwarp();
        double *Mr = M + goff[u] + (int64_t)a * c;
        for (int b = lane; b < c; b += 32) Mr[b] = acc[b];
        __syncwarp();
    }
}

constexpr int SEL_THREADS = 256;
constexpr int SEL_WARPS = SEL_THREADS / 32;

// Candidate of the partner search: the score's bit pattern (scores are
// non-negative doubles, so their bits order like their values), the local
// index, and the pivot row's G and M entries at that index.
struct Cand {
    unsigned long long key;
    int32_t idx;
    double g, m;
};

__device__ __forceinline__ bool cand_better(unsigned long long k1, int32_t i1,
                                            unsigned long long k2, int32_t i2) {
    return k1 > k2 || (k1 == k2 && i1 < i2);
}

__device__ __forceinline__ void cand_merge(Cand &a, const Cand &b) {
    if (cand_better(b.key, b.idx, a.key, a.idx)) a = b;
}

__device__ __forceinline__ Cand cand_make(double g, double m, double wy, int32_t y) {
    // |g| * w = |g * w| bit for bit (round to nearest is symmetric, w >= 0)
    return Cand{f64_bits(__dmul_rn(g, wy)) & F64_ABS, y, g, m};
}

// True when x is +0 or -0, tested on the bits (integer pipe, not FP64).
__device__ __forceinline__ bool is_zero(double x) {
    return (f64_bits(x) << 1) == 0ull;
}

// Same candidate as cand_make; a zero entry scores +0 (key 0) without an FP64
// multiply (|+-0| * w = +0 for the finite, non-negative w).
__device__ __forceinline__ Cand cand_make_sparse(double g, double m, double wy, int32_t y) {
    return is_zero(g) ? Cand{0ull, y, g, m} : cand_make(g, m, wy, y);
}

__device__ __forceinline__ Cand cand_none() { return Cand{0ull, 0x7fffffff, 0.0, 0.0}; }

__device__ __forceinline__ Cand warp_argmax(Cand c) {
    for (int o = 16; o > 0; o >>= 1) {
        Cand x;
        x.key = __shfl_xor_sync(0xffffffffu, c.key, o);
        x.idx = __shfl_xor_sync(0xffffffffu, c.idx, o);
        x.g = __shfl_xor_sync(0xffffffffu, c.g, o);
        x.m = __shfl_xor_sync(0xffffffffu, c.m, o);
        cand_merge(c, x);
    }
    return c;
}

// Warp argmax that moves only (key, index) between lanes; the lane that holds
// the winner writes the full candidate to *out.
__device__ __forceinline__ int warp_argmax_to(const Cand &mine, Cand *out) {
    unsigned long long k = mine.key;
    int32_t id = mine.idx;
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long ok = __shfl_xor_sync(0xffffffffu, k, o);
        const int32_t oi = __shfl_xor_sync(0xffffffffu, id, o);
        if (cand_better(ok, oi, k, id)) {
            k = ok;
            id = oi;
        }
    }
    const unsigned own = __ballot_sync(0xffffffffu, mine.idx == id && mine.key == k);
    if (own == 0) {
        if ((threadIdx.x & 31) == 0) *out = cand_none();
    } else if ((threadIdx.x & 31) == __ffs(own) - 1) {
        *out = mine;
    }
    return own ? id : -1;   // the warp's best index, in every lane
}

__device__ __forceinline__ bool is_active(const uint32_t *mask, int y) {
    return (mask[y >> 5] >> (y & 31)) & 1u;
}

// Position 'pos' among the set bits of mask, treating bit 'skip' as clear
// (one thread): word scan, then a popcount bisection inside the word.
__device__ int select_bit(const uint32_t *mask, int nwords, int64_t pos, int skip) {
    int rem = (int)pos;
    for (int wi = 0; wi < nwords; ++wi) {
        uint32_t m = mask[wi];
        if (skip >= 0 && (skip >> 5) == wi) m &= ~(1u << (skip & 31));
        const int pc = __popc(m);
        if (rem < pc) {
            int base = 0;
            for (int width = 16; width >= 1; width >>= 1) {
                const int lc = __popc((m >> base) & ((1u << width) - 1u));
                if (rem >= lc) {
                    rem -= lc;
                    base += width;
                }
            }
            return wi * 32 + base;
        }
        rem -= pc;
    }
    return -1;
}

// Group a cluster's rotations by dependency level (rotations of one level
// touch disjoint coordinates, so any order inside a level gives the same
// bits) and flag the eliminated coordinates.
__device__ void finish_cluster(int64_t u, int64_t r0, int e, int nl, const int32_t *members,
                               int64_t base, const RotRec *rec, int32_t *lcnt, Rot2 *lvlrot,
                               int32_t *lvl_off, int32_t *nlev, int32_t *elimflag, int64_t stage) {
    const int tid = threadIdx.x;
    for (int t = tid; t < e; t += blockDim.x) {
        const RotRec rr = rec[r0 + t];
        atomicAdd(&lcnt[rr.lvl], 1);
        elimflag[members[base + rr.le]] = (int32_t)stage;
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
    for (int t = tid; t < e; t += blockDim.x) {
        const RotRec rr = rec[r0 + t];
        const int slot = atomicAdd(&lcnt[rr.lvl], 1);
        lvlrot[r0 + slot] = Rot2{rr.li, rr.lj, rr.c, rr.s};
    }
}

// Generic search (any cluster size; used above 8 * SEL_THREADS coordinates).
// Shared memory: G and M diagonals, w, the active mask, per-coordinate
// dependency levels and level counters.
__global__ void __launch_bounds__(SEL_THREADS)
k_select(const int64_t *coff, const int32_t *members, const int64_t *goff, double *Gall,
         double *Mall, const int64_t *roff, uint64_t seed, int64_t stage, RotRec *rec, Rot2 *lvlrot,
         int32_t *lvl_off, int32_t *nlev, int32_t *elimflag, const int32_t *order,
         const uint64_t *useed, const int32_t *ords) {
    extern __shared__ double sh[];
    const int64_t u = order ? order[blockIdx.x] : blockIdx.x;
    const int64_t base = coff[u];
    const int c = (int)(coff[u + 1] - base);
    const int64_t r0 = roff[u];
    const int e = (int)(roff[u + 1] - r0);
    double *G = Gall + goff[u];
    double *M = Mall + goff[u];
    double *gd = sh;
    double *md = gd + c;
    double *w = md + c;
    const int nwords = (c + 31) / 32;
    uint32_t *mask = (uint32_t *)(w + c);
    int32_t *lvl = (int32_t *)(mask + nwords);
    int32_t *lcnt = lvl + c;          // e + 2 counters
    __shared__ Cand wbest[SEL_WARPS];
    __shared__ int s_i, s_j, s_maxlev;
    __shared__ double s_c, s_s;

    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    for (int a = tid; a < c; a += SEL_THREADS) {
        double g = G[(int64_t)a * c + a];
        gd[a] = g;
        md[a] = M[(int64_t)a * c + a];
        w[a] = g > 0.0 ? __ddiv_rn(1.0, __dsqrt_rn(g)) : 0.0;
        lvl[a] = 0;
    }
    for (int wi = tid; wi < nwords; wi += SEL_THREADS) {
        int rem = c - wi * 32;
        mask[wi] = rem >= 32 ? 0xffffffffu : ((1u << rem) - 1u);
    }
    for (int q = tid; q < e + 2; q += SEL_THREADS) lcnt[q] = 0;
    __syncthreads();
    if (tid == 0) {
        s_maxlev = 0;
        if (e > 0) s_i = select_bit(mask, nwords, (int64_t)__umul64hi(draw(useed ? useed[u] : seed, stage, useed ? 0 : (ords ? ords[u] : u), 0), (uint64_t)c), -1);
    }
    __syncthreads();

    for (int t = 0; t < e; ++t) {
        const int i = s_i < 0 ? 0 : s_i;
        const double *Gi = G + (int64_t)i * c;
        Cand best = cand_none();
        for (int y = tid; y < c; y += SEL_THREADS) {
            if (y == i || !is_active(mask, y)) continue;
            cand_merge(best, cand_make(Gi[y], 0.0, w[y], y));
        }
        best = warp_argmax(best);
        if (lane == 0) wbest[wid] = best;
        __syncthreads();
        if (tid == 0) {
            for (int q = 1; q < SEL_WARPS; ++q) cand_merge(best, wbest[q]);
            // at least two coordinates are active at every step (e_u <= c_u - 1);
            // the clamp only keeps a corrupted state from indexing out of bounds
            const int j = (best.idx >= 0 && best.idx < c && best.idx != i) ? best.idx : (i == 0 ? 1 : 0);
            double cc, ss;
            const double gij = G[(int64_t)i * c + j];
            jacobi2(gd[i], gij, gd[j], cc, ss);
            double na, nb, nd;
            rot_block(cc, ss, gd[i], gij, gd[j], na, nb, nd);
            G[(int64_t)i * c + i] = na;
            G[(int64_t)j * c + j] = nd;
            G[(int64_t)i * c + j] = nb;
            G[(int64_t)j * c + i] = nb;
            gd[i] = na;
            gd[j] = nd;
            const double mij = M[(int64_t)i * c + j];
            rot_block(cc, ss, md[i], mij, md[j], na, nb, nd);
            M[(int64_t)i * c + i] = na;
            M[(int64_t)j * c + j] = nd;
            M[(int64_t)i * c + j] = nb;
            M[(int64_t)j * c + i] = nb;
            md[i] = na;
            md[j] = nd;
            w[i] = gd[i] > 0.0 ? __ddiv_rn(1.0, __dsqrt_rn(gd[i])) : 0.0;
            w[j] = gd[j] > 0.0 ? __ddiv_rn(1.0, __dsqrt_rn(gd[j])) : 0.0;
            const double di = __dsub_rn(gd[i], __dmul_rn(md[i], md[i]));
            const double dj = __dsub_rn(gd[j], __dmul_rn(md[j], md[j]));
            const int le = di < dj ? i : j;
            const int L = 1 + max(lvl[i], lvl[j]);
            lvl[i] = L;
            lvl[j] = L;
            s_maxlev = max(s_maxlev, L);
            rec[r0 + t] = RotRec{i, j, le, L, cc, ss};
            mask[le >> 5] &= ~(1u << (le & 31));
            s_j = j;
            s_c = cc;
            s_s = ss;
            if (t + 1 < e)
                s_i = select_bit(mask, nwords,
                                 (int64_t)__umul64hi(draw(useed ? useed[u] : seed, stage, useed ? 0 : (ords ? ords[u] : u), t + 1), (uint64_t)(c - t - 1)), -1);
        }
        __syncthreads();
        // rows/columns i and j of G and M for every other active coordinate
        {
            const int j = s_j;
            const double cc = s_c, ss = s_s;
            double *Gw = G + (int64_t)i * c;
            double *Gj = G + (int64_t)j * c;
            double *Mi = M + (int64_t)i * c;
            double *Mj = M + (int64_t)j * c;
            for (int y = tid; y < c; y += SEL_THREADS) {
                if (y == i || y == j || !is_active(mask, y)) continue;
                double gi = Gw[y], gj = Gj[y];
                if (gi != 0.0 || gj != 0.0) {
                    double ni, nj;
                    rot_pair(cc, ss, gi, gj, ni, nj);
                    Gw[y] = ni;
                    Gj[y] = nj;
                    G[(int64_t)y * c + i] = ni;
                    G[(int64_t)y * c + j] = nj;
                }
                double mi = Mi[y], mj = Mj[y];
                if (mi != 0.0 || mj != 0.0) {
                    double ni, nj;
                    rot_pair(cc, ss, mi, mj, ni, nj);
                    Mi[y] = ni;
                    Mj[y] = nj;
                    M[(int64_t)y * c + i] = ni;
                    M[(int64_t)y * c + j] = nj;
                }
            }
        }
        __syncthreads();
    }
    finish_cluster(u, r0, e, s_maxlev, members, base, rec, lcnt, lvlrot, lvl_off, nlev, elimflag, stage);
}

// Restructured search for clusters of up to KPT * SEL_THREADS coordinates
// (thread t owns columns t, t + SEL_THREADS, ...).  Per step t with pivot i
// and partner j:
//   P1  thread 0: angle, 2x2 blocks of G and M, elimination, level, record.
//       Warp 1: the two rows that can be the pivot of step t + 2, for both
//       possible eliminations.  Every thread: prefetch its columns of rows i
//       and j and of the two rows a1, a2 that can be the pivot of step t + 1.
//   P2  every thread rotates its columns of rows i and j (and the mirrored
//       columns) and scores them for the next pivot; warp argmax.
// Two barriers per step.  The arithmetic, and so every bit, is k_select's.
// An entry of the per-step FP64 work list: a column y, what it needs, and the
// values its owner thread prefetched.
enum : int { W_G = 1, W_M = 2, W_SCORE = 4 };
struct Work {
    int32_t y, flags;
    double gi, gj, mi, mj, g1, m1, g2, m2;
};

// Warps of the restructured search: warps 0..3 (one per SM sub-partition,
// each with its own FP64 unit) share the step's serial FP64 work; warps
// 4..SEL_WARPS-1 own the columns.
constexpr int FP_WARPS = 4;
constexpr int NCT = SEL_THREADS - 32 * FP_WARPS;

// Barrier among the FP64 warps only (named barrier 1).
__device__ __forceinline__ void fp_sync() {
    asm volatile("bar.sync 1, %0;" ::"n"(32 * FP_WARPS) : "memory");
}

// Best of the per-warp candidates, computed by every warp in parallel.
template <int NWARPS>
__device__ __forceinline__ Cand block_best(const Cand *wb) {
    const int lane = threadIdx.x & 31;
    const Cand mine = lane < NWARPS ? wb[lane] : cand_none();
    unsigned long long k = mine.key;
    int32_t id = mine.idx;
    for (int o = NWARPS / 2; o > 0; o >>= 1) {
        const unsigned long long ok = __shfl_xor_sync(0xffffffffu, k, o);
        const int32_t oi = __shfl_xor_sync(0xffffffffu, id, o);
        if (cand_better(ok, oi, k, id)) {
            k = ok;
            id = oi;
        }
    }
    k = __shfl_sync(0xffffffffu, k, 0);
    id = __shfl_sync(0xffffffffu, id, 0);
    const unsigned own = __ballot_sync(0xffffffffu, lane < NWARPS && mine.idx == id && mine.key == k);
    const int src = own ? __ffs(own) - 1 : 0;
    Cand r;
    r.key = k;
    r.idx = id;
    r.g = __shfl_sync(0xffffffffu, mine.g, src);
    r.m = __shfl_sync(0xffffffffu, mine.m, src);
    return r;
}

// Restructured search for clusters of up to KPT * NCT coordinates (column
// thread t owns columns t, t + NCT, ...).  Per step t with pivot i, partner j:
//   P1   FP64 warps: warp 0 computes the angle (its prefix once, c and s
//        by two lanes of one divide), the four new diagonal entries of the
//        2x2 blocks (four lanes) and then the new weights of i and j (two
//        lanes), beside the elimination and bookkeeping (warp 2) and the
//        candidates for the pivot of step t + 2 (warp 3); an FP64 instruction
//        holds the SM's FP64 pipe whatever its lanes do, so one warp's lanes
//        take what several warps took before, at the same latency.  Column threads: load their
//        columns of rows i, j and of the two rows a1, a2 that can be the pivot
//        of step t + 1, classify them and list those that may need FP64 work.
//   P2   column threads: FP64 work on the listed columns (the survivor's row
//        and column; the eliminated coordinate's are never read again), zero
//        and nonzero candidates for the next pivot; warp argmax.  FP64 warps:
//        the block's best merged with the survivor's own candidate.
// Barriers per step: named barrier 4 between P1 and P2 (every warp but FP64
// warps 0 and 1), 2 (column warps arrive with their bests, FP64 warps wait)
// and 3 (FP64 warps arrive with the next (i, j), column warps wait); FP64
// warps also meet at named barrier 1.  The arithmetic, and so every bit, is
// k_select's.
template <int KPT, int NT, int MINB = (NT <= 256 ? 2 : 1)>
__global__ void __launch_bounds__(NT, MINB)
k_select_fast(const int64_t *coff, const int32_t *members, const int64_t *goff, double *Gall,
              double *Mall, const int64_t *roff, uint64_t seed, int64_t stage, RotRec *rec,
              Rot2 *lvlrot, int32_t *lvl_off, int32_t *nlev, int32_t *elimflag,
              const int32_t *order, const uint64_t *useed, const int32_t *ords) {
    constexpr int NW = NT / 32;                 // warps
    constexpr int NCTT = NT - 32 * FP_WARPS;    // column threads
    extern __shared__ double sh[];
    const int64_t u = order ? order[blockIdx.x] : blockIdx.x;
    const int64_t base = coff[u];
    const int c = (int)(coff[u + 1] - base);
    const int64_t r0 = roff[u];
    const int e = (int)(roff[u + 1] - r0);
    double *G = Gall + goff[u];
    double *M = Mall + goff[u];
    double *gd = sh;
    double *md = gd + c;
    double *w = md + c;
    uint64_t *draws = (uint64_t *)(w + c);
    const int nwords = (c + 31) / 32;
    uint32_t *mask = (uint32_t *)(draws + e + 1);
    int32_t *lvl = (int32_t *)(mask + nwords);
    int32_t *lcnt = lvl + c;          // e + 2 counters
    // c entries after the counters, 16-byte aligned (the launch adds the slack)
    Work *work = (Work *)(((uintptr_t)(lcnt + e + 2) + 15) & ~(uintptr_t)15);
    __shared__ Cand wbest[NW];
    __shared__ int s_le, s_maxlev, s_a1, s_a2;
    __shared__ int s_nwork[2];                  // by step parity
    __shared__ int s_nb[2][4];                  // by step parity: [skip i: p, p+1, skip j: p, p+1]
    __shared__ double s_c, s_s;
    __shared__ double s_x[FP_WARPS];            // exchange among the FP64 warps
    __shared__ double s_wn[2][2];               // new weights of i, j by step parity
    __shared__ double s_survg[2], s_survm[2];   // by step parity
    __shared__ int s_nx[4];                      // next step's i, j, a1, a2 (FP64 -> column warps)
    __shared__ double s_nxg, s_nxm;              // and its G_ij, M_ij

    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int ct = tid - 32 * FP_WARPS;         // column thread index (>= 0 in column warps)
    for (int a = tid; a < c; a += NT) {
        const double g = G[(int64_t)a * c + a];
        gd[a] = g;
        md[a] = M[(int64_t)a * c + a];
        w[a] = g > 0.0 ? __ddiv_rn(1.0, __dsqrt_rn(g)) : 0.0;
        lvl[a] = 0;
    }
    for (int wi = tid; wi < nwords; wi += NT) {
        const int rem = c - wi * 32;
        mask[wi] = rem >= 32 ? 0xffffffffu : ((1u << rem) - 1u);
    }
    for (int t = tid; t < e; t += NT) draws[t] = draw(useed ? useed[u] : seed, stage, useed ? 0 : (ords ? ords[u] : u), t);
    for (int q = tid; q < e + 2; q += NT) lcnt[q] = 0;
    __syncthreads();
    if (tid == 0) {
        s_maxlev = 0;
        s_a1 = s_a2 = -1;
        s_le = -1;
        s_nwork[0] = s_nwork[1] = 0;
        if (e > 1) {
            const int64_t p1 = (int64_t)__umul64hi(draws[1], (uint64_t)(c - 1));
            s_a1 = select_bit(mask, nwords, p1, -1);
            s_a2 = select_bit(mask, nwords, p1 + 1, -1);
        }
    }
    __syncthreads();
    if (e > 0) {
        int i = select_bit(mask, nwords, (int64_t)__umul64hi(draws[0], (uint64_t)c), -1);
        // partner search for the first pivot
        Cand best = cand_none();
        if (ct >= 0)
            for (int y = ct; y < c; y += NCTT) {
                if (y == i || !is_active(mask, y)) continue;
                cand_merge(best, cand_make_sparse(G[(int64_t)i * c + y], M[(int64_t)i * c + y], w[y], y));
            }
        warp_argmax_to(best, &wbest[wid]);
        __syncthreads();
        best = block_best<NW>(wbest);
        int j = best.idx;
        double gij = best.g, mij = best.m;
        int a1 = s_a1, a2 = s_a2;

        for (int t = 0; t < e; ++t) {
            const bool more = t + 1 < e;
            const int par = t & 1;
            if (i < 0 || i >= c) i = 0;                          // never taken; keeps
            if (j < 0 || j >= c || j == i) j = i == 0 ? 1 : 0;   // indices in range
            int zy[KPT];                                         // zero-score columns
#pragma unroll
            for (int k = 0; k < KPT; ++k) zy[k] = -1;
            if (ct >= 0) {
                // ---- P1, column threads: the loaded values are consumed here,
                // so the loads complete under the FP64 warps' chain
                double gi[KPT], gj[KPT], mi[KPT], mj[KPT], g1[KPT], m1[KPT], g2[KPT], m2[KPT];
                unsigned bal[KPT];
                int fl[KPT];
                int total = 0;
#pragma unroll
                for (int k = 0; k < KPT; ++k) {
                    const int y = ct + k * NCTT;
                    gi[k] = gj[k] = mi[k] = mj[k] = g1[k] = m1[k] = g2[k] = m2[k] = 0.0;
                    const bool live = y < c && y != i && y != j && is_active(mask, y);
                    if (live) {
                        gi[k] = G[(int64_t)i * c + y];
                        gj[k] = G[(int64_t)j * c + y];
                        mi[k] = M[(int64_t)i * c + y];
                        mj[k] = M[(int64_t)j * c + y];
                        if (more && a1 >= 0 && a1 != i && a1 != j) {
                            g1[k] = G[(int64_t)a1 * c + y];
                            m1[k] = M[(int64_t)a1 * c + y];
                        }
                        if (more && a2 >= 0 && a2 != i && a2 != j) {
                            g2[k] = G[(int64_t)a2 * c + y];
                            m2[k] = M[(int64_t)a2 * c + y];
                        }
                    }
                    int f = 0;
                    if (live) {
                        if (!(is_zero(gi[k]) && is_zero(gj[k]))) f |= W_G;
                        if (!(is_zero(mi[k]) && is_zero(mj[k]))) f |= W_M;
                        if (!is_zero(g1[k]) || !is_zero(g2[k])) f |= W_SCORE;
                    }
                    fl[k] = f;
                    zy[k] = (live && f == 0) ? y : -1;
                    bal[k] = __ballot_sync(0xffffffffu, f != 0);
                    total += __popc(bal[k]);
                }
                int wbase = 0;
                if (lane == 0 && total) wbase = atomicAdd(&s_nwork[par], total);
                wbase = __shfl_sync(0xffffffffu, wbase, 0);
#pragma unroll
                for (int k = 0; k < KPT; ++k) {
                    if (fl[k]) {
                        Work &it = work[wbase + __popc(bal[k] & ((1u << lane) - 1u))];
                        it.y = ct + k * NCTT;
                        it.flags = fl[k];
                        it.gi = gi[k];
                        it.gj = gj[k];
                        it.mi = mi[k];
                        it.mj = mj[k];
                        it.g1 = g1[k];
                        it.m1 = m1[k];
                        it.g2 = g2[k];
                        it.m2 = m2[k];
                    }
                    wbase += __popc(bal[k]);
                }
            } else {
                // ---- P1, FP64 warps (all lanes of a warp compute the same
                // values; an FP64 instruction costs the same for one lane or 32)
                const double a = gd[i], d = gd[j], ma0 = md[i], md0 = md[j];
                double cc, ss;
                const unsigned long long ABS = 0x7fffffffffffffffull;
                if ((f64_bits(gij) & ABS) == 0) {
                    cc = 1.0;
                    ss = 0.0;
                } else {
                    // the angle (jacobi2) by warp 0 alone: its prefix once,
                    // then c (lane 0) and s (the other lanes) as one divide
                    // with lane-dependent numerators, so warps 1-3 stay off the
                    // SM's FP64 pipe meanwhile
                    if (wid == 0) {
                        double h = __dsub_rn(d, a);
                        double g = __dmul_rn(2.0, gij);
                        const unsigned long long hm = f64_bits(h) & ABS, gm = f64_bits(g) & ABS;
                        const unsigned long long mm = hm > gm ? hm : gm;
                        if (mm > (unsigned long long)__double_as_longlong(0x1p500)) {
                            h = __dmul_rn(h, 0x1p-600);
                            g = __dmul_rn(g, 0x1p-600);
                        } else if (mm < (unsigned long long)__double_as_longlong(0x1p-500)) {
                            h = __dmul_rn(h, 0x1p600);
                            g = __dmul_rn(g, 0x1p600);
                        }
                        const unsigned long long hb = f64_bits(h);
                        const double habs = f64_from_bits(hb & ABS);
                        const bool hnonneg = (hb >> 63) == 0 || (hb & ABS) == 0;
                        const double g2v = __dmul_rn(g, g);
                        const double r = __dsqrt_rn(__dadd_rn(__dmul_rn(h, h), g2v));
                        const double q = __dadd_rn(habs, r);
                        const double den = __dsqrt_rn(__dadd_rn(__dmul_rn(q, q), g2v));
                        const double num = lane == 0 ? q : (hnonneg ? g : f64_from_bits(f64_bits(g) ^ ~ABS));
                        const double v = __ddiv_rn(num, den);
                        if (lane < 2) s_x[lane] = v;
                    }
                    fp_sync();
                    cc = s_x[0];
                    ss = s_x[1];
                    fp_sync();
                }
                // new diagonal entries of the 2x2 blocks (rot_block's na, nd):
                // G_ii, G_jj, M_ii, M_jj by lanes 0-3 of warp 0, one formula
                // with (p, q) = (c, -s) for the i entries and (s, c) for the j
                // entries: rot_block's operations, the negations exact
                if (wid == 0 && lane < 4) {
                    const bool gm = lane < 2, ev = (lane & 1) == 0;
                    const double xa = gm ? a : ma0;
                    const double xb = gm ? gij : mij;
                    const double xd = gm ? d : md0;
                    const double p = ev ? cc : ss;
                    const double qv = ev ? -ss : cc;
                    const double r1 = __fma_rn(p, xa, __dmul_rn(qv, xb));
                    const double r2 = __fma_rn(p, xb, __dmul_rn(qv, xd));
                    s_x[lane] = __fma_rn(r1, p, __dmul_rn(r2, qv));
                }
                fp_sync();
                const double na = s_x[0], nd = s_x[1], ma = s_x[2], md2 = s_x[3];
                if (wid == 0) {
                    // the new weights of i (lane 0) and j (lane 1), next to
                    // the elimination rather than after it; the survivor's is
                    // merged in P2 (the eliminated one is never read again)
                    const double x = lane == 0 ? na : nd;
                    const double wv = pos_bits(x) ? __ddiv_rn(1.0, __dsqrt_rn(x)) : 0.0;
                    if (lane < 2) {
                        s_wn[par][lane] = wv;
                        w[lane == 0 ? i : j] = wv;
                    }
                } else if (wid == 2 && lane == 0) {
                    const double di = __dsub_rn(na, __dmul_rn(ma, ma));
                    const double dj = __dsub_rn(nd, __dmul_rn(md2, md2));
                    const int le = lt_bits(di, dj) ? i : j;
                    gd[i] = na;
                    gd[j] = nd;
                    md[i] = ma;
                    md[j] = md2;
                    const int L = 1 + max(lvl[i], lvl[j]);
                    lvl[i] = L;
                    lvl[j] = L;
                    s_maxlev = max(s_maxlev, L);
                    mask[le >> 5] &= ~(1u << (le & 31));
                    s_c = cc;
                    s_s = ss;
                    s_le = le;
                    s_survg[par] = 0.0;
                    s_survm[par] = 0.0;
                    s_nwork[par ^ 1] = 0;                        // list count of step t + 1
                    rec[r0 + t] = RotRec{i, j, le, L, cc, ss};
                } else if (wid == 3 && lane < 4 && t + 2 < e) {
                    // candidates for the pivot of step t + 2, for both possible
                    // eliminations; the mask word may or may not show the update
                    // yet, but the matching hypothesis reads the same bits
                    const int64_t p2 = (int64_t)__umul64hi(draws[t + 2], (uint64_t)(c - t - 2));
                    s_nb[par][lane] = select_bit(mask, nwords, p2 + (lane & 1), lane < 2 ? i : j);
                }
            }
            // S1 (barrier 4): the column warps and FP64 warps 2 and 3, once per
            // step.  Warps 0 and 1 (the weights) go straight on to barrier 2
            // and read the elimination from behind it.
            if (wid >= 2) asm volatile("bar.sync 4, %0;" ::"n"(NT - 64) : "memory");
            // ---- P2.  Column warps: (A) score the candidates of the next
            // pivot and publish each warp's best (barrier 2, arrive), (B) write
            // the survivor's rotated row and column into G and M, then take the
            // next step's (i, j) (barrier 3, wait).  FP64 warps: (barrier 2,
            // wait) the block's best partner merged with the survivor's own
            // candidate, published with barrier 3 (arrive), and on to the next
            // step's chain while the column warps are still writing.  Both
            // roles pass barriers 2 and 3 exactly once per step with a next
            // step; the column warps' writes are visible to their next loads
            // through barrier 3.
            if (ct >= 0) {
                const double cc = s_c, ss = s_s;
                const int le = s_le;
                const int surv = le == i ? j : i;
                // the pivot of step t + 1 is the p-th survivor: a1 unless the
                // eliminated index sits at or before it
                const int inext = more ? (le <= a1 ? a2 : a1) : -1;
                if (more) {
                    const int nwork = s_nwork[par];
                    const bool si = surv == i;
                    Cand nbest = cand_none();
#pragma unroll
                    for (int k = 0; k < KPT; ++k)
                        if (zy[k] >= 0 && zy[k] != inext) cand_merge(nbest, Cand{0ull, zy[k], 0.0, 0.0});
                    // (A) the next pivot is the survivor, a1 or a2 (never the
                    // eliminated coordinate); only the survivor's row changed
                    for (int q = ct; q < nwork; q += NCTT) {
                        const Work it = work[q];
                        const int y = it.y;
                        if (y == inext || inext == surv) {
                            double sg = si ? it.gi : it.gj, sm = si ? it.mi : it.mj;
                            if (it.flags & W_G) sg = rot_pair_one(cc, ss, it.gi, it.gj, si);
                            if (it.flags & W_M) sm = rot_pair_one(cc, ss, it.mi, it.mj, si);
                            if (y == inext) {
                                // column inext of the survivor's new row
                                s_survg[par] = sg;
                                s_survm[par] = sm;
                                continue;
                            }
                            cand_merge(nbest, cand_make_sparse(sg, sm, w[y], y));
                        } else {
                            const bool o1 = inext == a1;
                            cand_merge(nbest, cand_make_sparse(o1 ? it.g1 : it.g2, o1 ? it.m1 : it.m2,
                                                               w[y], y));
                        }
                    }
                    const int pb = warp_argmax_to(nbest, &wbest[wid]);
                    asm volatile("bar.arrive 2, %0;" ::"n"(NT) : "memory");
                    // the next partner is one of the column warps' bests or
                    // the survivor: start moving this warp's best rows of G
                    // and M into L2 (the first stages' Gram blocks exceed it)
                    if (pb >= 0 && pb < c && lane * 16 < c) {
                        asm volatile("prefetch.L2 [%0];" ::"l"(G + (int64_t)pb * c + lane * 16));
                        asm volatile("prefetch.L2 [%0];" ::"l"(M + (int64_t)pb * c + lane * 16));
                    }
                    // (B) only the survivor's row and column are read again, so
                    // only its output of each rotated pair is formed
                    for (int q = ct; q < nwork; q += NCTT) {
                        const Work it = work[q];
                        const int y = it.y;
                        if (it.flags & W_G) {
                            const double sg = rot_pair_one(cc, ss, it.gi, it.gj, si);
                            G[(int64_t)surv * c + y] = sg;
                            G[(int64_t)y * c + surv] = sg;
                        }
                        if (it.flags & W_M) {
                            const double sm = rot_pair_one(cc, ss, it.mi, it.mj, si);
                            M[(int64_t)surv * c + y] = sm;
                            M[(int64_t)y * c + surv] = sm;
                        }
                    }
                    asm volatile("bar.sync 3, %0;" ::"n"(NT) : "memory");
                    i = s_nx[0];
                    j = s_nx[1];
                    a1 = s_nx[2];
                    a2 = s_nx[3];
                    gij = s_nxg;
                    mij = s_nxm;
                }
            } else {
                if (more) {
                    if (lane == 0) wbest[wid] = cand_none();
                    asm volatile("bar.sync 2, %0;" ::"n"(NT) : "memory");
                    const int le = s_le;
                    const int surv = le == i ? j : i;
                    const int inext = le <= a1 ? a2 : a1;
                    Cand nbest = block_best<NW>(wbest);
                    if (inext != i && inext != j)
                        cand_merge(nbest, cand_make_sparse(s_survg[par], s_survm[par],
                                                           s_wn[par][surv == i ? 0 : 1], surv));
                    if (t + 2 < e) {
                        a1 = le == i ? s_nb[par][0] : s_nb[par][2];
                        a2 = le == i ? s_nb[par][1] : s_nb[par][3];
                    } else {
                        a1 = a2 = -1;
                    }
                    i = inext;
                    j = nbest.idx;
                    gij = nbest.g;
                    mij = nbest.m;
                    if (wid == 0 && lane == 0) {
                        s_nx[0] = i;
                        s_nx[1] = j;
                        s_nx[2] = a1;
                        s_nx[3] = a2;
                        s_nxg = gij;
                        s_nxm = mij;
                    }
                    asm volatile("bar.arrive 3, %0;" ::"n"(NT) : "memory");
                }
            }
        }
    }
    __syncthreads();
    finish_cluster(u, r0, e, s_maxlev, members, base, rec, lcnt, lvlrot, lvl_off, nlev, elimflag, stage);
}

// Search of one cluster by a thread-block cluster of DSM_CL CTAs that hold G
// and M in their shared memory, row-sliced: CTA r keeps rows [r R, (r + 1) R)
// of both (R = ceil(c / DSM_CL)); every CTA keeps the diagonals, the weights,
// the active mask and the levels, and takes every decision of a step itself
// (the same inputs, so the same bits everywhere).  A step's loads are
// shared-memory loads, local or distributed, instead of L2 loads.
//
// Step t starts with (i, j, G_ij, M_ij) in every CTA's mailbox and with a1,
// a2: the active coordinates at positions p and p + 1 (p the position drawn
// for step t + 1), one of which is the next pivot once the eliminated
// coordinate is known (le <= a1 ? a2 : a1).  Then:
//   A  warps 0 and 13: the angle's c and s (the same prefix, the two divides
//      on two sub-partitions).  Warp 14: the new weights of the previous
//      step's pair.  Warps 1-4 (5-8) of the CTA holding row a1 (a2), once
//      those weights are in: the partner search of that row over every
//      candidate but i and j (its other entries and their weights do not
//      change in step t).  Warps 9-11: columns i and j of the CTA's rows
//      loaded.
//   B  warp 0: the new diagonal entries of the 2 x 2 blocks (lanes 0-3), then
//      elimination, level, record and the next pivot i'; warps 9-11: the
//      CTA's rows rotated, the mirrored entries stored into rows i and j
//      where they are held.
//   C  the CTA holding
//      row i' merges the survivor's entry (its score bounded in FP32 first,
//      so its exact weight is needed only when it could win) and writes the
//      next (i', j', G, M) into every mailbox.  If i' is the survivor itself
//      (its row was just rotated everywhere) a cluster barrier comes first
//      and the row is searched in full.  Warp 15: a1, a2 of step t + 2.
//   cluster barrier.
// The arithmetic, and so every bit, is k_select's.  CTA 0 writes the records
// and finishes the cluster.  The launch keeps 2 R <= DSM_ROT_N (one rotation
// task per thread).
constexpr int DSM_CL = 8;
constexpr int DSM_THREADS = 512;
constexpr int DSM_WARPS = DSM_THREADS / 32;
constexpr int DSM_SCORE_WARPS = 4;   // per speculative row: warps 1-4 and 5-8
constexpr int DSM_ROT_T0 = 288;      // warps 9-11 rotate the CTA's rows
constexpr int DSM_ROT_N = 96;
constexpr int DSM_S_WARP = 13;       // the angle's s (warp 0: c), on its own sub-partition
constexpr int DSM_W_WARP = 14;       // the previous step's new weights
constexpr int DSM_NEXT_WARP = 15;    // a1, a2 of step t + 2

struct DsmMail {
    double g, m;
    int32_t j, pad;
};

__device__ __forceinline__ void cluster_arrive_release() {
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}

__device__ __forceinline__ void cluster_wait_acquire() {
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Named barrier of `count` threads: wait, or arrive without waiting.
__device__ __forceinline__ void named_sync(int id, int count) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

__device__ __forceinline__ void named_arrive(int id, int count) {
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// A float no larger than the finite double x > 0 (its exponent and top mantissa
// bits), or -1 when x is outside the normal float range.  Integer pipe only.
__device__ __forceinline__ float f32_below(double x) {
    const unsigned long long b = f64_bits(x) & 0x7fffffffffffffffull;
    const int e = (int)(b >> 52) - 1023;
    if (e < -125 || e > 126) return -1.0f;
    return __uint_as_float((unsigned)((e + 127) << 23) | (unsigned)((b >> 29) & 0x7fffffu));
}

// A float no smaller than |x| for a finite double, or -1 out of range.
__device__ __forceinline__ float f32_above(double x) {
    const float f = f32_below(x);
    return f < 0.0f ? f : __uint_as_float(__float_as_uint(f) + 1u);
}

// True when a coordinate with entry g and diagonal gss surely scores below
// the candidate key kb (a non-negative double's bits): |g| / sqrt(gss)
// bounded above in FP32 with a margin of 2^-18 (the rounding of the exact
// score, the truncations and rsqrtf's error are far smaller).  False means
// "maybe not": the caller decides exactly.
__device__ __forceinline__ bool surely_below(double g, double gss, unsigned long long kb) {
    if (kb == 0ull || (f64_bits(gss) >> 63)) return false;
    const float ga = f32_above(g), gd = f32_below(gss), bb = f32_below(f64_from_bits(kb));
    if (ga < 0.0f || gd <= 0.0f || bb <= 0.0f) return false;
    return ga * rsqrtf(gd) * (1.0f + 0x1p-18f) < bb;
}

// Partner search of row x (held by this CTA) over the active candidates but
// `skip1`, `skip2` and x itself, by the warps [w0, w0 + nw) (thread index
// tid - 32 w0 of 32 nw); each warp's best goes to wb[warp - w0].
__device__ __forceinline__ void dsm_score_row(const double *Gx, const double *Mx, const double *w,
                                              const uint32_t *mask, int c, int x, int skip1, int skip2,
                                              int w0, int nw, Cand *wb) {
    const int t = threadIdx.x - 32 * w0;
    Cand best = cand_none();
    for (int y = t; y < c; y += 32 * nw) {
        if (y == x || y == skip1 || y == skip2 || !is_active(mask, y)) continue;
        cand_merge(best, cand_make(Gx[y], Mx[y], w[y], y));
    }
    warp_argmax_to(best, &wb[t >> 5]);
}

// Best of n (<= 32) candidates, in every lane of the calling warp.
__device__ __forceinline__ Cand dsm_best_of(const Cand *wb, int n) {
    const int lane = threadIdx.x & 31;
    return warp_argmax(lane < n ? wb[lane] : cand_none());
}

__global__ void __cluster_dims__(DSM_CL, 1, 1) __launch_bounds__(DSM_THREADS, 1)
k_select_dsm(const int64_t *coff, const int32_t *members, const int64_t *goff, const double *Gall,
             const double *Mall, const int64_t *roff, uint64_t seed, int64_t stage, RotRec *rec,
             Rot2 *lvlrot, int32_t *lvl_off, int32_t *nlev, int32_t *elimflag,
             const int32_t *order, const uint64_t *useed, const int32_t *ords) {
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    extern __shared__ double sh[];
    const int rank = (int)cluster.block_rank();
    const int64_t q = blockIdx.x / DSM_CL;
    const int64_t u = order ? order[q] : q;
    const int64_t base = coff[u];
    const int c = (int)(coff[u + 1] - base);
    const int64_t r0 = roff[u];
    const int e = (int)(roff[u + 1] - r0);
    const int R = (c + DSM_CL - 1) / DSM_CL;
    const int row0 = rank * R;
    const int nrow = max(0, min(c, row0 + R) - row0);
    const double *G = Gall + goff[u];
    const double *M = Mall + goff[u];
    double *Gs = sh;                          // R x c, this CTA's rows of G
    double *Ms = Gs + (size_t)R * c;          // R x c, of M
    double *gd = Ms + (size_t)R * c;
    double *md = gd + c;
    double *w = md + c;
    uint64_t *draws = (uint64_t *)(w + c);    // e + 1
    const int nwords = (c + 31) / 32;
    uint32_t *mask = (uint32_t *)(draws + e + 1);
    int32_t *lvl = (int32_t *)(mask + nwords);
    int32_t *lcnt = lvl + c;                  // e + 2 counters
    __shared__ DsmMail mail[2];               // by step parity
    __shared__ Cand wb[DSM_WARPS];            // per-warp bests
    __shared__ Cand spec[2];                  // partner searches of a1, a2
    __shared__ int s_a[2], s_le, s_ip, s_maxlev;
    __shared__ double s_c, s_s, s_blk[4];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;

    for (int64_t x = tid; x < (int64_t)nrow * c; x += DSM_THREADS) {
        Gs[x] = G[(int64_t)row0 * c + x];
        Ms[x] = M[(int64_t)row0 * c + x];
    }
    for (int a = tid; a < c; a += DSM_THREADS) {
        const double g = G[(int64_t)a * c + a];
        gd[a] = g;
        md[a] = M[(int64_t)a * c + a];
        w[a] = g > 0.0 ? __ddiv_rn(1.0, __dsqrt_rn(g)) : 0.0;
        lvl[a] = 0;
    }
    for (int wi = tid; wi < nwords; wi += DSM_THREADS) {
        const int rem = c - wi * 32;
        mask[wi] = rem >= 32 ? 0xffffffffu : ((1u << rem) - 1u);
    }
    for (int t = tid; t < e; t += DSM_THREADS)
        draws[t] = draw(useed ? useed[u] : seed, stage, useed ? 0 : (ords ? ords[u] : u), t);
    for (int x = tid; x < e + 2; x += DSM_THREADS) lcnt[x] = 0;
    __syncthreads();
    int i0 = 0;
    if (tid == 0) {
        s_maxlev = 0;
        s_a[0] = s_a[1] = -1;
        if (e > 1) {
            const int64_t p = (int64_t)__umul64hi(draws[1], (uint64_t)(c - 1));
            s_a[0] = select_bit(mask, nwords, p, -1);
            s_a[1] = select_bit(mask, nwords, p + 1, -1);
        }
        s_ip = e > 0 ? select_bit(mask, nwords, (int64_t)__umul64hi(draws[0], (uint64_t)c), -1) : 0;
    }
    __syncthreads();
    i0 = s_ip < 0 || s_ip >= c ? 0 : s_ip;
    // every CTA's shared memory is set before the first remote store
    cluster.sync();
    // the first pivot's partner, searched in full by the CTA holding its row
    if (e > 0 && rank == i0 / R) {
        dsm_score_row(Gs + (size_t)(i0 - row0) * c, Ms + (size_t)(i0 - row0) * c, w, mask, c, i0, -1, -1,
                      0, DSM_WARPS, wb);
        __syncthreads();
        if (wid == 0) {
            const Cand b = dsm_best_of(wb, DSM_WARPS);
            if (lane < DSM_CL) {
                DsmMail *dst = cluster.map_shared_rank(&mail[0], lane);
                dst->g = b.g;
                dst->m = b.m;
                dst->j = b.idx;
            }
        }
    }
    cluster.sync();

    // rotation task of this thread: G or M, one of the CTA's rows
    const int task = tid - DSM_ROT_T0;
    const bool has_task = task >= 0 && task < 2 * nrow;
    const int ly = has_task ? (task < nrow ? task : task - nrow) : 0;
    const int y = row0 + ly;
    double *Xs = (has_task && task >= nrow) ? Ms : Gs;
    double *Xr = Xs + (size_t)ly * c;

    int i = i0, pi = 0, pj = 0;   // this step's pivot; the previous step's pair
    for (int t = 0; t < e; ++t) {
        const int par = t & 1;
        const DsmMail mv = mail[par];
        // at least two coordinates are active at every step (e_u <= c_u - 1);
        // the clamps only keep a corrupted state from indexing out of bounds
        if (i < 0 || i >= c) i = 0;
        const int j = (mv.j >= 0 && mv.j < c && mv.j != i) ? mv.j : (i == 0 ? 1 : 0);
        const bool more = t + 1 < e;
        const int a1 = s_a[0], a2 = s_a[1];
        // ---- A
        const bool live = has_task && y != i && y != j && is_active(mask, y);
        double xa = 0.0, xb = 0.0;
        if (live) {
            xa = Xr[i];
            xb = Xr[j];
        }
        if (wid == 0 || wid == DSM_S_WARP) {
            if (lane == 0) {
                double cc, ss;
                jacobi2(gd[i], mv.g, gd[j], cc, ss);
                if (wid == 0) s_c = cc;
                else s_s = ss;
            }
        } else if (wid == DSM_W_WARP) {
            // the previous step's new weights (the eliminated one's is never
            // read again), before the partner searches read them
            if (t > 0 && lane < 2) {
                const double g = s_blk[lane];
                w[lane == 0 ? pi : pj] = g > 0.0 ? __ddiv_rn(1.0, __dsqrt_rn(g)) : 0.0;
            }
            __syncwarp();
            named_arrive(3, 32 * (1 + 2 * DSM_SCORE_WARPS));
        } else if (wid <= 2 * DSM_SCORE_WARPS) {
            named_sync(3, 32 * (1 + 2 * DSM_SCORE_WARPS));
            const int k = (wid - 1) / DSM_SCORE_WARPS;      // 0: a1, 1: a2
            const int w0 = 1 + k * DSM_SCORE_WARPS;
            const int a = k == 0 ? a1 : a2;
            const bool mine = more && a >= 0 && a < c && a != i && a != j && rank == a / R;
            if (mine) {
                dsm_score_row(Gs + (size_t)(a - row0) * c, Ms + (size_t)(a - row0) * c, w, mask, c, a, i, j,
                              w0, DSM_SCORE_WARPS, wb + w0);
                named_sync(1 + k, 32 * DSM_SCORE_WARPS);
                if (wid == w0) {
                    const Cand b = dsm_best_of(wb + w0, DSM_SCORE_WARPS);
                    if (lane == 0) spec[k] = b;
                }
            }
        }
        __syncthreads();
        const double cc = s_c, ss = s_s;
        // ---- B
        if (wid == 0 && lane < 4) {
            // the new diagonal entries of the 2 x 2 blocks: lanes 0, 1 for G
            // (a', d'), lanes 2, 3 for M; each is rot_block's chain written as
            // r1 = fma(p, a, q b), r2 = fma(p, b, q d), v = fma(r1, p, r2 q)
            // with (p, q) = (c, -s) for a' and (s, c) for d'
            const bool isM = lane >= 2;
            const double a = isM ? md[i] : gd[i], b = isM ? mv.m : mv.g, d = isM ? md[j] : gd[j];
            const double p = (lane & 1) ? ss : cc, qq = (lane & 1) ? cc : -ss;
            const double r1 = __fma_rn(p, a, __dmul_rn(qq, b));
            const double r2 = __fma_rn(p, b, __dmul_rn(qq, d));
            s_blk[lane] = __fma_rn(r1, p, __dmul_rn(r2, qq));
        }
        if (wid == 0) {
            __syncwarp();
            if (lane == 0) {
                gd[i] = s_blk[0];
                gd[j] = s_blk[1];
                md[i] = s_blk[2];
                md[j] = s_blk[3];
                const double di = __dsub_rn(gd[i], __dmul_rn(md[i], md[i]));
                const double dj = __dsub_rn(gd[j], __dmul_rn(md[j], md[j]));
                const int le = di < dj ? i : j;
                const int L = 1 + max(lvl[i], lvl[j]);
                lvl[i] = L;
                lvl[j] = L;
                s_maxlev = max(s_maxlev, L);
                if (rank == 0) rec[r0 + t] = RotRec{i, j, le, L, cc, ss};
                mask[le >> 5] &= ~(1u << (le & 31));
                s_le = le;
                s_ip = le <= a1 ? a2 : a1;
            }
        }
        if (live && !(is_zero(xa) && is_zero(xb))) {
            double na, nb;
            rot_pair(cc, ss, xa, xb, na, nb);
            Xr[i] = na;
            Xr[j] = nb;
            // the mirrored entries: rows i and j at column y
            const int oi = i / R, oj = j / R;
            cluster.map_shared_rank(Xs, oi)[(size_t)(i - oi * R) * c + y] = na;
            cluster.map_shared_rank(Xs, oj)[(size_t)(j - oj * R) * c + y] = nb;
        }
        __syncthreads();
        // ---- C
        const int le = s_le, sv = le == i ? j : i;   // eliminated, survivor
        const int ip = s_ip < 0 || s_ip >= c ? 0 : s_ip;
        if (more && ip == sv) {
            // the survivor is the next pivot: its row was rotated in every
            // CTA, so its partner is searched in full after the stores land
            cluster.sync();
            if (rank == ip / R) {
                dsm_score_row(Gs + (size_t)(ip - row0) * c, Ms + (size_t)(ip - row0) * c, w, mask, c, ip, -1, -1,
                              0, DSM_WARPS, wb);
                __syncthreads();
                if (wid == 0) {
                    const Cand b = dsm_best_of(wb, DSM_WARPS);
                    if (lane < DSM_CL) {
                        DsmMail *dst = cluster.map_shared_rank(&mail[par ^ 1], lane);
                        dst->g = b.g;
                        dst->m = b.m;
                        dst->j = b.idx;
                    }
                }
            }
        } else if (more && wid == 0 && rank == ip / R) {
            // the partner search of row ip over everything but i and j, merged
            // with the survivor's rotated entry
            Cand b = spec[ip == a1 ? 0 : 1];
            const double gv = Gs[(size_t)(ip - row0) * c + sv];
            const double mvv = Ms[(size_t)(ip - row0) * c + sv];
            const double gss = gd[sv];
            bool take;
            if (b.idx == 0x7fffffff) {
                take = true;                            // no other candidate
            } else if (is_zero(gv) || surely_below(gv, gss, b.key)) {
                take = is_zero(gv) && b.key == 0ull && sv < b.idx;   // a zero entry scores +0
            } else {
                const double ws = gss > 0.0 ? __ddiv_rn(1.0, __dsqrt_rn(gss)) : 0.0;
                const Cand cs = cand_make(gv, mvv, ws, sv);
                take = cand_better(cs.key, cs.idx, b.key, b.idx);
            }
            if (take) {
                b.idx = sv;
                b.g = gv;
                b.m = mvv;
            }
            if (lane < DSM_CL) {
                DsmMail *dst = cluster.map_shared_rank(&mail[par ^ 1], lane);
                dst->g = b.g;
                dst->m = b.m;
                dst->j = b.idx;
            }
        }
        cluster_arrive_release();
        if (wid == DSM_NEXT_WARP && lane == 0 && t + 2 < e) {
            // the two possible pivots of step t + 2
            const int64_t p = (int64_t)__umul64hi(draws[t + 2], (uint64_t)(c - t - 2));
            s_a[0] = select_bit(mask, nwords, p, -1);
            s_a[1] = select_bit(mask, nwords, p + 1, -1);
        }
        __syncwarp();
        cluster_wait_acquire();
        __syncthreads();
        pi = i;
        pj = j;
        i = ip;
    }
    if (rank == 0)
        finish_cluster(u, r0, e, s_maxlev, members, base, rec, lcnt, lvlrot, lvl_off, nlev, elimflag, stage);
}

}  // namespace

pmmf_status gram_blocks(const StageClusters &cls, GramBlocks &gb, cudaStream_t st, int64_t total) {
    const int64_t m = cls.m;
    PMMF_TRY(gb.goff.alloc(m + 1, st));
    k_square_sizes<<<grid_for(m, 256), 256, 0, st>>>(cls.coff.p, m, gb.goff.p);
    PMMF_TRY(launched("square_sizes"));
    PMMF_TRY(scan_i64(gb.goff.p, gb.goff.p, m, st));
    if (total >= 0) {
        gb.total = total;
    } else {
        PMMF_CUDA_TRY(cudaMemcpyAsync(&gb.total, gb.goff.p + m, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        PMMF_CUDA_TRY(cudaStreamSynchronize(st));
    }
    PMMF_TRY(gb.G.alloc(gb.total, st));   // the Gram kernels write every entry of every block
    PMMF_TRY(gb.M.alloc(gb.total, st));
    return PMMF_OK;
}

pmmf_status gram_and_select(const Csr &A, const int32_t *act_ids, const int32_t *pos,
                            const int32_t *cl, const int32_t *loc, const StageClusters &cls,
                            int64_t cmax, uint64_t seed, int64_t stage, StageRotations &rot,
                            int32_t *elimflag, cudaStream_t st, const int32_t *order,
                            const uint64_t *useed, unsigned *status, int64_t gram_total,
                            const int32_t *ords, int64_t nmem) {
    GramBlocks gb;
    PMMF_TRY(gram_blocks(cls, gb, st, gram_total));
    const int64_t s = A.rows;
    // the transpose of the active matrix
    DBuf<int64_t> trp, tcur, tul;
    DBuf<double> tv;
    PMMF_TRY(trp.zeros(s + 1, st));
    PMMF_TRY(tcur.alloc(s + 1, st));
    PMMF_TRY(tul.alloc(std::max<int64_t>(A.nnz, 1), st));
    PMMF_TRY(tv.alloc(std::max<int64_t>(A.nnz, 1), st));
    k_tcount<<<grid_for(A.nnz, 256), 256, 0, st>>>(A.rowptr.p, A.col.p, s, pos, trp.p);
    PMMF_TRY(launched("tcount"));
    PMMF_TRY(scan_i64_dup(trp.p, trp.p, tcur.p, s, st));
    k_tscatter<<<grid_for(s * 32, 256), 256, 0, st>>>(A.rowptr.p, A.col.p, A.val.p, s, pos,
                                                       act_ids, cl, loc, tcur.p, tul.p, tv.p);
    PMMF_TRY(launched("tscatter"));
    int warps = tuned(TUNE_GRAM_WARPS, cmax, 8);
    while (warps > 1 && sizeof(double) * (size_t)cmax * warps > 96 * 1024) warps >>= 1;
    const size_t gsh = sizeof(double) * (size_t)cmax * warps;
    PMMF_CUDA_TRY(allow_smem(k_gram_rows, gsh));
    prof_begin(KF_GRAM, st);
    k_gram_rows<<<grid_for(s * 32, 32 * warps), 32 * warps, gsh, st>>>(
        A.rowptr.p, A.col.p, A.val.p, trp.p, tul.p, tv.p, pos, cl, loc, cls.coff.p, cls.members.p,
        nmem >= 0 ? nmem : s, cmax, gb.goff.p, gb.G.p, gb.M.p);
    // compulsory traffic: the active matrix (12 B per entry) and its
    // transpose (16 B per entry) once, their row pointers, and both c_u x c_u
    // outputs
    prof_end(KF_GRAM, st, 28.0 * (double)A.nnz + 16.0 * (double)s + 16.0 * (double)gb.total, 0.0);
    PMMF_TRY(launched("gram"));
    return select_stage(cls, cmax, gb, seed, stage, rot, elimflag, st, order, useed, status, ords);
}

namespace {

// Shared memory of k_select_dsm for clusters of up to cmax coordinates.
size_t dsm_smem(int64_t cmax) {
    const size_t R = (size_t)((cmax + DSM_CL - 1) / DSM_CL);
    return sizeof(double) * (2 * R * (size_t)cmax + 3 * (size_t)cmax) + sizeof(uint64_t) * (size_t)(cmax + 1) +
           sizeof(uint32_t) * (size_t)((cmax + 31) / 32) + sizeof(int32_t) * (size_t)(2 * cmax + 2);
}

}  // namespace

pmmf_status select_stage(const StageClusters &cls, int64_t cmax, GramBlocks &gb, uint64_t seed,
                         int64_t stage, StageRotations &rot, int32_t *elimflag, cudaStream_t st,
                         const int32_t *order, const uint64_t *useed, unsigned *status,
                         const int32_t *ords) {
    const int64_t m = cls.m;
    DBuf<int64_t> &goff = gb.goff;
    DBuf<double> &G = gb.G, &M = gb.M;
    if (rot.K > 2) {
        if (!status) {
            set_error("k-point search needs a status word");
            return PMMF_ERR_INVALID_ARG;
        }
        return select_kpoint(cls, cmax, goff.p, G.p, M.p, seed, stage, rot, elimflag, st, order,
                             useed, status, ords);
    }
    PMMF_TRY(rot.rec.alloc(rot.nrot > 0 ? rot.nrot : 1, st));
    PMMF_TRY(rot.lvl.alloc(rot.nrot > 0 ? rot.nrot : 1, st));
    PMMF_TRY(rot.lvl_off.alloc(rot.nrot + m + 1, st));
    PMMF_TRY(rot.nlev.zeros(m, st));
    const size_t shb = sizeof(double) * 3 * (size_t)cmax + sizeof(uint32_t) * (size_t)((cmax + 31) / 32) +
                       sizeof(int32_t) * (size_t)(2 * cmax + 4);
    const size_t shf = shb + sizeof(uint64_t) * (size_t)(cmax + 1) + sizeof(Work) * (size_t)cmax + 16;
    // the fast kernels need shf bytes of shared memory, the generic one shb
    const bool fits_fast = shf <= 220 * 1024;
    if (shb > 220 * 1024) {
        set_error("cluster too large for the selection kernel");
        return PMMF_ERR_UNSUPPORTED;
    }
    double sel_flops = 0.0;
    if (prof_on(KF_SELECT)) {
        // per step with n_a active coordinates: n_a score products and 12 flops
        // per other active coordinate for the two rotated rows of G and M
        std::vector<int64_t> hc((size_t)m + 1), hr((size_t)m + 1);
        PMMF_CUDA_TRY(cudaMemcpyAsync(hc.data(), cls.coff.p, sizeof(int64_t) * hc.size(), cudaMemcpyDeviceToHost, st));
        PMMF_CUDA_TRY(cudaMemcpyAsync(hr.data(), rot.roff.p, sizeof(int64_t) * hr.size(), cudaMemcpyDeviceToHost, st));
        PMMF_CUDA_TRY(cudaStreamSynchronize(st));
        for (int64_t u = 0; u < m; ++u) {
            int64_t c = hc[u + 1] - hc[u], e = hr[u + 1] - hr[u];
            for (int64_t t = 0; t < e; ++t) sel_flops += 13.0 * (double)(c - t);
        }
    }
    prof_begin(KF_SELECT, st);
    // The search by thread-block clusters holding G and M in shared memory
    // (PMMF_TUNE_SELECT_DSM = 2) for stages whose clusters fit; measured on
    // GB300 it is slower than the one-CTA search on the late stages of the
    // kNN workload (clusters ~256: ~7,300 against ~7,100 cycles per step, the
    // angle's dependent FP64 chain and the per-step cluster barrier on the
    // critical path), so it runs only when asked for.
    {
        const int dsm = tuned(TUNE_SELECT_DSM, cmax, 1);
        const size_t need = dsm_smem(cmax);
        const bool fits = need <= 225 * 1024 && 2 * ((cmax + DSM_CL - 1) / DSM_CL) <= DSM_ROT_N;
        if (fits && m > 0 && m <= INT32_MAX / DSM_CL && dsm == 2) {
            PMMF_CUDA_TRY(cudaFuncSetAttribute(k_select_dsm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need));
            k_select_dsm<<<(unsigned)(m * DSM_CL), DSM_THREADS, need, st>>>(
                cls.coff.p, cls.members.p, goff.p, G.p, M.p, rot.roff.p, seed, stage, rot.rec.p, rot.lvl.p,
                rot.lvl_off.p, rot.nlev.p, elimflag, order, useed, ords);
            prof_end(KF_SELECT, st, 0.0, sel_flops);
            PMMF_TRY(launched("select"));
            return PMMF_OK;
        }
    }
    // 256 threads (128 column threads) up to 512 coordinates, 512 threads
    // (384 column threads) up to 1,536, the generic kernel beyond.  The wide
    // CTA spreads a step's loads and FP64 work over 12 column warps; measured
    // on GB300 it is slower for clusters the narrow one covers (kNN
    // Laplacians, clusters ~256: 5.1 vs 4.7 ms of search per factorization),
    // so it is used only beyond 512 coordinates unless tuned otherwise.
    const int kpt = (int)((cmax + NCT - 1) / NCT);
    const int kpt512 = (int)((cmax + 383) / 384);
    int sw = tuned(TUNE_SELECT_WARPS, cmax, 0);
    if (sw == 0) sw = 8;
    if (kpt > 4) sw = 16;
    auto launch = [&](auto kern, int nt) -> pmmf_status {
        PMMF_CUDA_TRY(allow_smem(kern, shf));
        kern<<<(unsigned)m, nt, shf, st>>>(cls.coff.p, cls.members.p, goff.p, G.p, M.p, rot.roff.p,
                                           seed, stage, rot.rec.p, rot.lvl.p, rot.lvl_off.p,
                                           rot.nlev.p, elimflag, order, useed, ords);
        return PMMF_OK;
    };
    // A stage with many more clusters than SMs is bound by throughput, not by
    // one cluster's chain: fewer registers per thread fit more CTAs per SM
    // (PMMF_TUNE_SELECT_BLOCKS: 2, 3 or 4 CTAs of 256 threads per SM).
    // Measured on GB300 (128^3 Poisson, 8,192 and 4,096 clusters of 256):
    // 4 CTAs per SM 13.2 -> 9.4 and 7.0 -> 4.9 ms per stage; the largest
    // instantiation spills at 3 per SM and gains only with thousands of
    // clusters (2,048: 3.78 -> 3.53 ms), loses on fewer (kNN stages).
    int nsm = 152;
    {
        int dev = 0;
        if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    }
    const int occ = tuned(TUNE_SELECT_BLOCKS, cmax, 0);
    const int minb = occ                         ? occ
                     : kpt <= 2 && m >= 4 * nsm ? 4
                     : kpt <= 4 && m >= 6 * nsm ? 3
                                                : 2;
    if (fits_fast && sw == 8 && kpt <= 1 && minb >= 3) PMMF_TRY(launch(k_select_fast<1, 256, 4>, 256));
    else if (fits_fast && sw == 8 && kpt <= 2 && minb == 3) PMMF_TRY(launch(k_select_fast<2, 256, 3>, 256));
    else if (fits_fast && sw == 8 && kpt <= 2 && minb == 4) PMMF_TRY(launch(k_select_fast<2, 256, 4>, 256));
    else if (fits_fast && sw == 8 && kpt <= 4 && kpt > 2 && minb >= 3) PMMF_TRY(launch(k_select_fast<4, 256, 3>, 256));
    else if (fits_fast && sw == 8 && kpt <= 1) PMMF_TRY(launch(k_select_fast<1, 256>, 256));
    else if (fits_fast && sw == 8 && kpt <= 2) PMMF_TRY(launch(k_select_fast<2, 256>, 256));
    else if (fits_fast && sw == 8 && kpt <= 4) PMMF_TRY(launch(k_select_fast<4, 256>, 256));
    else if (fits_fast && kpt512 <= 1) PMMF_TRY(launch(k_select_fast<1, 512>, 512));
    else if (fits_fast && kpt512 <= 2) PMMF_TRY(launch(k_select_fast<2, 512>, 512));
    else if (fits_fast && kpt512 <= 4) PMMF_TRY(launch(k_select_fast<4, 512>, 512));
    else {
        PMMF_CUDA_TRY(allow_smem(k_select, shb));
        k_select<<<(unsigned)m, SEL_THREADS, shb, st>>>(cls.coff.p, cls.members.p, goff.p, G.p, M.p,
                                                        rot.roff.p, seed, stage, rot.rec.p, rot.lvl.p,
                                                        rot.lvl_off.p, rot.nlev.p, elimflag, order,
                                                        useed, ords);
    }
    prof_end(KF_SELECT, st, 0.0, sel_flops);
    PMMF_TRY(launched("select"));
    return PMMF_OK;
}

}  // namespace pmmf
