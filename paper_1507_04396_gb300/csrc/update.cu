// update.cu -- the blocked update of Algorithm 1,
//     [A_p]_{u,v} <- Qbar_{p,u} [A_{p-1}]_{u,v} Qbar_{p,v}^T   for all u, v,
// computed as A_p = (A_{p-1} Q^T)^T Q^T: the stage's rotations are applied to
// every row (a row-local operation), the result is transposed, and the
// rotations are applied to every row again.  Fused into the second pass: the
// residual of the eliminated coordinates, the diagonal of H and the
// compaction of A_p to the surviving coordinates S_p.
//
// Row kernel: one warp per row.  The row's entries are grouped by cluster;
// each cluster's part is expanded into a dense vector in shared memory and the
// cluster's rotations are applied level by level (rotations of one dependency
// level touch disjoint coordinates, so lanes apply them concurrently and the
// bits equal a sequential application in step order).  A rotation whose two
// inputs are both zero leaves them zero and is skipped.  Exact zeros are
// dropped from the output.
//
// The counting passes that size the outputs run on the sparsity pattern only
// (a rotation makes both of its coordinates nonzero when either is): integer
// work, no FP64, and an upper bound of the numeric counts, which differ only
// where a value cancels to exactly zero.  For clusters of up to 1,024
// coordinates the pattern of a row segment is the union of per-coordinate
// reach sets computed once per stage; larger clusters run the level loop on
// the pattern.  Pass 1 writes W into rows of that capacity (each row's end is
// its write cursor); pass 2 writes A_p into rows of that capacity and a
// compaction copies them to their exact positions.
#include <algorithm>
#include <climits>

#include "common.cuh"
#include "rotmath.cuh"
#include "stage.cuh"

namespace pmmf {

namespace {

enum Mode { P1_COUNT = 0, P1_WRITE = 1, P2_COUNT = 2, P2_WRITE = 3 };

struct RowArgs {
    const int64_t *rp;
    const int64_t *rend;       // row ends (NULL: rp[r + 1])
    const int32_t *ci;
    const double *v;
    int64_t rows;
    const int32_t *act;        // row -> global id
    const int32_t *pos;        // global id -> row (stage start)
    const int32_t *cl, *loc;
    const int64_t *coff;
    const int64_t *roff;
    const int32_t *lvl_off, *nlev;
    const Rot2 *lvlrot;
    const RotRec *rec;         // k = 2: the rotations in step order
    int K;                     // k >= 3: tuples, blocks and level slots below
    const int32_t *kidx, *kkv, *lvlidx;
    const double *kO;
    int64_t cmax;
    int outcap;
    // per cluster member j (cluster order): its stage position (pass 1's
    // destination row) and its global id with bit 31 set when this stage
    // eliminates it (pass 2), so an emitted entry needs one load, not two
    const int32_t *mpos, *mge;
    // counting passes: reach sets (NULL: run the level loop on the pattern)
    const uint32_t *reach;
    int reach_words;           // words per coordinate (a multiple of 4)
    // pass 1
    int64_t *wcnt;             // W row counts (COUNT)
    int64_t *wcur;             // W write cursors (WRITE)
    int32_t *wcol;
    double *wval;
    const int64_t *wtotal;     // WRITE: W's entries (the scan's total) ...
    int64_t wcap;              // ... must fit the allocation, else nothing is written
    unsigned long long *wover; // and this flag is set
    // pass 2
    const int32_t *elimflag;
    int32_t stage;
    const int64_t *newrow;     // exclusive scan of surviving flags
    int64_t *ocnt;             // COUNT: output row capacities (by new row)
    const int64_t *orp;        // WRITE: row starts of capacity rowptr
    int64_t *acnt;             // WRITE: exact output row lengths (by new row)
    int32_t *ocol;
    double *oval;
    double *hdiag;
    double *contrib;
    double *contrib_cl;        // optional: per-cluster residual (indexed by cl of the row)
    unsigned *status;
    unsigned long long *maxlen;
};

// Per-warp shared memory of the row kernel: the dense local vector (cmax
// doubles, all zero between segments), its touched-position bitmask (one bit
// per local index, an even number of words), the touched positions listed in
// ascending order (cmax int32, even) and, for the output pass, the row's kept
// entries.
__host__ __device__ inline int64_t rows_mask_words(int64_t cmax) {
    const int64_t w = (cmax + 31) / 32;
    return w + (w & 1);
}
__host__ __device__ inline int64_t rows_per_warp(int64_t cmax, int64_t outcap, bool write2) {
    return cmax + rows_mask_words(cmax) / 2 + (cmax + 1) / 2 + (write2 ? outcap * 3 / 2 + 1 : 0);
}

// Row entries a lane keeps in registers (rows up to 32 * ROW_CACHE entries
// are read from global memory once; longer rows are re-read per segment).
constexpr int ROW_CACHE = 2;

// Reach sets of a stage's rotations: R_u[x] = the local coordinates of
// cluster u that a nonzero at x (before the stage) makes nonzero, i.e. those
// reachable from x through rotations taken in step order.  A rotation makes
// all of its coordinates nonzero when one is, so the pattern a row segment
// has after the cluster's rotations is the union of R_u over its entries.
// Built backwards: R[x] = {x}, then for each rotation from the last to the
// first, every coordinate of its tuple receives the union of the tuple's sets.
// One warp per cluster; lane w owns word w of every set (words never mix, so
// the lanes need no synchronisation); the sets live in shared memory.
constexpr int REACH_MAX_C = 1024;   // 32 words per set: one word per lane

__global__ void k_reach(const int64_t *coff, const int64_t *roff, const RotRec *rec, int K,
                        const int32_t *kidx, const int32_t *kkv, int words, int64_t cmax,
                        uint32_t *reach) {
    extern __shared__ uint32_t rs[];
    const int64_t u = blockIdx.x;
    const int64_t cb = coff[u];
    const int c = (int)(coff[u + 1] - cb);
    const int nw = (c + 31) / 32;
    const int lane = threadIdx.x;
    const int64_t r0 = roff[u];
    const int e = (int)(roff[u + 1] - r0);
    // the sets (stride 32 words), then the rotations' tuples (KS slots each;
    // slot K holds the tuple size for k >= 3), staged by all lanes
    const int KS = K <= 2 ? 2 : K + 1;
    int32_t *tup = (int32_t *)(rs + 32 * cmax);
    for (int t = lane; t < e; t += 32) {
        if (K <= 2) {
            const RotRec q = rec[r0 + t];
            tup[2 * t] = q.li;
            tup[2 * t + 1] = q.lj;
        } else {
            for (int z = 0; z < K; ++z) tup[t * KS + z] = kidx[(r0 + t) * K + z];
            tup[t * KS + K] = kkv[r0 + t];
        }
    }
    for (int idx = lane; idx < c * nw; idx += 32) {
        const int x = idx / nw, w = idx - x * nw;
        rs[x * 32 + w] = (x >> 5) == w ? 1u << (x & 31) : 0u;
    }
    __syncwarp();
    if (lane < nw) {
        const int w = lane;
        if (K <= 2) {
            for (int t = e - 1; t >= 0; --t) {
                const int li = tup[2 * t], lj = tup[2 * t + 1];
                const uint32_t v = rs[li * 32 + w] | rs[lj * 32 + w];
                rs[li * 32 + w] = v;
                rs[lj * 32 + w] = v;
            }
        } else {
            for (int t = e - 1; t >= 0; --t) {
                const int32_t *T = tup + t * KS;
                const int kk = T[K];
                uint32_t v = 0u;
                for (int q = 0; q < kk; ++q) v |= rs[T[q] * 32 + w];
                for (int q = 0; q < kk; ++q) rs[T[q] * 32 + w] = v;
            }
        }
    }
    __syncwarp();
    // rows of 'words' words, zero beyond the cluster's own (coalesced)
    for (int idx = lane; idx < c * words; idx += 32) {
        const int x = idx / words, w = idx - x * words;
        reach[(cb + x) * words + w] = w < nw ? rs[x * 32 + w] : 0u;
    }
}

// KP: the stage's rotations are k-point (k >= 3) blocks; the k = 2
// instantiation carries no k-point code (fewer registers, more warps).
template <int MODE, bool KP>
__global__ void __launch_bounds__(256, 4) k_rows(RowArgs a) {
    constexpr bool COUNT = MODE == P1_COUNT || MODE == P2_COUNT;
    extern __shared__ double smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    if (MODE == P1_WRITE && *a.wtotal > a.wcap) {
        if (threadIdx.x == 0 && blockIdx.x == 0) *a.wover = 1ull;
        return;
    }
    const int64_t per_warp = rows_per_warp(a.cmax, a.outcap, MODE == P2_WRITE);
    double *dense = smem + per_warp * wib;
    uint32_t *tb = (uint32_t *)(dense + a.cmax);
    const int nwmax = (int)rows_mask_words(a.cmax);
    int32_t *plist = (int32_t *)(tb + nwmax);
    int32_t *scol = plist + (a.cmax + (a.cmax & 1));
    double *sval = (double *)(scol + (a.outcap + (a.outcap & 1)));
    for (int64_t l = lane; l < a.cmax; l += 32) dense[l] = 0.0;
    for (int l = lane; l < nwmax; l += 32) tb[l] = 0u;
    __syncwarp();
    double part = 0.0;
    for (int64_t r = blockIdx.x * (int64_t)wpb + wib; r < a.rows; r += (int64_t)gridDim.x * wpb) {
        const int64_t e0 = a.rp[r], e1 = a.rend ? a.rend[r] : a.rp[r + 1];
        const int32_t y = a.act[r];
        const bool yelim = (MODE >= P2_COUNT) && a.elimflag[y] == a.stage;
        int64_t nout = 0;
        int nseg = 0;
        int prev = -1;
        double prow = 0.0;   // this row's residual terms (per-cluster accounting)
        // the row's entries (cluster, local index, value) in registers
        const bool cached = e1 - e0 <= 32 * ROW_CACHE;
        int cu[ROW_CACHE], cloc[ROW_CACHE];
        double cv[ROW_CACHE];
#pragma unroll
        for (int k = 0; k < ROW_CACHE; ++k) {
            const int64_t q = e0 + lane + 32 * k;
            cu[k] = INT_MAX;
            cloc[k] = 0;
            cv[k] = 0.0;
            if (cached && q < e1) {
                const int32_t g = a.ci[q];
                cu[k] = a.cl[g];
                cloc[k] = a.loc[g];
                if (!COUNT) cv[k] = a.v[q];
            }
        }
        for (;;) {
            int mu = INT_MAX;
            if (cached) {
#pragma unroll
                for (int k = 0; k < ROW_CACHE; ++k)
                    if (cu[k] > prev && cu[k] < mu) mu = cu[k];
            } else {
                for (int64_t q = e0 + lane; q < e1; q += 32) {
                    int uq = a.cl[a.ci[q]];
                    if (uq > prev && uq < mu) mu = uq;
                }
            }
            for (int o = 16; o > 0; o >>= 1) mu = min(mu, __shfl_xor_sync(0xffffffffu, mu, o));
            if (mu == INT_MAX) break;
            ++nseg;
            const int64_t cb = a.coff[mu];
            const int c = (int)(a.coff[mu + 1] - cb);
            const int nw = (c + 31) / 32;
            if (COUNT && a.reach) {
                // the segment's pattern after the cluster's rotations: the
                // union of its entries' reach sets
                auto add_reach = [&](int l) {
                    const uint4 *R = (const uint4 *)(a.reach + (cb + l) * a.reach_words);
                    for (int w4 = 0; 4 * w4 < nw; ++w4) {
                        const uint4 v = __ldg(R + w4);
                        const uint32_t vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                        for (int z = 0; z < 4; ++z)
                            if (4 * w4 + z < nw && vv[z]) atomicOr(&tb[4 * w4 + z], vv[z]);
                    }
                };
                if (cached) {
#pragma unroll
                    for (int k = 0; k < ROW_CACHE; ++k)
                        if (cu[k] == mu) add_reach(cloc[k]);
                } else {
                    for (int64_t q = e0 + lane; q < e1; q += 32) {
                        const int32_t g = a.ci[q];
                        if (a.cl[g] == mu) add_reach(a.loc[g]);
                    }
                }
            } else if (cached) {
#pragma unroll
                for (int k = 0; k < ROW_CACHE; ++k)
                    if (cu[k] == mu) {
                        const int l = cloc[k];
                        if (!COUNT) dense[l] = cv[k];
                        atomicOr(&tb[l >> 5], 1u << (l & 31));
                    }
            } else {
                for (int64_t q = e0 + lane; q < e1; q += 32) {
                    int32_t g = a.ci[q];
                    if (a.cl[g] == mu) {
                        const int l = a.loc[g];
                        if (!COUNT) dense[l] = a.v[q];
                        atomicOr(&tb[l >> 5], 1u << (l & 31));
                    }
                }
            }
            __syncwarp();
            const int32_t *lo = a.lvl_off + a.roff[mu] + mu;
            const int nl = (COUNT && a.reach) ? 0 : a.nlev[mu];
            if (!KP) {
                // level offsets in registers (lane L holds lo[L]) and the first
                // 32 rotations of the next level loaded while this one runs
                const int lol = lane <= nl ? lo[lane] : 0;
                // lo[L] for a warp-uniform L
                auto level_start = [&](int L) {
                    const int v = __shfl_sync(0xffffffffu, lol, L & 31);
                    return L < 32 ? v : lo[L];
                };
                int b0 = level_start(0);
                int b1 = level_start(1);
                Rot2 cur = Rot2{0, 0, 1.0, 0.0};
                if (nl > 0 && b0 + lane < b1) cur = a.lvlrot[b0 + lane];
                for (int L = 0; L < nl; ++L) {
                    const int c0 = b0, c1 = b1;
                    if (L + 1 < nl) {
                        b0 = c1;
                        b1 = level_start(L + 2);
                    }
                    Rot2 nxt = Rot2{0, 0, 1.0, 0.0};
                    if (L + 1 < nl && b0 + lane < b1) nxt = a.lvlrot[b0 + lane];
                    for (int idx = c0 + lane; idx < c1; idx += 32) {
                        const Rot2 q = idx == c0 + lane ? cur : a.lvlrot[idx];
                        if (COUNT) {
                            // pattern only: both coordinates nonzero if either is
                            const bool bi = (tb[q.li >> 5] >> (q.li & 31)) & 1u;
                            const bool bj = (tb[q.lj >> 5] >> (q.lj & 31)) & 1u;
                            if (bi != bj) {
                                atomicOr(&tb[q.li >> 5], 1u << (q.li & 31));
                                atomicOr(&tb[q.lj >> 5], 1u << (q.lj & 31));
                            }
                            continue;
                        }
                        double vi = dense[q.li], vj = dense[q.lj];
                        if (nonzero_bits(vi) || nonzero_bits(vj)) {
                            double ni, nj;
                            rot_pair(q.c, q.s, vi, vj, ni, nj);
                            dense[q.li] = ni;
                            dense[q.lj] = nj;
                            atomicOr(&tb[q.li >> 5], 1u << (q.li & 31));
                            atomicOr(&tb[q.lj >> 5], 1u << (q.lj & 31));
                        }
                    }
                    __syncwarp();
                    cur = nxt;
                }
            } else {
            for (int L = 0; L < nl; ++L) {
                {
                    for (int idx = lo[L] + lane; idx < lo[L + 1]; idx += 32) {
                        const int64_t t = a.lvlidx[idx];
                        const int kk = a.kkv[t];
                        const int32_t *T = a.kidx + t * a.K;
                        if (COUNT) {
                            bool any = false;
                            for (int q = 0; q < kk; ++q) any |= (tb[T[q] >> 5] >> (T[q] & 31)) & 1u;
                            if (any)
                                for (int q = 0; q < kk; ++q) atomicOr(&tb[T[q] >> 5], 1u << (T[q] & 31));
                            continue;
                        }
                        double in[8];
                        bool nz = false;
                        for (int q = 0; q < kk; ++q) {
                            in[q] = dense[T[q]];
                            nz |= nonzero_bits(in[q]);
                        }
                        if (nz) {
                            const double *O = a.kO + t * a.K * a.K;
                            double out[8];
                            for (int q = 0; q < kk; ++q) out[q] = rot_row(O, kk, q, in);
                            for (int q = 0; q < kk; ++q) {
                                dense[T[q]] = out[q];
                                atomicOr(&tb[T[q] >> 5], 1u << (T[q] & 31));
                            }
                        }
                    }
                }
                __syncwarp();
            }
            }
            // emit: list the touched positions in ascending order (lane =
            // word) and reset the mask, then one lane per position, so the
            // dependent loads and atomics of 32 positions overlap
            int ntouch = 0;
            for (int w0 = 0; w0 < nw; w0 += 32) {
                const int wi = w0 + lane;
                const uint32_t bits = wi < nw ? tb[wi] : 0u;
                if (wi < nw) tb[wi] = 0u;
                const int cntw = __popc(bits);
                int inc = cntw;   // inclusive scan over lanes
                for (int o = 1; o < 32; o <<= 1) {
                    const int t2 = __shfl_up_sync(0xffffffffu, inc, o);
                    if (lane >= o) inc += t2;
                }
                int off = ntouch + inc - cntw;
                for (uint32_t m = bits; m; m &= m - 1) plist[off++] = wi * 32 + __ffs(m) - 1;
                ntouch += __shfl_sync(0xffffffffu, inc, 31);
            }
            __syncwarp();
            for (int k0 = 0; k0 < ntouch; k0 += 32) {
                const int k = k0 + lane;
                const int l = k < ntouch ? plist[k] : 0;
                double x = 0.0;
                bool nz = k < ntouch;
                if (!COUNT && nz) {
                    x = dense[l];
                    dense[l] = 0.0;
                    nz = nonzero_bits(x);
                }
                if (MODE == P1_COUNT) {
                    if (nz) atomicAdd((unsigned long long *)&a.wcnt[a.mpos[cb + l]], 1ull);
                } else if (MODE == P1_WRITE) {
                    if (nz) {
                        const int64_t slot =
                            (int64_t)atomicAdd((unsigned long long *)&a.wcur[a.mpos[cb + l]], 1ull);
                        a.wcol[slot] = y;
                        a.wval[slot] = x;
                    }
                } else {
                    const int32_t mg = nz ? a.mge[cb + l] : 0;
                    const int32_t g = mg & 0x7fffffff;
                    bool keep = false;
                    if (nz) {
                        bool term = false;
                        if (yelim) {
                            if (g == y) {
                                if (MODE == P2_WRITE) a.hdiag[y] = x;
                            } else {
                                term = true;
                            }
                        } else if (mg < 0) {
                            term = true;
                        } else {
                            keep = true;
                        }
                        if (MODE == P2_WRITE && term) {
                            if (a.contrib_cl) prow = __fma_rn(x, x, prow);
                            else part = __fma_rn(x, x, part);
                        }
                    }
                    // kept entries in ascending position order
                    const unsigned kb = __ballot_sync(0xffffffffu, keep);
                    if (MODE == P2_WRITE && keep) {
                        const int64_t slot = nout + __popc(kb & ((1u << lane) - 1u));
                        if (slot < a.outcap) {
                            scol[slot] = g;
                            sval[slot] = x;
                        }
                    }
                    nout += __popc(kb);
                }
            }
            __syncwarp();
            prev = mu;
        }
        if (MODE == P2_WRITE && a.contrib_cl) {
            prow = warp_sum(prow);
            if (lane == 0 && prow != 0.0) atomicAdd(a.contrib_cl + a.cl[y], prow);
        }
        if (MODE == P2_COUNT && !yelim && lane == 0) {
            a.ocnt[a.newrow[r]] = nout;
            atomicMax(a.maxlen, (unsigned long long)nout);
        }
        if (MODE == P2_WRITE && !yelim) {
            if (lane == 0) a.acnt[a.newrow[r]] = nout;
            if (nout > a.outcap) {
                if (lane == 0) atomicOr(a.status, ST_ROW_TOO_LONG);
            } else {
                __syncwarp();
                const int64_t ob = a.orp[a.newrow[r]];
                const int n = (int)nout;
                // entries of one cluster segment are already ascending; a single
                // segment needs no reordering, several are ranked by key
                for (int q = lane; q < n; q += 32) {
                    int32_t g = scol[q];
                    int rank = q;
                    if (nseg > 1) {
                        rank = 0;
                        for (int z = 0; z < n; ++z) rank += scol[z] < g;
                    }
                    a.ocol[ob + rank] = g;
                    a.oval[ob + rank] = sval[q];
                }
                __syncwarp();
            }
        }
    }
    if (MODE == P2_WRITE) {
        part = warp_sum(part);
        if (lane == 0 && part != 0.0) atomicAdd(a.contrib, part);
    }
}

// ---------------------------------------------------------------- thread-per-row update
//
// The same four passes with one thread per row instead of one warp.  A row
// segment (the row's entries in one cluster) needs only the few rotations of
// its cluster that touch its growing pattern (4 to 10 of ~c/2 on the sparse
// workloads), so the thread applies exactly those, in step order: every
// pattern coordinate carries its position in its incidence list (the steps of
// the rotations it belongs to, ascending), the next rotation is the smallest
// step among them, and a coordinate a rotation reaches joins the pattern with
// value 0.  Applying the rotations of one segment in step order and skipping
// only rotations whose inputs are all zero is what the warp kernel (and the
// oracle's dense vector) computes, bit for bit; the FP64 instructions of a
// warp now carry up to 32 rows' rotations instead of a few lanes of one row.
// The counting passes take each segment's pattern from the reach sets.
//
// A thread's pattern lives in LANE_PS slots in shared memory (slot-major, so a
// warp's threads touch distinct banks) and, beyond them, in its own region of
// a global scratch buffer (cmax - LANE_PS slots), so no segment overflows:
// a pattern never leaves its cluster.
constexpr int LANE_NT = 128;                 // threads per CTA
constexpr int LANE_PS = 32;                  // pattern slots per thread in shared memory
constexpr int LANE_CTAS_PER_SM = 3;          // 64 KB of slots per CTA
constexpr int LANE_MAX_C = 1024;             // cluster sizes the thread path takes
constexpr uint32_t INC_END = 0xffffu;        // end of an incidence list (a step never reaches it)
constexpr size_t LANE_SMEM = (sizeof(uint2) + sizeof(double)) * LANE_PS * LANE_NT;   // 64 KB

struct LaneArgs {
    const int32_t *inc_off;    // s + 1, by cluster member position coff[u] + l
    const uint16_t *inc;       // each member's steps, ascending, then INC_END
    uint2 *ometa;              // overflow slots, ovf per thread
    double *oval;
    int ovf;
};

// Incidence lists, pass 1: every member's list length (its rotations plus the
// end marker).  One CTA per cluster.
__global__ void k_inc_count(const int64_t *coff, const int64_t *roff, const RotRec *rec, int K,
                            const int32_t *kidx, const int32_t *kkv, int64_t *cnt) {
    const int64_t u = blockIdx.x;
    const int64_t cb = coff[u];
    const int c = (int)(coff[u + 1] - cb);
    const int64_t r0 = roff[u];
    const int e = (int)(roff[u + 1] - r0);
    for (int l = threadIdx.x; l < c; l += blockDim.x) atomicAdd((unsigned long long *)&cnt[cb + l], 1ull);
    for (int t = threadIdx.x; t < e; t += blockDim.x) {
        if (K <= 2) {
            const RotRec q = rec[r0 + t];
            atomicAdd((unsigned long long *)&cnt[cb + q.li], 1ull);
            atomicAdd((unsigned long long *)&cnt[cb + q.lj], 1ull);
        } else {
            const int kk = kkv[r0 + t];
            for (int z = 0; z < kk; ++z)
                atomicAdd((unsigned long long *)&cnt[cb + kidx[(r0 + t) * K + z]], 1ull);
        }
    }
}

// Pass 2: the steps, in any order (cursor per member), as 16-bit steps.
__global__ void k_inc_fill(const int64_t *coff, const int64_t *roff, const RotRec *rec, int K,
                           const int32_t *kidx, const int32_t *kkv, int64_t *cur, uint16_t *inc) {
    const int64_t u = blockIdx.x;
    const int64_t cb = coff[u];
    const int64_t r0 = roff[u];
    const int e = (int)(roff[u + 1] - r0);
    for (int t = threadIdx.x; t < e; t += blockDim.x) {
        if (K <= 2) {
            const RotRec q = rec[r0 + t];
            inc[atomicAdd((unsigned long long *)&cur[cb + q.li], 1ull)] = (uint16_t)t;
            inc[atomicAdd((unsigned long long *)&cur[cb + q.lj], 1ull)] = (uint16_t)t;
        } else {
            const int kk = kkv[r0 + t];
            for (int z = 0; z < kk; ++z)
                inc[atomicAdd((unsigned long long *)&cur[cb + kidx[(r0 + t) * K + z]], 1ull)] =
                    (uint16_t)t;
        }
    }
}

// Pass 3: each list sorted ascending (they are short) and ended by INC_END;
// the offsets narrowed to int32.
__global__ void k_inc_finish(const int64_t *off64, int64_t s, uint16_t *inc, int32_t *off32) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j <= s;
         j += (int64_t)gridDim.x * blockDim.x) {
        off32[j] = (int32_t)off64[j];
        if (j == s) continue;
        const int64_t b = off64[j], n = off64[j + 1] - b - 1;   // the last slot is the end marker
        for (int64_t x = 1; x < n; ++x) {
            const uint16_t v = inc[b + x];
            int64_t y = x - 1;
            while (y >= 0 && inc[b + y] > v) {
                inc[b + y + 1] = inc[b + y];
                --y;
            }
            inc[b + y + 1] = v;
        }
        inc[b + n] = (uint16_t)INC_END;
    }
}

// A pattern slot: .x = next step << 16 | local index, .y = position in the
// member's incidence list of that next step.
__device__ __forceinline__ uint32_t slot_loc(uint2 m) { return m.x & 0xffffu; }
__device__ __forceinline__ uint32_t slot_next(uint2 m) { return m.x >> 16; }

template <int MODE, bool KP>
__global__ void __launch_bounds__(LANE_NT) k_rows_lane(RowArgs a, LaneArgs b) {
    constexpr bool COUNT = MODE == P1_COUNT || MODE == P2_COUNT;
    // LANE_SMEM bytes of dynamic shared memory: the slots' metadata, then values
    extern __shared__ __align__(16) unsigned char lane_sh[];
    uint2 *smeta = (uint2 *)lane_sh;
    double *sval = (double *)(lane_sh + sizeof(uint2) * LANE_PS * LANE_NT);
    const int tid = threadIdx.x;
    const int64_t gt = blockIdx.x * (int64_t)LANE_NT + tid;
    const int64_t gs = (int64_t)gridDim.x * LANE_NT;
    if (MODE == P1_WRITE && *a.wtotal > a.wcap) {
        if (gt == 0) *a.wover = 1ull;
        return;
    }
    uint2 *gmeta = b.ometa + gt * (int64_t)b.ovf;
    double *gval = b.oval + gt * (int64_t)b.ovf;
    auto meta = [&](int k) -> uint2 & { return k < LANE_PS ? smeta[k * LANE_NT + tid] : gmeta[k - LANE_PS]; };
    auto val = [&](int k) -> double & { return k < LANE_PS ? sval[k * LANE_NT + tid] : gval[k - LANE_PS]; };
    double part = 0.0;
    for (int64_t r = gt; r < a.rows; r += gs) {
        const int64_t e0 = a.rp[r], e1 = a.rend ? a.rend[r] : a.rp[r + 1];
        const int32_t y = a.act[r];
        const bool yelim = (MODE >= P2_COUNT) && a.elimflag[y] == a.stage;
        int64_t nout = 0;
        int64_t ob = 0, ocap = 0;     // the output row's capacity slots
        if (MODE == P2_WRITE && !yelim) {
            ob = a.orp[a.newrow[r]];
            ocap = a.orp[a.newrow[r] + 1] - ob;
        }
        double prow = 0.0;
        int prev = -1;
        for (;;) {
            // the next cluster segment of the row (ascending cluster ordinal)
            int mu = INT_MAX;
            for (int64_t q = e0; q < e1; ++q) {
                const int uq = a.cl[a.ci[q]];
                if (uq > prev && uq < mu) mu = uq;
            }
            if (mu == INT_MAX) break;
            prev = mu;
            const int64_t cb = a.coff[mu];
            // the segment's entries: local index, value, first incidence
            int np = 0;
            for (int64_t q = e0; q < e1; ++q) {
                const int32_t g = a.ci[q];
                if (a.cl[g] != mu) continue;
                const uint32_t l = (uint32_t)a.loc[g];
                if (COUNT) {
                    meta(np) = make_uint2(l, 0u);
                } else {
                    const int32_t p = b.inc_off[cb + l];
                    meta(np) = make_uint2(((uint32_t)b.inc[p] << 16) | l, (uint32_t)p);
                    val(np) = a.v[q];
                }
                ++np;
            }
            if (COUNT) {
                // the pattern after the cluster's rotations: union of the
                // entries' reach sets, one word at a time
                const int c = (int)(a.coff[mu + 1] - cb);
                const int nw = (c + 31) / 32;
                for (int w = 0; w < nw; ++w) {
                    uint32_t f = 0u;
                    for (int k = 0; k < np; ++k)
                        f |= __ldg(a.reach + (cb + slot_loc(meta(k))) * a.reach_words + w);
                    for (; f; f &= f - 1u) {
                        const int z = w * 32 + __ffs(f) - 1;
                        if (MODE == P1_COUNT) {
                            atomicAdd((unsigned long long *)&a.wcnt[a.mpos[cb + z]], 1ull);
                        } else if (!yelim && a.mge[cb + z] >= 0) {
                            ++nout;
                        }
                    }
                }
                continue;
            }
            const int64_t r0 = a.roff[mu];
            auto find = [&](uint32_t l) -> int {
                for (int k = 0; k < np; ++k)
                    if (slot_loc(meta(k)) == l) return k;
                return -1;
            };
            // a coordinate reached by the rotation at step t joins with value 0
            auto join = [&](uint32_t l, uint32_t t) -> int {
                int32_t p = b.inc_off[cb + l];
                while (b.inc[p] != t && b.inc[p] != (uint16_t)INC_END) ++p;
                const int k = np++;
                meta(k) = make_uint2((t << 16) | l, (uint32_t)p);
                val(k) = 0.0;
                return k;
            };
            // past step t (a slot at its end marker stays there, so the read
            // never leaves the incidence array)
            auto advance = [&](int k) {
                const uint2 m = meta(k);
                const uint32_t p = b.inc[m.y] == (uint16_t)INC_END ? m.y : m.y + 1u;
                meta(k) = make_uint2(((uint32_t)b.inc[p] << 16) | slot_loc(m), p);
            };
            for (;;) {
                uint32_t t = INC_END;
                for (int k = 0; k < np; ++k) t = min(t, slot_next(meta(k)));
                if (t == INC_END) break;
                if (!KP) {
                    const RotRec q = a.rec[r0 + t];
                    int ka = find((uint32_t)q.li), kb = find((uint32_t)q.lj);
                    if (ka < 0) ka = join((uint32_t)q.li, t);
                    if (kb < 0) kb = join((uint32_t)q.lj, t);
                    const double vi = val(ka), vj = val(kb);
                    if (nonzero_bits(vi) || nonzero_bits(vj)) {
                        double ni, nj;
                        rot_pair(q.c, q.s, vi, vj, ni, nj);
                        val(ka) = ni;
                        val(kb) = nj;
                    }
                    advance(ka);
                    advance(kb);
                } else {
                    const int64_t tg = r0 + t;
                    const int kk = a.kkv[tg];
                    const int32_t *T = a.kidx + tg * a.K;
                    int ks[8];
                    double in[8];
                    bool nz = false;
                    for (int z = 0; z < kk; ++z) {
                        int k = find((uint32_t)T[z]);
                        if (k < 0) k = join((uint32_t)T[z], t);
                        ks[z] = k;
                        in[z] = val(k);
                        nz |= nonzero_bits(in[z]);
                    }
                    if (nz) {
                        const double *O = a.kO + tg * a.K * a.K;
                        for (int z = 0; z < kk; ++z) val(ks[z]) = rot_row(O, kk, z, in);
                    }
                    for (int z = 0; z < kk; ++z) advance(ks[z]);
                }
            }
            // emit the segment's nonzero entries
            for (int k = 0; k < np; ++k) {
                const double x = val(k);
                if (!nonzero_bits(x)) continue;
                const uint32_t l = slot_loc(meta(k));
                if (MODE == P1_WRITE) {
                    const int64_t slot =
                        (int64_t)atomicAdd((unsigned long long *)&a.wcur[a.mpos[cb + l]], 1ull);
                    a.wcol[slot] = y;
                    a.wval[slot] = x;
                } else {
                    const int32_t mg = a.mge[cb + l];
                    const int32_t g = mg & 0x7fffffff;
                    bool term = false;
                    if (yelim) {
                        if (g == y) a.hdiag[y] = x;
                        else term = true;
                    } else if (mg < 0) {
                        term = true;
                    } else {
                        if (nout < ocap) {
                            a.ocol[ob + nout] = g;
                            a.oval[ob + nout] = x;
                        }
                        ++nout;
                    }
                    if (term) {
                        if (a.contrib_cl) prow = __fma_rn(x, x, prow);
                        else part = __fma_rn(x, x, part);
                    }
                }
            }
        }
        if (MODE == P2_COUNT && !yelim) {
            a.ocnt[a.newrow[r]] = nout;
            atomicMax(a.maxlen, (unsigned long long)nout);
        }
        if (MODE == P2_WRITE) {
            if (a.contrib_cl && prow != 0.0) atomicAdd(a.contrib_cl + a.cl[y], prow);
            if (!yelim) {
                a.acnt[a.newrow[r]] = nout;
                if (nout > ocap) {
                    atomicOr(a.status, ST_ROW_TOO_LONG);
                } else {
                    // the row's kept entries by ascending global id (short rows:
                    // insertion sort in place)
                    for (int64_t x = 1; x < nout; ++x) {
                        const int32_t g = a.ocol[ob + x];
                        const double v = a.oval[ob + x];
                        int64_t z = x - 1;
                        while (z >= 0 && a.ocol[ob + z] > g) {
                            a.ocol[ob + z + 1] = a.ocol[ob + z];
                            a.oval[ob + z + 1] = a.oval[ob + z];
                            --z;
                        }
                        a.ocol[ob + z + 1] = g;
                        a.oval[ob + z + 1] = v;
                    }
                }
            }
        }
    }
    if (MODE == P2_WRITE) {
        part = warp_sum(part);
        if ((tid & 31) == 0 && part != 0.0) atomicAdd(a.contrib, part);
    }
}

// Member maps of a stage (see RowArgs::mpos, mge).
__global__ void k_member_maps(const int32_t *members, int64_t s, const int32_t *pos,
                              const int32_t *elimflag, int32_t stage, int32_t *mpos, int32_t *mge) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < s;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int32_t g = members[j];
        mpos[j] = pos[g];
        mge[j] = elimflag[g] == stage ? (int32_t)((uint32_t)g | 0x80000000u) : g;
    }
}

// mge of RowArgs alone (the row passes that need no destination positions).
__global__ void k_member_ge(const int32_t *members, int64_t s, const int32_t *elimflag,
                            int32_t stage, int32_t *mge) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < s;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int32_t g = members[j];
        mge[j] = elimflag[g] == stage ? (int32_t)((uint32_t)g | 0x80000000u) : g;
    }
}

__global__ void k_survivors(const int32_t *act, int64_t s, const int32_t *elimflag, int32_t stage,
                            int32_t *flag) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < s;
         r += (int64_t)gridDim.x * blockDim.x)
        flag[r] = elimflag[act[r]] == stage ? 0 : 1;
}

// A_p's rows from their capacity slots to their exact positions (warp per row).
__global__ void k_compact_rows(const int64_t *caprp, const int64_t *rp, int64_t rows,
                               const int32_t *icol, const double *ival, int32_t *ocol,
                               double *oval) {
    const int lane = threadIdx.x & 31;
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = w; r < rows; r += nw) {
        const int64_t src = caprp[r], dst = rp[r], cnt = rp[r + 1] - dst;
        for (int64_t q = lane; q < cnt; q += 32) {
            ocol[dst + q] = icol[src + q];
            oval[dst + q] = ival[src + q];
        }
    }
}

__global__ void k_compact_act(const int32_t *act, int64_t s, const int32_t *flag,
                              const int64_t *newrow, int32_t *nact) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < s;
         r += (int64_t)gridDim.x * blockDim.x)
        if (flag[r]) nact[newrow[r]] = act[r];
}

__global__ void k_set_pos(const int32_t *act, int64_t s, int32_t *pos) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < s;
         r += (int64_t)gridDim.x * blockDim.x)
        pos[act[r]] = (int32_t)r;
}

__global__ void k_core(const int64_t *rp, const int32_t *ci, const double *v, int64_t s,
                       const int32_t *pos, const int32_t *act, double *core, double *hdiag) {
    int lane = threadIdx.x & 31;
    int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = w; r < s; r += nw) {
        for (int64_t q = rp[r] + lane; q < rp[r + 1]; q += 32) {
            int64_t b = pos[ci[q]];
            core[r * s + b] = v[q];
            if (b == r) hdiag[act[r]] = v[q];
        }
    }
}

int sm_count() {
    static int n = 0;
    if (n == 0) {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
            n = v;
        else
            n = 152;
    }
    return n;
}

// CTAs of the thread-per-row kernel: LANE_CTAS_PER_SM per SM at most (its
// shared memory), fewer for small stages.
unsigned lane_grid(int64_t rows) {
    const int64_t full = (int64_t)sm_count() * LANE_CTAS_PER_SM;
    const int64_t need = (rows + LANE_NT - 1) / LANE_NT;
    return (unsigned)std::max<int64_t>(1, std::min(full, need));
}

template <int MODE>
pmmf_status launch_rows(RowArgs &a, int64_t nnz_in, int64_t nnz_out, cudaStream_t st,
                        const LaneArgs *lb = nullptr) {
    if (lb) {
        auto kern = a.K > 2 ? k_rows_lane<MODE, true> : k_rows_lane<MODE, false>;
        PMMF_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)LANE_SMEM));
        prof_begin(KF_ROWS, st);
        kern<<<lane_grid(a.rows), LANE_NT, LANE_SMEM, st>>>(a, *lb);
        double bytes = 12.0 * (double)nnz_in + 8.0 * (double)(a.rows + 1);
        if (MODE == P1_WRITE || MODE == P2_WRITE) bytes += 12.0 * (double)nnz_out;
        prof_end(KF_ROWS, st, bytes, 0.0);
        return launched("rows_lane");
    }
    const int64_t per_warp = rows_per_warp(a.cmax, a.outcap, MODE == P2_WRITE);
    size_t per = sizeof(double) * (size_t)per_warp;
    int warps = tuned(TUNE_ROWS_WARPS, a.cmax, 8);
    while (warps > 1 && per * warps > 200 * 1024) warps >>= 1;
    if (per * warps > 220 * 1024) {
        set_error("row transform: cluster or output row too large for shared memory");
        return PMMF_ERR_UNSUPPORTED;
    }
    size_t sh = per * warps;
    auto kern = a.K > 2 ? k_rows<MODE, true> : k_rows<MODE, false>;
    PMMF_CUDA_TRY(allow_smem(kern, sh));
    unsigned grid = grid_for(a.rows, warps, 152 * 16);
    prof_begin(KF_ROWS, st);
    kern<<<grid, 32 * warps, sh, st>>>(a);
    // input rows (12 B per entry, 8 B per row pointer) plus written entries
    double bytes = 12.0 * (double)nnz_in + 8.0 * (double)(a.rows + 1);
    if (MODE == P1_WRITE || MODE == P2_WRITE) bytes += 12.0 * (double)nnz_out;
    prof_end(KF_ROWS, st, bytes, 0.0);
    return launched("rows");
}

// Pass 2's capacity, its longest row, W's exact size and pass 1's overflow
// flag, gathered for one readback.
__global__ void k_pass2_sizes(const int64_t *cap, const unsigned long long *maxlen,
                              const int64_t *wsize, const unsigned long long *wover, int64_t *out) {
    if (threadIdx.x == 0) {
        out[0] = *cap;
        out[1] = (int64_t)*maxlen;
        out[2] = *wsize;
        out[3] = (int64_t)*wover;
    }
}

}  // namespace

pmmf_status set_positions(const int32_t *act, int64_t s, int32_t *pos, cudaStream_t st) {
    if (s <= 0) return PMMF_OK;
    k_set_pos<<<grid_for(s, 256), 256, 0, st>>>(act, s, pos);
    return launched("set_pos");
}

pmmf_status survivors_stage(const int32_t *act, int64_t s, int64_t nrot, const int32_t *elimflag,
                            int64_t stage, Survivors &sv, cudaStream_t st) {
    PMMF_TRY(sv.flag.alloc(s, st));
    PMMF_TRY(sv.newrow.alloc(s + 1, st));
    sv.count = s - nrot;
    PMMF_TRY(sv.act.alloc(sv.count, st));
    if (s <= 0) return PMMF_OK;
    k_survivors<<<grid_for(s, 256), 256, 0, st>>>(act, s, elimflag, (int32_t)stage, sv.flag.p);
    PMMF_TRY(launched("survivors"));
    PMMF_TRY(scan_i32_to_i64(sv.flag.p, sv.newrow.p, s, st));
    k_compact_act<<<grid_for(s, 256), 256, 0, st>>>(act, s, sv.flag.p, sv.newrow.p, sv.act.p);
    return launched("compact_act");
}

pmmf_status update_stage(const Csr &A, const int32_t *act, int64_t n, const int32_t *pos,
                         const int32_t *cl, const int32_t *loc, const StageClusters &cls,
                         int64_t cmax, const StageRotations &rot, const int32_t *elimflag,
                         int64_t stage, const Survivors &sv, double *hdiag, double *contrib,
                         UpdateOut &out, unsigned *status, cudaStream_t st, double *contrib_cl) {
    (void)n;
    const int64_t s = A.rows;
    RowArgs a{};
    a.act = act;
    a.pos = pos;
    a.cl = cl;
    a.loc = loc;
    a.coff = cls.coff.p;
    a.roff = rot.roff.p;
    a.lvl_off = rot.lvl_off.p;
    a.nlev = rot.nlev.p;
    a.lvlrot = rot.lvl.p;
    a.rec = rot.rec.p;
    a.K = rot.K;
    a.kidx = rot.kidx.p;
    a.kkv = rot.kk.p;
    a.lvlidx = rot.lvlidx.p;
    a.kO = rot.kO.p;
    a.cmax = cmax;
    a.elimflag = elimflag;
    a.stage = (int32_t)stage;
    a.status = status;
    a.contrib = contrib;
    a.contrib_cl = contrib_cl;
    a.hdiag = hdiag;

    DBuf<int32_t> mpos, mge;
    PMMF_TRY(mpos.alloc(std::max<int64_t>(s, 1), st));
    PMMF_TRY(mge.alloc(std::max<int64_t>(s, 1), st));
    if (s > 0) {
        k_member_maps<<<grid_for(s, 256), 256, 0, st>>>(cls.members.p, s, pos, elimflag,
                                                        (int32_t)stage, mpos.p, mge.p);
        PMMF_TRY(launched("member_maps"));
    }
    a.mpos = mpos.p;
    a.mge = mge.p;

    // thread-per-row passes (clusters of up to LANE_MAX_C) when the tuning
    // knob PMMF_TUNE_ROWS_KERNEL asks for them (2); the warp-per-row kernel is
    // the default: measured on GB300 it is faster on every workload here (a
    // thread's dependent loads of its row are serialized, and the threads of
    // a warp diverge across segments and rows)
    const bool lane = s > 0 && cmax <= LANE_MAX_C && cmax <= REACH_MAX_C &&
                      tuned(TUNE_ROWS_KERNEL, cmax, 1) == 2;
    // the counting passes take the fill pattern from the reach sets when the
    // stage has enough clusters to amortise building them (one warp per
    // cluster walks its rotations, ~10-20 us whatever the stage's size), and
    // always on the thread-per-row path
    DBuf<uint32_t> reach;
    if (cmax <= REACH_MAX_C && s > 0 && (lane || cls.m >= tuned(TUNE_REACH_CLUSTERS, 1, 64))) {
        const int words = (int)((rows_mask_words(cmax) + 3) / 4 * 4);
        PMMF_TRY(reach.alloc(s * words, st));
        // sets (32 words per coordinate) and tuples (at most cmax rotations)
        const int KS = rot.K <= 2 ? 2 : rot.K + 1;
        const size_t sh = sizeof(uint32_t) * (32 + (size_t)KS) * (size_t)cmax;
        PMMF_CUDA_TRY(allow_smem(k_reach, sh));
        k_reach<<<(unsigned)cls.m, 32, sh, st>>>(cls.coff.p, rot.roff.p, rot.rec.p, rot.K, rot.kidx.p,
                                                 rot.kk.p, words, cmax, reach.p);
        PMMF_TRY(launched("reach"));
        a.reach = reach.p;
        a.reach_words = words;
    }

    // incidence lists and the threads' overflow slots of the thread-per-row path
    LaneArgs lb{};
    DBuf<int64_t> inc_cnt, inc_cur;
    DBuf<int32_t> inc_off;
    DBuf<uint16_t> inc;
    DBuf<uint2> ometa;
    DBuf<double> oval;
    if (lane) {
        PMMF_TRY(inc_cnt.zeros(s + 1, st));
        PMMF_TRY(inc_cur.alloc(s + 1, st));
        k_inc_count<<<(unsigned)cls.m, 128, 0, st>>>(cls.coff.p, rot.roff.p, rot.rec.p, rot.K,
                                                     rot.kidx.p, rot.kk.p, inc_cnt.p);
        PMMF_TRY(launched("inc_count"));
        PMMF_TRY(scan_i64_dup(inc_cnt.p, inc_cnt.p, inc_cur.p, s, st));
        // at most K entries per rotation plus one end marker per member
        const int64_t inc_cap = (int64_t)std::max(rot.K, 2) * rot.nrot + s;
        if (inc_cap >= INT32_MAX) {
            set_error("blocked update: incidence lists exceed 2^31 entries");
            return PMMF_ERR_UNSUPPORTED;
        }
        PMMF_TRY(inc.alloc(inc_cap, st));
        PMMF_TRY(inc_off.alloc(s + 1, st));
        k_inc_fill<<<(unsigned)cls.m, 128, 0, st>>>(cls.coff.p, rot.roff.p, rot.rec.p, rot.K,
                                                    rot.kidx.p, rot.kk.p, inc_cur.p, inc.p);
        PMMF_TRY(launched("inc_fill"));
        k_inc_finish<<<grid_for(s + 1, 256), 256, 0, st>>>(inc_cnt.p, s, inc.p, inc_off.p);
        PMMF_TRY(launched("inc_finish"));
        lb.inc_off = inc_off.p;
        lb.inc = inc.p;
        lb.ovf = (int)std::max<int64_t>(0, cmax - LANE_PS);
        if (lb.ovf > 0) {
            const int64_t threads = (int64_t)lane_grid(s) * LANE_NT;
            PMMF_TRY(ometa.alloc(threads * lb.ovf, st));
            PMMF_TRY(oval.alloc(threads * lb.ovf, st));
            lb.ometa = ometa.p;
            lb.oval = oval.p;
        }
    }
    const LaneArgs *lbp = lane ? &lb : nullptr;

    // pass 1: V = A Q^T, scattered straight into the rows of W = V^T
    DBuf<int64_t> wrp, wcur;
    PMMF_TRY(wrp.zeros(s + 1, st));
    a.rp = A.rowptr.p;
    a.ci = A.col.p;
    a.v = A.val.p;
    a.rows = s;
    a.wcnt = wrp.p;
    PMMF_TRY(launch_rows<P1_COUNT>(a, A.nnz, 0, st, lbp));
    // row starts of W, and a copy as the write cursors of pass 1
    PMMF_TRY(wcur.alloc(s + 1, st));
    PMMF_TRY(scan_i64_dup(wrp.p, wrp.p, wcur.p, s, st));
    // W is allocated from an estimate, without waiting for the count: when the
    // count exceeds it, pass 1 writes nothing, W's rows stay empty, and the
    // size read with pass 2's below triggers a second, exact round
    Csr W;
    W.rows = s;
    int64_t wcap = out.w_hint > 0 ? out.w_hint
                                  : (int64_t)tuned(TUNE_PASS1_ESTIMATE, 0, 8) * A.nnz + 1024;
    // pass 1's overflow flag and pass 2's longest row, zeroed together
    DBuf<unsigned long long> flags;
    PMMF_TRY(flags.zeros(2, st));
    unsigned long long *wover = flags.p, *maxlen = flags.p + 1;
    PMMF_TRY(W.col.alloc(wcap, st));
    PMMF_TRY(W.val.alloc(wcap, st));
    auto pass1_write = [&](bool again) -> pmmf_status {
        if (again)
            PMMF_CUDA_TRY(cudaMemcpyAsync(wcur.p, wrp.p, sizeof(int64_t) * (size_t)(s + 1),
                                          cudaMemcpyDeviceToDevice, st));
        a.rp = A.rowptr.p;
        a.rend = nullptr;
        a.ci = A.col.p;
        a.v = A.val.p;
        a.wcur = wcur.p;
        a.wcol = W.col.p;
        a.wval = W.val.p;
        a.wtotal = wrp.p + s;
        a.wcap = wcap;
        a.wover = wover;
        return launch_rows<P1_WRITE>(a, A.nnz, wcap, st, lbp);
    };
    PMMF_TRY(pass1_write(false));
    // W's row r holds wrp[r] .. wcur[r] - 1 (the written part of its capacity)

    const int64_t s2 = sv.count;       // one elimination per rotation

    // pass 2: A_p = W Q^T with accounting and compaction
    out.next.rows = s2;
    // every surviving row writes its slot of caprp and acnt: no zeroing
    DBuf<int64_t> caprp, acnt;
    PMMF_TRY(caprp.alloc(s2 + 1, st));
    PMMF_TRY(acnt.alloc(s2 + 1, st));
    // hv: pass 2's capacity and longest row, W's exact size, pass 1's overflow
    int64_t hv[4] = {0, 0, 0, 0};
    int64_t *mb_d = nullptr;
    const volatile int64_t *mb = host_mailbox(&mb_d);
    if (!mb) return PMMF_ERR_CUDA;
    auto pass2_count = [&]() -> pmmf_status {
        a.rp = wrp.p;
        a.rend = wcur.p;
        a.ci = W.col.p;
        a.v = W.val.p;
        a.newrow = sv.newrow.p;
        a.ocnt = caprp.p;
        a.maxlen = maxlen;
        PMMF_TRY(launch_rows<P2_COUNT>(a, wcap, 0, st, lbp));
        PMMF_TRY(scan_i64(caprp.p, caprp.p, s2, st));
        // the four sizes in one write to the host mailbox
        k_pass2_sizes<<<1, 32, 0, st>>>(caprp.p + s2, maxlen, wrp.p + s, wover,
                                        mb_d + MB_PASS2);
        PMMF_TRY(launched("pass2_sizes"));
        PMMF_CUDA_TRY(cudaStreamSynchronize(st));
        for (int i = 0; i < 4; ++i) hv[i] = mb[MB_PASS2 + i];
        return PMMF_OK;
    };
    PMMF_TRY(pass2_count());
    if (hv[3]) {
        // the estimate was short: W at its exact size, and pass 1's writes and
        // pass 2's count again
        wcap = hv[2];
        PMMF_TRY(W.col.alloc(wcap, st));
        PMMF_TRY(W.val.alloc(wcap, st));
        PMMF_CUDA_TRY(cudaMemsetAsync(flags.p, 0, 2 * sizeof(unsigned long long), st));
        PMMF_TRY(pass1_write(true));
        PMMF_TRY(pass2_count());
    }
    out.w_nnz = hv[2];
    DBuf<int32_t> tcol;
    DBuf<double> tval;
    PMMF_TRY(tcol.alloc(hv[0], st));
    PMMF_TRY(tval.alloc(hv[0], st));
    a.outcap = (int)(hv[1] > 0 ? hv[1] : 1);
    a.orp = caprp.p;
    a.ocol = tcol.p;
    a.oval = tval.p;
    a.acnt = acnt.p;
    PMMF_TRY(launch_rows<P2_WRITE>(a, hv[2], hv[0], st, lbp));
    // exact row pointers, and the rows moved there; nnz is the capacity (an
    // upper bound), the exact count is rowptr[s2] on the device
    PMMF_TRY(out.next.rowptr.alloc(s2 + 1, st));
    PMMF_TRY(scan_i64(acnt.p, out.next.rowptr.p, s2, st));
    out.next.nnz = hv[0];
    out.next.nnz_exact = false;
    PMMF_TRY(out.next.col.alloc(hv[0], st));
    PMMF_TRY(out.next.val.alloc(hv[0], st));
    if (s2 > 0) {
        k_compact_rows<<<grid_for(s2 * 32, 256), 256, 0, st>>>(caprp.p, out.next.rowptr.p, s2, tcol.p,
                                                                tval.p, out.next.col.p, out.next.val.p);
        PMMF_TRY(launched("compact_rows"));
    }
    return PMMF_OK;
}

pmmf_status transform_stage(const Csr &R, const int32_t *ids, const int32_t *cl, const int32_t *loc,
                            const StageClusters &cls, int64_t cmax, const StageRotations &rot,
                            const int32_t *elimflag, int32_t stage, double *hdiag,
                            double *contrib, Csr &out, DBuf<int32_t> &out_ids,
                            unsigned *status, cudaStream_t st) {
    const int64_t s = R.rows;
    RowArgs a{};
    a.act = ids;
    a.cl = cl;
    a.loc = loc;
    a.coff = cls.coff.p;
    a.roff = rot.roff.p;
    a.lvl_off = rot.lvl_off.p;
    a.nlev = rot.nlev.p;
    a.lvlrot = rot.lvl.p;
    a.rec = rot.rec.p;
    a.K = rot.K;
    a.kidx = rot.kidx.p;
    a.kkv = rot.kk.p;
    a.lvlidx = rot.lvlidx.p;
    a.kO = rot.kO.p;
    a.cmax = cmax;
    a.elimflag = elimflag;
    a.stage = stage;
    a.status = status;
    a.contrib = contrib;
    a.hdiag = hdiag;
    // member -> global id, with bit 31 when this stage eliminates it
    int64_t nmem = 0;
    PMMF_CUDA_TRY(cudaMemcpyAsync(&nmem, cls.coff.p + cls.m, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    PMMF_CUDA_TRY(cudaStreamSynchronize(st));
    DBuf<int32_t> mge;
    PMMF_TRY(mge.alloc(std::max<int64_t>(nmem, 1), st));
    if (nmem > 0) {
        k_member_ge<<<grid_for(nmem, 256), 256, 0, st>>>(cls.members.p, nmem, elimflag, stage, mge.p);
        PMMF_TRY(launched("member_ge"));
    }
    a.mge = mge.p;
    // the surviving rows and their output positions
    Survivors sv;
    PMMF_TRY(sv.flag.alloc(std::max<int64_t>(s, 1), st));
    PMMF_TRY(sv.newrow.alloc(s + 1, st));
    int64_t s2 = 0;
    if (s > 0) {
        k_survivors<<<grid_for(s, 256), 256, 0, st>>>(ids, s, elimflag, stage, sv.flag.p);
        PMMF_TRY(launched("survivors"));
    }
    PMMF_TRY(scan_i32_to_i64(sv.flag.p, sv.newrow.p, s, st));
    PMMF_CUDA_TRY(cudaMemcpyAsync(&s2, sv.newrow.p + s, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    PMMF_CUDA_TRY(cudaStreamSynchronize(st));
    PMMF_TRY(out_ids.alloc(std::max<int64_t>(s2, 1), st));
    if (s > 0) {
        k_compact_act<<<grid_for(s, 256), 256, 0, st>>>(ids, s, sv.flag.p, sv.newrow.p, out_ids.p);
        PMMF_TRY(launched("compact_ids"));
    }
    a.rp = R.rowptr.p;
    a.rend = nullptr;
    a.ci = R.col.p;
    a.v = R.val.p;
    a.rows = s;
    a.newrow = sv.newrow.p;
    DBuf<int64_t> caprp, acnt;
    DBuf<unsigned long long> maxlen;
    PMMF_TRY(caprp.alloc(s2 + 1, st));
    PMMF_TRY(acnt.alloc(s2 + 1, st));
    PMMF_TRY(maxlen.zeros(1, st));
    a.ocnt = caprp.p;
    a.maxlen = maxlen.p;
    if (s > 0) PMMF_TRY(launch_rows<P2_COUNT>(a, R.nnz, 0, st));
    PMMF_TRY(scan_i64(caprp.p, caprp.p, s2, st));
    int64_t cap = 0;
    unsigned long long ml = 0;
    PMMF_CUDA_TRY(cudaMemcpyAsync(&cap, caprp.p + s2, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    PMMF_CUDA_TRY(cudaMemcpyAsync(&ml, maxlen.p, sizeof(ml), cudaMemcpyDeviceToHost, st));
    PMMF_CUDA_TRY(cudaStreamSynchronize(st));
    DBuf<int32_t> tcol;
    DBuf<double> tval;
    PMMF_TRY(tcol.alloc(std::max<int64_t>(cap, 1), st));
    PMMF_TRY(tval.alloc(std::max<int64_t>(cap, 1), st));
    a.outcap = (int)(ml > 0 ? ml : 1);
    a.orp = caprp.p;
    a.ocol = tcol.p;
    a.oval = tval.p;
    a.acnt = acnt.p;
    if (s > 0) PMMF_TRY(launch_rows<P2_WRITE>(a, R.nnz, cap, st));
    out.rows = s2;
    PMMF_TRY(out.rowptr.alloc(s2 + 1, st));
    PMMF_TRY(scan_i64(acnt.p, out.rowptr.p, s2, st));
    PMMF_CUDA_TRY(cudaMemcpyAsync(&out.nnz, out.rowptr.p + s2, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    PMMF_CUDA_TRY(cudaStreamSynchronize(st));
    out.nnz_exact = true;
    PMMF_TRY(out.col.alloc(std::max<int64_t>(out.nnz, 1), st));
    PMMF_TRY(out.val.alloc(std::max<int64_t>(out.nnz, 1), st));
    if (s2 > 0) {
        k_compact_rows<<<grid_for(s2 * 32, 256), 256, 0, st>>>(caprp.p, out.rowptr.p, s2, tcol.p,
                                                                tval.p, out.col.p, out.val.p);
        PMMF_TRY(launched("compact_rows"));
    }
    // the scratch above is freed stream-ordered on st; the results stay
    return PMMF_OK;
}

pmmf_status extract_core(const Csr &A, const int32_t *pos, int64_t s, double *core, double *hdiag,
                         const int32_t *act, cudaStream_t st) {
    if (s <= 0) return PMMF_OK;
    PMMF_CUDA_TRY(cudaMemsetAsync(core, 0, sizeof(double) * (size_t)(s * s), st));
    k_core<<<grid_for(s * 32, 256), 256, 0, st>>>(A.rowptr.p, A.col.p, A.val.p, s, pos, act, core,
                                                  hdiag);
    return launched("core");
}

}  // namespace pmmf
