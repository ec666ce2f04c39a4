// partition.cu -- Algorithm 1, "cluster the active columns": k-means on the
// coordinates' points, in exact integer arithmetic so that every assignment is
// reproducible bit for bit, plus the per-stage elimination schedule.
//
// Points are quantized once to 15-bit integers per dimension over the bounding
// box of all n points.  Each stage initialises m centroids as the rounded means
// of m equal chunks of the active points in Morton order (ties by id), then
// runs Lloyd iterations: squared integer distance (uint32 is exact: 3 * 32767^2
// < 2^32), ties to the lower centroid, centroid = round(sum / count) with halves
// up, an empty cluster keeps its centroid.  Sums are integers, so the atomics
// that accumulate them are order independent.
#include <cooperative_groups.h>

#include <algorithm>
#include <climits>

#include "common.cuh"
#include "stage.cuh"

namespace pmmf {

namespace {

constexpr uint32_t QMAX = 32767u;

// Order-preserving map of a (not NaN) double to an unsigned key and back:
// min and max of the keys are the min and max of the values, in integer
// instructions (the FP64 pipe is narrow on GB300).
__device__ __forceinline__ unsigned long long ord_key(double x) {
    const unsigned long long u = f64_bits(x);
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}
__device__ __forceinline__ double ord_val(unsigned long long k) {
    return f64_from_bits((k >> 63) ? (k & 0x7fffffffffffffffull) : ~k);
}

// Bounding box of the points: keys[d] = min key, keys[dim + d] = max key of
// coordinate d (keys preset to all ones / zero); flags non-finite values.
__global__ void k_bbox(const double *x, int64_t n, int dim, unsigned long long *keys,
                       unsigned *status) {
    bool bad = false;
    for (int d = 0; d < dim; ++d) {
        unsigned long long lo = ~0ull, hi = 0ull;
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
             i += (int64_t)gridDim.x * blockDim.x) {
            const double v = x[i * dim + d];
            bad |= ((f64_bits(v) >> 52) & 0x7ffull) == 0x7ffull;   // inf or NaN
            const unsigned long long k = ord_key(v);
            lo = k < lo ? k : lo;
            hi = k > hi ? k : hi;
        }
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long a = __shfl_xor_sync(0xffffffffu, lo, o);
            const unsigned long long b = __shfl_xor_sync(0xffffffffu, hi, o);
            lo = a < lo ? a : lo;
            hi = b > hi ? b : hi;
        }
        if ((threadIdx.x & 31) == 0) {
            atomicMin(&keys[d], lo);
            atomicMax(&keys[dim + d], hi);
        }
    }
    if (bad) atomicOr(status, ST_NONFINITE);
}

__global__ void k_quantize(const double *x, int64_t n, int dim, const unsigned long long *keys,
                           int32_t *q, uint64_t *code) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t qq[3] = {0, 0, 0};
        for (int d = 0; d < dim; ++d) {
            const double lo = ord_val(keys[d]), hi = ord_val(keys[dim + d]);
            double span = __dsub_rn(hi, lo);
            double scale = span > 0.0 ? __ddiv_rn((double)QMAX, span) : 0.0;
            double f = floor(__dmul_rn(__dsub_rn(x[i * dim + d], lo), scale));
            uint32_t v = f <= 0.0 ? 0u : (f >= (double)QMAX ? QMAX : (uint32_t)f);
            qq[d] = v;
            q[i * dim + d] = (int32_t)v;
        }
        uint64_t c = 0;
        for (int b = 0; b < 15; ++b)
            for (int d = 0; d < dim; ++d) c |= (uint64_t)((qq[d] >> b) & 1u) << (b * dim + d);
        code[i] = c;
    }
}

// flag[i] = 1 if the i-th point of the global Morton order is active
__global__ void k_active_flags(const int32_t *morder, int64_t n, const int32_t *pos,
                               int32_t *flag) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        flag[i] = pos[morder[i]] >= 0 ? 1 : 0;
}

__global__ void k_compact_order(const int32_t *morder, int64_t n, const int32_t *pos,
                                const int64_t *ex, int32_t *out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        if (pos[morder[i]] >= 0) out[ex[i]] = morder[i];
}

// Initial centroids: chunk t holds Morton-order positions [floor(t s/m), floor((t+1) s/m)).
// Chunk t holds Morton positions r with t = ((r + 1) m - 1) / s (contiguous
// and nondecreasing in r): each warp sums its lanes' points per chunk first
// (segments are runs of lanes) and one lane per segment adds the total.
__global__ void k_chunk_sums(const int32_t *amorder, int64_t s, int64_t m, const int32_t *q,
                             int dim, unsigned long long *sum, unsigned long long *cnt) {
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); r0 < s; r0 += stride) {
        const int64_t r = r0 + lane;
        const bool in = r < s;
        const int64_t t = in ? ((r + 1) * m - 1) / s : -1 - lane;
        const int32_t g = in ? amorder[r] : 0;
        unsigned long long v[3], c = in ? 1ull : 0ull;
        for (int d = 0; d < dim; ++d) v[d] = in ? (unsigned long long)q[(int64_t)g * dim + d] : 0ull;
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t to = __shfl_down_sync(0xffffffffu, t, o);
            const unsigned long long co = __shfl_down_sync(0xffffffffu, c, o);
            unsigned long long vo[3];
            for (int d = 0; d < dim; ++d) vo[d] = __shfl_down_sync(0xffffffffu, v[d], o);
            if (lane + o < 32 && to == t) {
                c += co;
                for (int d = 0; d < dim; ++d) v[d] += vo[d];
            }
        }
        const int64_t tp = __shfl_up_sync(0xffffffffu, t, 1);
        if (in && (lane == 0 || tp != t)) {
            for (int d = 0; d < dim; ++d) atomicAdd(&sum[t * dim + d], v[d]);
            atomicAdd(&cnt[t], c);
        }
    }
}

__global__ void k_centroids(int64_t m, int dim, const unsigned long long *sum,
                            const unsigned long long *cnt, int32_t *cen) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m;
         t += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long c = cnt[t];
        if (c == 0) continue;
        for (int d = 0; d < dim; ++d) cen[t * dim + d] = (int32_t)((sum[t * dim + d] + c / 2) / c);
    }
}

// Assignment step: nearest centroid in squared integer distance, ties to the
// lower index; accumulate the new sums.
template <int DIM>
__global__ void k_assign(const int32_t *act, int64_t s, const int32_t *q, const int32_t *cen,
                         int64_t m, int32_t *label, unsigned long long *sum,
                         unsigned long long *cnt) {
    extern __shared__ int32_t sc[];
    for (int64_t t = threadIdx.x; t < m * DIM; t += blockDim.x) sc[t] = cen[t];
    __syncthreads();
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < s;
         r += (int64_t)gridDim.x * blockDim.x) {
        int32_t g = act[r];
        int32_t p[DIM];
        for (int d = 0; d < DIM; ++d) p[d] = q[(int64_t)g * DIM + d];
        uint32_t best = 0xffffffffu;
        int64_t bt = 0;
        for (int64_t t = 0; t < m; ++t) {
            uint32_t dd = 0;
            for (int d = 0; d < DIM; ++d) {
                int32_t z = p[d] - sc[t * DIM + d];
                dd += (uint32_t)(z * z);
            }
            if (dd < best) { best = dd; bt = t; }
        }
        label[r] = (int32_t)bt;
        for (int d = 0; d < DIM; ++d) atomicAdd(&sum[bt * DIM + d], (unsigned long long)p[d]);
        atomicAdd(&cnt[bt], 1ull);
    }
}

// Candidate centroids kept per warp by nearest_centroid (more: a full scan).
constexpr int LL_CAND = 128;
constexpr int LL_WARPS = 8;   // k_lloyd's blocks are 256 threads

// Nearest centroid (squared integer distance, ties to the lower index) of the
// point p of every live lane of a warp whose points are close together (all
// 32 lanes call it).  Centroids that cannot be nearest to any point of the
// warp's bounding box are skipped: with U the smallest, over the centroids, of
// the largest squared distance from the box, a centroid whose smallest squared
// distance from the box exceeds U is farther from every point of the box than
// that centroid.  The candidates, in ascending index, therefore include every
// nearest centroid of every point, ties included, and the strict comparison
// in index order keeps the lowest: the result is the full scan's.  Squared
// distances of 15-bit coordinates fit 32 bits.
template <int DIM>
__device__ __forceinline__ int64_t nearest_centroid(const int32_t (&p)[DIM], bool live, const int32_t *sc,
                                                    int64_t m, int32_t *cand) {
    const int lane = threadIdx.x & 31;
    const unsigned full = 0xffffffffu;
    int32_t lo[DIM], hi[DIM];
    for (int d = 0; d < DIM; ++d) {
        lo[d] = __reduce_min_sync(full, live ? p[d] : INT_MAX);
        hi[d] = __reduce_max_sync(full, live ? p[d] : INT_MIN);
    }
    uint32_t U = 0xffffffffu;
    for (int64_t t = lane; t < m; t += 32) {
        uint32_t ub = 0;
        for (int d = 0; d < DIM; ++d) {
            const int32_t c = sc[t * DIM + d];
            const int32_t z = max(abs(c - lo[d]), abs(c - hi[d]));
            ub += (uint32_t)(z * z);
        }
        U = min(U, ub);
    }
    U = __reduce_min_sync(full, U);
    int n = 0;
    for (int64_t t0 = 0; t0 < m; t0 += 32) {
        const int64_t t = t0 + lane;
        bool ok = false;
        if (t < m) {
            uint32_t lb = 0;
            for (int d = 0; d < DIM; ++d) {
                const int32_t c = sc[t * DIM + d];
                const int32_t z = max(0, max(lo[d] - c, c - hi[d]));
                lb += (uint32_t)(z * z);
            }
            ok = lb <= U;
        }
        const unsigned b = __ballot_sync(full, ok);
        const int at = n + __popc(b & ((1u << lane) - 1u));
        if (ok && at < LL_CAND) cand[at] = (int32_t)t;
        n += __popc(b);
    }
    __syncwarp();
    uint32_t best = 0xffffffffu;
    int64_t bt = 0;
    if (n <= LL_CAND) {
        for (int k = 0; k < n; ++k) {
            const int64_t t = cand[k];
            uint32_t dd = 0;
            for (int d = 0; d < DIM; ++d) {
                const int32_t z = p[d] - sc[t * DIM + d];
                dd += (uint32_t)(z * z);
            }
            if (dd < best) {
                best = dd;
                bt = t;
            }
        }
    } else {
        for (int64_t t = 0; t < m; ++t) {
            uint32_t dd = 0;
            for (int d = 0; d < DIM; ++d) {
                const int32_t z = p[d] - sc[t * DIM + d];
                dd += (uint32_t)(z * z);
            }
            if (dd < best) {
                best = dd;
                bt = t;
            }
        }
    }
    __syncwarp();   // the list is reused by the warp's next points
    return bt;
}

// All Lloyd iterations in one cooperative launch (every block resident):
// per iteration the accumulators are cleared, every point is assigned to its
// nearest centroid (as k_assign) and, except after the last iteration, the
// centroids are recomputed (as k_centroids), with a grid-wide barrier between
// the phases.  Integer sums, so the result is independent of the order of the
// atomics.
// One grid barrier per iteration: the sums rotate through three buffers (the
// one being accumulated, the previous iteration's, which every block turns
// into the centroids in its own shared memory, and the next one, zeroed
// meanwhile; sum and cnt hold 3 m DIM and 3 m entries, buffer 0 zero on
// entry).  The last iteration's counts are in buffer (iters - 1) % 3.
// Points are taken in Morton order (order[r'] = the r'-th active point's id,
// pos[id] = its active index), so a warp's points are neighbours that mostly
// share their nearest centroid: the warp searches only the centroids that
// can be nearest to its points' bounding box (nearest_centroid), and lanes
// with the same centroid add their coordinates and count with one atomic
// each (integer sums, so the order of the additions does not matter).
// Shared memory: the centroids, then LL_CAND candidate slots per warp.
template <int DIM>
__global__ void k_lloyd(const int32_t *order, const int32_t *pos, int64_t s, const int32_t *q,
                        const int32_t *cen, int64_t m, int iters, int32_t *label,
                        unsigned long long *sum, unsigned long long *cnt) {
    namespace cg = cooperative_groups;
    cg::grid_group grid = cg::this_grid();
    extern __shared__ int32_t sc[];
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t gs = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = threadIdx.x; t < m * DIM; t += blockDim.x) sc[t] = cen[t];
    for (int it = 0; it < iters; ++it) {
        unsigned long long *sacc = sum + (int64_t)(it % 3) * m * DIM, *cacc = cnt + (int64_t)(it % 3) * m;
        unsigned long long *snext = sum + (int64_t)((it + 1) % 3) * m * DIM, *cnext = cnt + (int64_t)((it + 1) % 3) * m;
        if (it + 1 < iters) {
            for (int64_t t = gt; t < m * DIM; t += gs) snext[t] = 0ull;
            for (int64_t t = gt; t < m; t += gs) cnext[t] = 0ull;
        }
        if (it > 0) {
            // the previous iteration's centroids (an empty cluster keeps its own)
            const unsigned long long *sp = sum + (int64_t)((it + 2) % 3) * m * DIM;
            const unsigned long long *cp = cnt + (int64_t)((it + 2) % 3) * m;
            for (int64_t t = threadIdx.x; t < m; t += blockDim.x) {
                const unsigned long long c = cp[t];
                if (c == 0) continue;
                for (int d = 0; d < DIM; ++d) sc[t * DIM + d] = (int32_t)((sp[t * DIM + d] + c / 2) / c);
            }
        }
        __syncthreads();
        const int lane = threadIdx.x & 31;
        int32_t *cand = (int32_t *)(sc + m * DIM) + (threadIdx.x >> 5) * LL_CAND;
        for (int64_t r0 = gt - lane; r0 < s; r0 += gs) {
            const int64_t r = r0 + lane;
            const bool live = r < s;
            const int32_t g = live ? order[r] : 0;
            int32_t p[DIM];
            for (int d = 0; d < DIM; ++d) p[d] = live ? q[(int64_t)g * DIM + d] : 0;
            const int64_t bt = nearest_centroid<DIM>(p, live, sc, m, cand);
            // quantized coordinates are below 2^16, so 32 of them sum in 32 bits
            const unsigned lm = __ballot_sync(0xffffffffu, live);
            if (live) {
                label[pos[g]] = (int32_t)bt;
                const unsigned grp = __match_any_sync(lm, (int)bt);
                const bool leader = lane == __ffs(grp) - 1;
                for (int d = 0; d < DIM; ++d) {
                    const unsigned v = __reduce_add_sync(grp, (unsigned)p[d]);
                    if (leader) atomicAdd(&sacc[bt * DIM + d], (unsigned long long)v);
                }
                if (leader) atomicAdd(&cacc[bt], (unsigned long long)__popc(grp));
            }
        }
        grid.sync();
    }
}

// Nonempty labels become cluster ordinals in ascending label order.
__global__ void k_nonempty(const unsigned long long *cnt, int64_t m, int32_t *flag) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m;
         t += (int64_t)gridDim.x * blockDim.x)
        flag[t] = cnt[t] > 0 ? 1 : 0;
}

__global__ void k_cluster_sizes(const unsigned long long *cnt, int64_t m, const int64_t *ord,
                                int64_t *size) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m;
         t += (int64_t)gridDim.x * blockDim.x)
        if (cnt[t] > 0) size[ord[t]] = (int64_t)cnt[t];
}

__global__ void k_members(const int32_t *act, const int32_t *label, const int32_t *perm, int64_t s,
                          const int64_t *ord, const int64_t *coff, int32_t *members, int32_t *cl,
                          int32_t *loc) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < s;
         j += (int64_t)gridDim.x * blockDim.x) {
        int32_t r = perm[j];
        int32_t g = act[r];
        int64_t u = ord[label[r]];
        members[j] = g;
        cl[g] = (int32_t)u;
        loc[g] = (int32_t)(j - coff[u]);
    }
}

__global__ void k_one_cluster(const int32_t *act, int64_t s, int32_t *members, int32_t *cl,
                              int32_t *loc, int64_t *coff) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < s;
         r += (int64_t)gridDim.x * blockDim.x) {
        int32_t g = act[r];
        members[r] = g;
        cl[g] = 0;
        loc[g] = (int32_t)r;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) { coff[0] = 0; coff[1] = s; }
}

// Elimination schedule: e_u = floor(eta c_u); while the total exceeds
// s - core_size, the largest e_u is decremented (ties to the lowest u).  That
// greedy equals capping every e_u at the smallest level L with
// sum_u min(e_u, L) >= target and then decrementing the first
// (sum - target) clusters (ascending u) that sit at L.  out[0] = total,
// out[1] = 1 if no cluster can rotate (the caller then uses one cluster).
// Block-wide reductions and exclusive scan of int64 (every thread gets the
// result); red holds one slot per warp plus one.
template <bool MAX>
__device__ int64_t block_reduce_i64(int64_t v, int64_t *red) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        const int64_t x = __shfl_xor_sync(0xffffffffu, v, o);
        v = MAX ? (x > v ? x : v) : v + x;
    }
    if (lane == 0) red[w] = v;
    __syncthreads();
    if (w == 0) {
        v = lane < nw ? red[lane] : 0;
        for (int o = 16; o > 0; o >>= 1) {
            const int64_t x = __shfl_xor_sync(0xffffffffu, v, o);
            v = MAX ? (x > v ? x : v) : v + x;
        }
        if (lane == 0) red[32] = v;
    }
    __syncthreads();
    v = red[32];
    __syncthreads();
    return v;
}

__device__ int64_t block_exscan_i64(int64_t v, int64_t *red) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    int64_t inc = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t x = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += x;
    }
    if (lane == 31) red[w] = inc;
    __syncthreads();
    if (w == 0) {
        int64_t t = lane < nw ? red[lane] : 0, ti = t;
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t x = __shfl_up_sync(0xffffffffu, ti, o);
            if (lane >= o) ti += x;
        }
        if (lane < nw) red[lane] = ti - t;     // exclusive warp offsets
    }
    __syncthreads();
    const int64_t r = red[w] + inc - v;
    __syncthreads();
    return r;
}

constexpr int SCHED_THREADS = 1024;

// Rotations per cluster for one stage (one block; thread t owns the
// contiguous clusters [t * chunk, (t + 1) * chunk)): e_u = floor(eta c_u),
// capped when the total would take the active set below the core size (the
// largest cap L keeping the total >= s - core, then the surplus taken one by
// one from the first clusters at the cap, in cluster order); a single
// cluster of the whole stage when no cluster can rotate.  Writes e, roff
// (exclusive scan of e) and out = [total, one-cluster fallback, largest
// cluster, sum of squared cluster sizes].
__global__ void __launch_bounds__(SCHED_THREADS)
k_schedule(const int64_t *coff, int64_t mm_host, const int64_t *mm_dev, int64_t s, int64_t core,
           double eta, int64_t *e, int64_t *roff, int64_t *out) {
    __shared__ int64_t red[33];
    const int64_t mm = mm_dev ? *mm_dev : mm_host;
    if (threadIdx.x == 0) out[4] = mm;
    const int64_t chunk = (mm + SCHED_THREADS - 1) / SCHED_THREADS;
    const int64_t u0 = threadIdx.x * chunk, u1 = u0 + chunk < mm ? u0 + chunk : mm;
    int64_t tot = 0, emx = 0, cmx = 0, sq = 0;
    for (int64_t u = u0; u < u1; ++u) {
        const int64_t c = coff[u + 1] - coff[u];
        const int64_t v = (int64_t)floor(__dmul_rn(eta, (double)c));
        e[u] = v;
        tot += v;
        emx = v > emx ? v : emx;
        cmx = c > cmx ? c : cmx;
        sq += c * c;
    }
    int64_t total = block_reduce_i64<false>(tot, red);
    const int64_t emax = block_reduce_i64<true>(emx, red);
    const int64_t cmax = block_reduce_i64<true>(cmx, red);
    const int64_t sqs = block_reduce_i64<false>(sq, red);
    const int64_t target = s - core;
    if (total > target) {
        int64_t lo = 0, hi = emax;   // smallest L with sum_u min(e_u, L) >= target
        while (lo < hi) {
            const int64_t mid = (lo + hi) / 2;
            int64_t f = 0;
            for (int64_t u = u0; u < u1; ++u) f += e[u] < mid ? e[u] : mid;
            f = block_reduce_i64<false>(f, red);
            if (f >= target) hi = mid; else lo = mid + 1;
        }
        const int64_t L = lo;
        int64_t f = 0, atL = 0;
        for (int64_t u = u0; u < u1; ++u) {
            if (e[u] > L) e[u] = L;
            f += e[u];
            atL += e[u] == L;
        }
        f = block_reduce_i64<false>(f, red);
        const int64_t before = block_exscan_i64(atL, red);   // clusters at L before mine
        const int64_t excess = f - target;
        int64_t rank = before;
        for (int64_t u = u0; u < u1; ++u)
            if (e[u] == L) {
                if (rank < excess) e[u] -= 1;
                ++rank;
            }
        total = f - (excess > 0 ? excess : 0);
    }
    if (total == 0) {
        // every cluster too small to rotate: one cluster for the stage
        if (threadIdx.x == 0) {
            int64_t ee = (int64_t)floor(__dmul_rn(eta, (double)s));
            if (ee > target) ee = target;
            if (ee < 1) ee = 1;
            e[0] = ee;
            roff[0] = 0;
            roff[1] = ee;
            out[0] = ee;
            out[1] = 1;
            out[2] = s;
            out[3] = s * s;
        }
        return;
    }
    int64_t mine = 0;
    for (int64_t u = u0; u < u1; ++u) mine += e[u];
    int64_t acc = block_exscan_i64(mine, red);
    if (threadIdx.x == 0) roff[0] = 0;
    for (int64_t u = u0; u < u1; ++u) {
        acc += e[u];
        roff[u + 1] = acc;
    }
    if (threadIdx.x == 0) {
        out[0] = total;
        out[1] = 0;
        out[2] = cmax;
        out[3] = sqs;
    }
}

}  // namespace

pmmf_status quantize_points(const double *coords, int64_t n, int dim, int32_t *q, uint64_t *code,
                            unsigned *status, cudaStream_t st) {
    DBuf<unsigned long long> keys;
    PMMF_TRY(keys.alloc(2 * dim, st));
    PMMF_CUDA_TRY(cudaMemsetAsync(keys.p, 0xFF, sizeof(unsigned long long) * (size_t)dim, st));
    PMMF_CUDA_TRY(cudaMemsetAsync(keys.p + dim, 0, sizeof(unsigned long long) * (size_t)dim, st));
    k_bbox<<<grid_for(n, 256), 256, 0, st>>>(coords, n, dim, keys.p, status);
    PMMF_TRY(launched("bbox"));
    k_quantize<<<grid_for(n, 256), 256, 0, st>>>(coords, n, dim, keys.p, q, code);
    return launched("quantize");
}

// Clusters from labels in [0, m) with their counts: the nonempty labels in
// ascending order, members ascending by global id (R10's order).
static pmmf_status clusters_from_labels(const PartitionIn &in, DBuf<int32_t> &label,
                                        const unsigned long long *cnt, int64_t m,
                                        StageClusters &out, cudaStream_t st) {
    const int64_t s = in.s;
    DBuf<int32_t> perm, nflag;
    DBuf<int64_t> ord, size;
    PMMF_TRY(nflag.alloc(m, st));
    PMMF_TRY(ord.alloc(m + 1, st));
    k_nonempty<<<grid_for(m, 256), 256, 0, st>>>(cnt, m, nflag.p);
    PMMF_TRY(launched("nonempty"));
    PMMF_TRY(scan_i32_to_i64(nflag.p, ord.p, m, st));
    // the nonempty count stays on the device (read with the schedule); the
    // arrays are sized for all m labels, the empty ones last with size 0
    PMMF_TRY(out.count_d.alloc(1, st));
    PMMF_CUDA_TRY(cudaMemcpyAsync(out.count_d.p, ord.p + m, sizeof(int64_t), cudaMemcpyDeviceToDevice, st));
    PMMF_TRY(size.zeros(m + 1, st));
    k_cluster_sizes<<<grid_for(m, 256), 256, 0, st>>>(cnt, m, ord.p, size.p);
    PMMF_TRY(launched("cluster_sizes"));
    PMMF_TRY(out.coff.alloc(m + 1, st));
    PMMF_TRY(scan_i64(size.p, out.coff.p, m, st));
    PMMF_TRY(perm.alloc(s, st));
    PMMF_TRY(stable_sort_by_key((const uint32_t *)label.p, s, m, perm.p, st));
    k_members<<<grid_for(s, 256), 256, 0, st>>>(in.act, label.p, perm.p, s, ord.p, out.coff.p,
                                                 out.members.p, in.cl, in.loc);
    PMMF_TRY(launched("members"));
    out.m = m;
    return PMMF_OK;
}

__global__ void k_check_labels(const int32_t *lab, int64_t n, int64_t m, unsigned *status) {
    bool bad = false;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        bad |= lab[i] < 0 || lab[i] >= m;
    if (bad) atomicOr(status, ST_BAD_LABEL);
}

__global__ void k_gather_labels(const int32_t *act, int64_t s, const int32_t *labels, int32_t *label,
                                unsigned long long *cnt) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < s;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int32_t l = labels[act[r]];
        label[r] = l;
        atomicAdd(&cnt[l], 1ull);
    }
}

pmmf_status check_labels(const int32_t *labels, int64_t n, int64_t m, unsigned *status,
                         cudaStream_t st) {
    k_check_labels<<<grid_for(n, 256), 256, 0, st>>>(labels, n, m, status);
    return launched("check_labels");
}

pmmf_status partition_from_labels(const PartitionIn &in, const int32_t *labels, int64_t m,
                                  StageClusters &out, cudaStream_t st) {
    const int64_t s = in.s;
    PMMF_TRY(out.members.alloc(s, st));
    DBuf<int32_t> label;
    DBuf<unsigned long long> cnt;
    PMMF_TRY(label.alloc(s, st));
    PMMF_TRY(cnt.zeros(m, st));
    k_gather_labels<<<grid_for(s, 256), 256, 0, st>>>(in.act, s, labels, label.p, cnt.p);
    PMMF_TRY(launched("gather_labels"));
    return clusters_from_labels(in, label, cnt.p, m, out, st);
}

pmmf_status partition_stage(const PartitionIn &in, int64_t m, int iters, StageClusters &out,
                            cudaStream_t st) {
    const int64_t s = in.s;
    const int dim = in.dim;
    PMMF_TRY(out.members.alloc(s, st));
    if (m <= 1 || !in.q) {
        PMMF_TRY(out.coff.alloc(2, st));
        k_one_cluster<<<grid_for(s, 256), 256, 0, st>>>(in.act, s, out.members.p, in.cl, in.loc,
                                                         out.coff.p);
        PMMF_TRY(launched("one_cluster"));
        out.m = 1;
        return PMMF_OK;
    }
    // active points in Morton order
    DBuf<int32_t> flag, amorder, label, cen;
    DBuf<int64_t> ex;
    DBuf<unsigned long long> sum, cnt;
    PMMF_TRY(flag.alloc(in.n, st));
    PMMF_TRY(ex.alloc(in.n + 1, st));
    PMMF_TRY(amorder.alloc(s, st));
    k_active_flags<<<grid_for(in.n, 256), 256, 0, st>>>(in.morder, in.n, in.pos, flag.p);
    PMMF_TRY(launched("active_flags"));
    PMMF_TRY(scan_i32_to_i64(flag.p, ex.p, in.n, st));
    k_compact_order<<<grid_for(in.n, 256), 256, 0, st>>>(in.morder, in.n, in.pos, ex.p, amorder.p);
    PMMF_TRY(launched("compact_order"));
    // initial centroids
    PMMF_TRY(sum.zeros(m * dim, st));
    PMMF_TRY(cnt.zeros(m, st));
    PMMF_TRY(cen.alloc(m * dim, st));
    k_chunk_sums<<<grid_for(s, 256), 256, 0, st>>>(amorder.p, s, m, in.q, dim, sum.p, cnt.p);
    PMMF_TRY(launched("chunk_sums"));
    k_centroids<<<grid_for(m, 256), 256, 0, st>>>(m, dim, sum.p, cnt.p, cen.p);
    PMMF_TRY(launched("centroids"));
    // Lloyd iterations
    PMMF_TRY(label.alloc(s, st));
    size_t sh = sizeof(int32_t) * (size_t)(m * dim);
    const size_t sh_lloyd = sh + sizeof(int32_t) * LL_WARPS * LL_CAND;
    if (sh > 200 * 1024) {
        set_error("too many clusters for the assignment kernel");
        return PMMF_ERR_UNSUPPORTED;
    }
    if (iters <= 0) {
        set_error("lloyd_iters must be positive");
        return PMMF_ERR_INVALID_ARG;
    }
    // one cooperative launch for all iterations when every block fits at once
    const void *lloyd = dim == 1 ? (const void *)k_lloyd<1> : dim == 2 ? (const void *)k_lloyd<2>
                                                                   : (const void *)k_lloyd<3>;
    PMMF_CUDA_TRY(allow_smem(lloyd, sh_lloyd));
    int dev = 0, nsm = 0, per_sm = 0, coop = 0;
    PMMF_CUDA_TRY(cudaGetDevice(&dev));
    PMMF_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    PMMF_CUDA_TRY(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    PMMF_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lloyd, 32 * LL_WARPS, sh_lloyd));
    DBuf<unsigned long long> lsum, lcnt;
    const unsigned long long *fcnt = cnt.p;   // the last assignment's counts
    if (coop && per_sm > 0) {
        const int64_t want = (s + 255) / 256;
        const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)nsm * per_sm));
        PMMF_TRY(lsum.zeros(3 * m * dim, st));
        PMMF_TRY(lcnt.zeros(3 * m, st));
        const int32_t *a_order = amorder.p;
        const int32_t *a_pos = in.pos;
        const int32_t *a_q = in.q;
        const int32_t *a_cen = cen.p;
        int32_t *a_label = label.p;
        int64_t a_s = s, a_m = m;
        int a_it = iters;
        unsigned long long *a_sum = lsum.p, *a_cnt = lcnt.p;
        void *args[] = {&a_order, &a_pos, &a_s, &a_q, &a_cen, &a_m, &a_it, &a_label, &a_sum, &a_cnt};
        prof_begin(KF_PARTITION, st);
        PMMF_CUDA_TRY(cudaLaunchCooperativeKernel(lloyd, dim3(g), dim3(32 * LL_WARPS), args, sh_lloyd, st));
        prof_end(KF_PARTITION, st, (double)iters * (double)s * (8.0 + 4.0 * dim),
                 3.0 * dim * (double)iters * (double)s * (double)m);
        PMMF_TRY(launched("lloyd"));
        fcnt = lcnt.p + (int64_t)((iters - 1) % 3) * m;
    } else {
    auto assign = dim == 1 ? (void *)k_assign<1> : dim == 2 ? (void *)k_assign<2> : (void *)k_assign<3>;
    PMMF_CUDA_TRY(allow_smem(assign, sh));
    for (int it = 0; it < iters; ++it) {
        PMMF_CUDA_TRY(cudaMemsetAsync(sum.p, 0, sizeof(unsigned long long) * (size_t)(m * dim), st));
        PMMF_CUDA_TRY(cudaMemsetAsync(cnt.p, 0, sizeof(unsigned long long) * (size_t)m, st));
        unsigned g = grid_for(s, 256, 152 * 8);
        prof_begin(KF_PARTITION, st);
        if (dim == 1) k_assign<1><<<g, 256, sh, st>>>(in.act, s, in.q, cen.p, m, label.p, sum.p, cnt.p);
        else if (dim == 2) k_assign<2><<<g, 256, sh, st>>>(in.act, s, in.q, cen.p, m, label.p, sum.p, cnt.p);
        else k_assign<3><<<g, 256, sh, st>>>(in.act, s, in.q, cen.p, m, label.p, sum.p, cnt.p);
        // per point: its id, its quantized coordinates and its label; integer
        // work of s * m distance evaluations (3 ops per dimension)
        prof_end(KF_PARTITION, st, (double)s * (8.0 + 4.0 * dim), 3.0 * dim * (double)s * (double)m);
        PMMF_TRY(launched("assign"));
        if (it + 1 < iters) {
            k_centroids<<<grid_for(m, 256), 256, 0, st>>>(m, dim, sum.p, cnt.p, cen.p);
            PMMF_TRY(launched("centroids"));
        }
    }
    }
    return clusters_from_labels(in, label, fcnt, m, out, st);
}

pmmf_status schedule_launch(const int64_t *coff, int64_t mm, const int64_t *mm_dev, int64_t s,
                            int64_t core, double eta, DBuf<int64_t> &e, DBuf<int64_t> &roff,
                            cudaStream_t st) {
    int64_t *mb_d = nullptr;
    if (!host_mailbox(&mb_d)) return PMMF_ERR_CUDA;
    PMMF_TRY(e.alloc(mm > 1 ? mm : 1, st));
    PMMF_TRY(roff.alloc(mm + 1 > 2 ? mm + 1 : 2, st));
    k_schedule<<<1, SCHED_THREADS, 0, st>>>(coff, mm, mm_dev, s, core, eta, e.p, roff.p,
                                            mb_d + MB_SCHED);
    return launched("schedule");
}

void schedule_read(int64_t *host_out) {
    int64_t *mb_d = nullptr;
    const volatile int64_t *mb = host_mailbox(&mb_d);
    for (int i = 0; i < 5; ++i) host_out[i] = mb[MB_SCHED + i];
}

pmmf_status schedule_stage(const int64_t *coff, int64_t mm, const int64_t *mm_dev, int64_t s,
                           int64_t core, double eta, DBuf<int64_t> &e, DBuf<int64_t> &roff,
                           int64_t *host_out, cudaStream_t st) {
    PMMF_TRY(schedule_launch(coff, mm, mm_dev, s, core, eta, e, roff, st));
    PMMF_CUDA_TRY(cudaStreamSynchronize(st));
    schedule_read(host_out);
    return PMMF_OK;
}

pmmf_status one_cluster(const int32_t *act, int64_t s, StageClusters &out, int32_t *cl,
                        int32_t *loc, cudaStream_t st) {
    PMMF_TRY(out.members.alloc(s, st));
    PMMF_TRY(out.coff.alloc(2, st));
    k_one_cluster<<<grid_for(s, 256), 256, 0, st>>>(act, s, out.members.p, cl, loc, out.coff.p);
    PMMF_TRY(launched("one_cluster"));
    out.m = 1;
    return PMMF_OK;
}

}  // namespace pmmf
