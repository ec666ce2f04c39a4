// prim.cu -- data-movement primitives of the pMMF library: scans, stable
// counting sort / radix sort, CSR construction and validation, reductions.
#include <cstdlib>
#include <algorithm>
#include <mutex>
#include <vector>
#include <string>

#include <cooperative_groups.h>

#include "common.cuh"

namespace pmmf {

std::atomic<uint64_t> g_launches{0};
std::atomic<uint64_t> g_allocs{0};

namespace {
thread_local std::string t_last_error;
std::atomic<int64_t> g_alloc_countdown{-1};
std::once_flag g_alloc_env_once;
}  // namespace

void set_error(const std::string &msg) { t_last_error = msg; }

// Page-locked, device-mapped host words (one set per host thread): kernels
// write small results straight into them, so a readback is a wait on the
// stream or an event instead of a copy.  Allocated once per thread and kept
// for the life of the process.
int64_t *host_mailbox(int64_t **dev) {
    thread_local int64_t *h = nullptr;
    thread_local int64_t *d = nullptr;
    if (!h) {
        void *p = nullptr;
        if (cudaHostAlloc(&p, sizeof(int64_t) * MAILBOX_SLOTS,
                          cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess) {
            cudaGetLastError();
            set_error("page-locked host allocation failed");
            return nullptr;
        }
        void *dp = nullptr;
        if (cudaHostGetDevicePointer(&dp, p, 0) != cudaSuccess) {
            cudaGetLastError();
            cudaFreeHost(p);
            set_error("mapping page-locked host memory failed");
            return nullptr;
        }
        h = (int64_t *)p;
        d = (int64_t *)dp;
    }
    *dev = d;
    return h;
}
const char *last_error_cstr() { return t_last_error.c_str(); }

// Test hook: PMMF_FAIL_ALLOC_AFTER=N makes the (N+1)-th device allocation of
// the process fail with PMMF_ERR_OOM, to exercise the cleanup paths.
pmmf_status dev_alloc(void **p, size_t bytes, cudaStream_t st) {
    std::call_once(g_alloc_env_once, [] {
        const char *e = std::getenv("PMMF_FAIL_ALLOC_AFTER");
        if (e && *e) g_alloc_countdown.store(std::atoll(e));
    });
    *p = nullptr;
    int64_t c = g_alloc_countdown.load();
    if (c >= 0) {
        if (c == 0) {
            set_error("device allocation failed (PMMF_FAIL_ALLOC_AFTER test hook)");
            return PMMF_ERR_OOM;
        }
        g_alloc_countdown.fetch_sub(1);
    }
    g_allocs.fetch_add(1, std::memory_order_relaxed);
    cudaError_t e = cudaMallocAsync(p, bytes, st);
    if (e != cudaSuccess) {
        *p = nullptr;
        set_error(std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? PMMF_ERR_OOM : PMMF_ERR_CUDA;
    }
    return PMMF_OK;
}

namespace {
thread_local bool t_free_sync = false;
}
void set_free_sync(bool on) { t_free_sync = on; }

// Buffers are released stream-ordered on the stream that allocated them,
// except while a handle is torn down (the caller's stream may be gone by then).
void dev_free(void *p, cudaStream_t st) {
    if (!p) return;
    if (t_free_sync) cudaFree(p);
    else cudaFreeAsync(p, st);
}

// ---------------------------------------------------------------- scan

namespace {

constexpr int SCAN_THREADS = 512;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

template <class T>
__device__ int64_t block_exclusive_scan(int64_t v, int64_t *total) {
    __shared__ int64_t warp_tot[SCAN_THREADS / 32];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[w] = x;
    __syncthreads();
    if (w == 0) {
        int64_t t = lane < SCAN_THREADS / 32 ? warp_tot[lane] : 0;
        int64_t ti = t;
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, ti, o);
            if (lane >= o) ti += y;
        }
        if (lane < SCAN_THREADS / 32) warp_tot[lane] = ti - t;
        if (lane == 31) *total = ti;
    }
    __syncthreads();
    int64_t r = x - v + warp_tot[w];
    __syncthreads();
    return r;
}

// Longer inputs: one cooperative launch in three phases separated by grid
// barriers (tile sums; the tile sums scanned by block 0, partial[nb] = total;
// every tile scanned with its offset), each block taking tiles b, b + grid, ...
// Every read of 'in' (phase 1 reads all of it) precedes the first write of
// 'out', so the two may alias.
template <class T>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_coop(const T *in, int64_t *out, int64_t *out2,
                                                            int64_t n, int64_t nb, int64_t *partial) {
    namespace cg = cooperative_groups;
    cg::grid_group grid = cg::this_grid();
    __shared__ int64_t tot;
    for (int64_t b = blockIdx.x; b < nb; b += gridDim.x) {
        const int64_t base = b * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
        int64_t sum = 0;
        for (int q = 0; q < SCAN_ITEMS; ++q)
            if (base + q < n) sum += (int64_t)in[base + q];
        block_exclusive_scan<int64_t>(sum, &tot);
        if (threadIdx.x == 0) partial[b] = tot;
    }
    grid.sync();
    if (blockIdx.x == 0) {
        int64_t carry = 0;
        for (int64_t b0 = 0; b0 < nb; b0 += SCAN_THREADS) {
            const int64_t b = b0 + threadIdx.x;
            const int64_t v = b < nb ? partial[b] : 0;
            const int64_t ex = block_exclusive_scan<int64_t>(v, &tot);
            if (b < nb) partial[b] = ex + carry;
            carry += tot;
            __syncthreads();
        }
        if (threadIdx.x == 0) partial[nb] = carry;
    }
    grid.sync();
    for (int64_t b = blockIdx.x; b < nb; b += gridDim.x) {
        const int64_t base = b * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
        int64_t v[SCAN_ITEMS];
        int64_t sum = 0;
        for (int q = 0; q < SCAN_ITEMS; ++q) {
            v[q] = base + q < n ? (int64_t)in[base + q] : 0;
            sum += v[q];
        }
        int64_t ex = block_exclusive_scan<int64_t>(sum, &tot) + partial[b];
        for (int q = 0; q < SCAN_ITEMS; ++q) {
            if (base + q < n) {
                out[base + q] = ex;
                if (out2) out2[base + q] = ex;
            }
            ex += v[q];
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        out[n] = partial[nb];
        if (out2) out2[n] = partial[nb];
    }
}

// Short inputs: one CTA walks the tiles in order with a running carry (one
// launch instead of three).
template <class T>
__global__ void k_scan_one(const T *in, int64_t *out, int64_t *out2, int64_t n) {
    __shared__ int64_t tot;
    int64_t carry = 0;
    for (int64_t t0 = 0; t0 < n; t0 += SCAN_TILE) {
        const int64_t base = t0 + (int64_t)threadIdx.x * SCAN_ITEMS;
        int64_t v[SCAN_ITEMS];
        int64_t sum = 0;
        for (int q = 0; q < SCAN_ITEMS; ++q) {
            v[q] = base + q < n ? (int64_t)in[base + q] : 0;
            sum += v[q];
        }
        int64_t ex = block_exclusive_scan<int64_t>(sum, &tot) + carry;
        __syncthreads();  // reads of this tile precede its writes (aliasing)
        for (int q = 0; q < SCAN_ITEMS; ++q) {
            if (base + q < n) {
                out[base + q] = ex;
                if (out2) out2[base + q] = ex;
            }
            ex += v[q];
        }
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[n] = carry;
        if (out2) out2[n] = carry;
    }
}

template <class T>
pmmf_status scan_impl(const T *in, int64_t *out, int64_t *out2, int64_t n, cudaStream_t st) {
    if (n <= 0) {
        PMMF_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(int64_t), st));
        if (out2) PMMF_CUDA_TRY(cudaMemsetAsync(out2, 0, sizeof(int64_t), st));
        return PMMF_OK;
    }
    if (n <= 4 * SCAN_TILE) {
        k_scan_one<T><<<1, SCAN_THREADS, 0, st>>>(in, out, out2, n);
        return launched("scan_one");
    }
    const int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    DBuf<int64_t> part;
    PMMF_TRY(part.alloc(nb + 1, st));
    // co-resident blocks for the grid barriers (queried once per element type)
    static int resident = 0;
    if (resident == 0) {
        int dev = 0, nsm = 0, per = 0;
        PMMF_CUDA_TRY(cudaGetDevice(&dev));
        PMMF_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        PMMF_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_scan_coop<T>, SCAN_THREADS, 0));
        resident = std::max(1, nsm * per);
    }
    const unsigned g = (unsigned)std::min<int64_t>(nb, resident);
    const T *a_in = in;
    int64_t *a_out = out, *a_out2 = out2, *a_part = part.p;
    int64_t a_n = n, a_nb = nb;
    void *args[] = {&a_in, &a_out, &a_out2, &a_n, &a_nb, &a_part};
    PMMF_CUDA_TRY(cudaLaunchCooperativeKernel((const void *)k_scan_coop<T>, dim3(g), dim3(SCAN_THREADS),
                                              args, 0, st));
    return launched("scan");
}

}  // namespace

pmmf_status scan_i64(const int64_t *in, int64_t *out, int64_t n, cudaStream_t st) {
    return scan_impl<int64_t>(in, out, nullptr, n, st);
}
pmmf_status scan_i64_dup(const int64_t *in, int64_t *out, int64_t *out2, int64_t n, cudaStream_t st) {
    return scan_impl<int64_t>(in, out, out2, n, st);
}
pmmf_status scan_i32_to_i64(const int32_t *in, int64_t *out, int64_t n, cudaStream_t st) {
    return scan_impl<int32_t>(in, out, nullptr, n, st);
}

// ---------------------------------------------------------------- stable counting sort

namespace {


__global__ void k_sort_hist(const uint32_t *key, int64_t n, int64_t nbins, int64_t nblocks,
                            int64_t tile, int64_t *hist) {
    extern __shared__ int32_t sh[];
    for (int64_t b = threadIdx.x; b < nbins; b += blockDim.x) sh[b] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * tile;
    int64_t end = base + tile < n ? base + tile : n;
    for (int64_t i = base + threadIdx.x; i < end; i += blockDim.x) atomicAdd(&sh[key[i]], 1);
    __syncthreads();
    for (int64_t b = threadIdx.x; b < nbins; b += blockDim.x)
        hist[b * nblocks + blockIdx.x] = sh[b];
}

// One warp per tile walks the tile in order, 32 items at a time, so equal
// keys keep their input order.
__global__ void k_sort_scatter(const uint32_t *key, int64_t n, int64_t nbins, int64_t nblocks,
                               int64_t tile, const int64_t *offs, int32_t *perm) {
    extern __shared__ int32_t cnt[];
    int lane = threadIdx.x;
    for (int64_t b = lane; b < nbins; b += 32) cnt[b] = 0;
    __syncwarp();
    int64_t base = (int64_t)blockIdx.x * tile;
    int64_t end = base + tile < n ? base + tile : n;
    for (int64_t c = base; c < end; c += 32) {
        int64_t i = c + lane;
        bool ok = i < end;
        unsigned act = __ballot_sync(0xffffffffu, ok);
        if (ok) {
            uint32_t k = key[i];
            unsigned peers = __match_any_sync(act, k);
            unsigned lt = (1u << lane) - 1u;
            int rank = __popc(peers & lt);
            int64_t pos = offs[(int64_t)k * nblocks + blockIdx.x] + cnt[k] + rank;
            perm[pos] = (int32_t)i;
            __syncwarp(act);
            if ((peers & lt) == 0) cnt[k] += __popc(peers);
        }
        __syncwarp();
    }
}

constexpr int RADIX_BITS = 11;
constexpr uint32_t RADIX_MASK = (1u << RADIX_BITS) - 1u;

// First pass's digits (identity order).
__global__ void k_digit(const uint64_t *key, int64_t n, uint32_t *d) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        d[i] = (uint32_t)(key[i] & RADIX_MASK);
}

// next = cur o perm (cur NULL: the identity), and unless shift < 0 the next
// pass's digits in that order.
__global__ void k_compose(const int32_t *cur, const int32_t *perm, int64_t n, int32_t *next,
                          const uint64_t *key, int shift, uint32_t *d) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t x = cur ? cur[perm[i]] : perm[i];
        next[i] = x;
        if (shift >= 0) d[i] = (uint32_t)((key[x] >> shift) & RADIX_MASK);
    }
}

__global__ void k_iota(int32_t *p, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = (int32_t)i;
}

}  // namespace

pmmf_status iota_i32(int32_t *p, int64_t n, cudaStream_t st) {
    if (n <= 0) return PMMF_OK;
    k_iota<<<grid_for(n, 256), 256, 0, st>>>(p, n);
    return launched("iota");
}

pmmf_status stable_sort_by_key(const uint32_t *key, int64_t n, int64_t nbins, int32_t *perm,
                               cudaStream_t st) {
    if (n <= 0) return PMMF_OK;
    if (nbins * (int64_t)sizeof(int32_t) > 200 * 1024) {
        set_error("stable_sort_by_key: too many bins");
        return PMMF_ERR_UNSUPPORTED;
    }
    // one warp walks each tile in order; tiles small enough to give the GPU
    // many warps, large enough to keep the per-tile histograms under ~4M entries
    int64_t tile = 512;
    while (tile < n && nbins * ((n + tile - 1) / tile) > (int64_t(1) << 22)) tile *= 2;
    int64_t nblocks = (n + tile - 1) / tile;
    DBuf<int64_t> hist;
    PMMF_TRY(hist.alloc(nbins * nblocks + 1, st));
    size_t sh = sizeof(int32_t) * (size_t)nbins;
    PMMF_CUDA_TRY(allow_smem(k_sort_hist, sh));
    PMMF_CUDA_TRY(allow_smem(k_sort_scatter, sh));
    k_sort_hist<<<(unsigned)nblocks, 256, sh, st>>>(key, n, nbins, nblocks, tile, hist.p);
    PMMF_TRY(launched("sort_hist"));
    PMMF_TRY(scan_i64(hist.p, hist.p, nbins * nblocks, st));
    k_sort_scatter<<<(unsigned)nblocks, 32, sh, st>>>(key, n, nbins, nblocks, tile, hist.p, perm);
    PMMF_TRY(launched("sort_scatter"));
    return PMMF_OK;
}

pmmf_status radix_sort_u64(const uint64_t *key, int64_t n, int bits, int32_t *perm,
                           cudaStream_t st) {
    if (n <= 0) return PMMF_OK;
    if (bits <= 0) return iota_i32(perm, n, st);
    // LSD passes of RADIX_BITS bits; the permutation so far alternates
    // between 'other' and perm so that the last pass writes perm
    const int passes = (bits + RADIX_BITS - 1) / RADIX_BITS;
    DBuf<int32_t> other, tmp;
    DBuf<uint32_t> digit;
    PMMF_TRY(other.alloc(n, st));
    PMMF_TRY(tmp.alloc(n, st));
    PMMF_TRY(digit.alloc(n, st));
    k_digit<<<grid_for(n, 256), 256, 0, st>>>(key, n, digit.p);
    PMMF_TRY(launched("radix_digit"));
    const int32_t *cur = nullptr;
    for (int p = 0; p < passes; ++p) {
        PMMF_TRY(stable_sort_by_key(digit.p, n, int64_t(1) << RADIX_BITS, tmp.p, st));
        int32_t *next = ((passes - 1 - p) % 2 == 0) ? perm : other.p;
        const int shift = p + 1 < passes ? (p + 1) * RADIX_BITS : -1;
        k_compose<<<grid_for(n, 256), 256, 0, st>>>(cur, tmp.p, n, next, key, shift, digit.p);
        PMMF_TRY(launched("radix_compose"));
        cur = next;
    }
    return PMMF_OK;
}

// ---------------------------------------------------------------- CSR construction

namespace {

// One warp per row: count nonzero entries of a dense row.
__global__ void k_dense_count(const double *a, int64_t n, int64_t ld, int64_t *cnt) {
    int lane = threadIdx.x & 31;
    int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = w; r < n; r += nw) {
        int64_t c = 0;
        for (int64_t j = lane; j < n; j += 32) c += a[r * ld + j] != 0.0;
        c = warp_sum_i64(c);
        if (lane == 0) cnt[r] = c;
    }
}

__global__ void k_dense_write(const double *a, int64_t n, int64_t ld, const int64_t *rp,
                              int32_t *col, double *val) {
    int lane = threadIdx.x & 31;
    int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = w; r < n; r += nw) {
        int64_t o = rp[r];
        for (int64_t j0 = 0; j0 < n; j0 += 32) {
            int64_t j = j0 + lane;
            double v = j < n ? a[r * ld + j] : 0.0;
            unsigned m = __ballot_sync(0xffffffffu, v != 0.0);
            if (v != 0.0) {
                int64_t q = o + __popc(m & ((1u << lane) - 1u));
                col[q] = (int32_t)j;
                val[q] = v;
            }
            o += __popc(m);
        }
    }
}

__global__ void k_csr_count(int64_t n, const int64_t *rp, const double *v, int64_t *cnt) {
    int lane = threadIdx.x & 31;
    int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = w; r < n; r += nw) {
        int64_t c = 0;
        for (int64_t q = rp[r] + lane; q < rp[r + 1]; q += 32) c += v[q] != 0.0;
        c = warp_sum_i64(c);
        if (lane == 0) cnt[r] = c;
    }
}

__global__ void k_csr_write(int64_t n, const int64_t *rp, const int32_t *ci, const double *v,
                            const int64_t *orp, int32_t *col, double *val) {
    int lane = threadIdx.x & 31;
    int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = w; r < n; r += nw) {
        int64_t o = orp[r];
        for (int64_t q0 = rp[r]; q0 < rp[r + 1]; q0 += 32) {
            int64_t q = q0 + lane;
            double x = q < rp[r + 1] ? v[q] : 0.0;
            unsigned m = __ballot_sync(0xffffffffu, x != 0.0);
            if (x != 0.0) {
                int64_t d = o + __popc(m & ((1u << lane) - 1u));
                col[d] = ci[q];
                val[d] = x;
            }
            o += __popc(m);
        }
    }
}

// Structure (rows, ascending columns), finiteness and, with SYM, exact
// symmetry: the entry (y, x) must exist for every stored (x, y) and carry the
// same bits.
template <bool SYM>
__global__ void k_validate(int64_t n, const int64_t *rp, const int32_t *ci, const double *v,
                           unsigned *status) {
    int lane = threadIdx.x & 31;
    int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned bad = 0;
    for (int64_t r = w; r < n; r += nw) {
        int64_t b = rp[r], e = rp[r + 1];
        if (e < b) { bad |= ST_BAD_CSR; continue; }
        for (int64_t q = b + lane; q < e; q += 32) {
            int32_t y = ci[q];
            double x = v[q];
            if (y < 0 || y >= n || (q > b && ci[q - 1] >= y)) { bad |= ST_BAD_CSR; continue; }
            if (!isfinite(x)) bad |= ST_NONFINITE;
            if (!SYM) continue;
            int64_t lo = rp[y], hi = rp[y + 1];
            bool found = false;
            while (lo < hi) {
                int64_t mid = (lo + hi) >> 1;
                int32_t cm = ci[mid];
                if (cm < r) lo = mid + 1;
                else if (cm > r) hi = mid;
                else { found = __double_as_longlong(v[mid]) == __double_as_longlong(x); break; }
            }
            if (!found) bad |= ST_NOT_SYMMETRIC;
        }
    }
    for (int o = 16; o > 0; o >>= 1) bad |= __shfl_xor_sync(0xffffffffu, bad, o);
    if (lane == 0 && bad) atomicOr(status, bad);
}

constexpr int RED_BLOCKS = 304;

__global__ void k_sumsq_partial(const double *v, int64_t n, double *part) {
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        s = __fma_rn(v[i], v[i], s);
    s = warp_sum(s);
    __shared__ double ws[32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += ws[q];
        part[blockIdx.x] = t;
    }
}

// Sum of the partials in a fixed tree order (one block, one thread per
// partial, np <= blockDim.x <= 1024): deterministic, no serial chain.
__global__ void k_sum_tree(const double *part, int np, double *out) {
    double t = threadIdx.x < (unsigned)np ? part[threadIdx.x] : 0.0;
    t = warp_sum(t);
    __shared__ double ws[32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x < 32) {
        t = threadIdx.x < (blockDim.x >> 5) ? ws[threadIdx.x] : 0.0;
        t = warp_sum(t);
        if (threadIdx.x == 0) *out = t;
    }
}

}  // namespace

pmmf_status dense_to_csr(const double *a, int64_t n, int64_t ld, DBuf<int64_t> &rowptr,
                         DBuf<int32_t> &col, DBuf<double> &val, cudaStream_t st) {
    PMMF_TRY(rowptr.alloc(n + 1, st));
    k_dense_count<<<grid_for(n * 32, 256), 256, 0, st>>>(a, n, ld, rowptr.p);
    PMMF_TRY(launched("dense_count"));
    PMMF_TRY(scan_i64(rowptr.p, rowptr.p, n, st));
    int64_t nnz = 0;
    PMMF_CUDA_TRY(cudaMemcpyAsync(&nnz, rowptr.p + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    PMMF_CUDA_TRY(cudaStreamSynchronize(st));
    PMMF_TRY(col.alloc(nnz, st));
    PMMF_TRY(val.alloc(nnz, st));
    k_dense_write<<<grid_for(n * 32, 256), 256, 0, st>>>(a, n, ld, rowptr.p, col.p, val.p);
    return launched("dense_write");
}

pmmf_status csr_drop_zeros(int64_t n, const int64_t *rp, const int32_t *ci, const double *v,
                           DBuf<int64_t> &rowptr, DBuf<int32_t> &col, DBuf<double> &val,
                           cudaStream_t st) {
    PMMF_TRY(rowptr.alloc(n + 1, st));
    k_csr_count<<<grid_for(n * 32, 256), 256, 0, st>>>(n, rp, v, rowptr.p);
    PMMF_TRY(launched("csr_count"));
    PMMF_TRY(scan_i64(rowptr.p, rowptr.p, n, st));
    int64_t nnz = 0;
    PMMF_CUDA_TRY(cudaMemcpyAsync(&nnz, rowptr.p + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    PMMF_CUDA_TRY(cudaStreamSynchronize(st));
    PMMF_TRY(col.alloc(nnz, st));
    PMMF_TRY(val.alloc(nnz, st));
    k_csr_write<<<grid_for(n * 32, 256), 256, 0, st>>>(n, rp, ci, v, rowptr.p, col.p, val.p);
    return launched("csr_write");
}

pmmf_status validate_csr(int64_t n, const int64_t *rp, const int32_t *ci, const double *v,
                         unsigned *status, cudaStream_t st, bool symmetry) {
    if (symmetry) k_validate<true><<<grid_for(n * 32, 256), 256, 0, st>>>(n, rp, ci, v, status);
    else k_validate<false><<<grid_for(n * 32, 256), 256, 0, st>>>(n, rp, ci, v, status);
    return launched("validate");
}

pmmf_status sum_squares(const double *v, int64_t n, double *out, cudaStream_t st) {
    DBuf<double> part;
    PMMF_TRY(part.alloc(RED_BLOCKS, st));
    k_sumsq_partial<<<RED_BLOCKS, 256, 0, st>>>(v, n, part.p);
    PMMF_TRY(launched("sumsq_partial"));
    k_sum_tree<<<1, (RED_BLOCKS + 31) / 32 * 32, 0, st>>>(part.p, RED_BLOCKS, out);
    return launched("sum_tree");
}

}  // namespace pmmf

// ---------------------------------------------------------------- profiler

namespace pmmf {
namespace {

struct ProfRec {
    int family;
    cudaEvent_t a, b;
    double bytes, flops;
};

std::mutex g_prof_mu;
unsigned g_prof_mask = 0;
std::vector<ProfRec> g_prof;
std::vector<cudaEvent_t> g_prof_pool;
thread_local cudaEvent_t t_open = nullptr;

cudaEvent_t prof_event() {
    if (!g_prof_pool.empty()) {
        cudaEvent_t e = g_prof_pool.back();
        g_prof_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

}  // namespace

bool prof_on(int family) { return (g_prof_mask & (1u << family)) != 0; }

void prof_begin(int family, cudaStream_t st) {
    if (!(g_prof_mask & (1u << family))) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    t_open = prof_event();
    cudaEventRecord(t_open, st);
}

void prof_end(int family, cudaStream_t st, double bytes, double flops) {
    if (!(g_prof_mask & (1u << family)) || !t_open) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    cudaEvent_t b = prof_event();
    cudaEventRecord(b, st);
    g_prof.push_back(ProfRec{family, t_open, b, bytes, flops});
    t_open = nullptr;
}

namespace {
struct TuneTable {
    std::mutex mu;
    std::vector<std::pair<int64_t, int>> b[TUNE_COUNT];   // (bucket bound, value), ascending
};
TuneTable &tune_table() {
    static TuneTable t;
    return t;
}
}  // namespace

int tuned(int param, int64_t size, int fallback) {
    if (param < 0 || param >= TUNE_COUNT) return fallback;
    TuneTable &t = tune_table();
    std::lock_guard<std::mutex> g(t.mu);
    for (const auto &e : t.b[param])
        if (size <= e.first) return e.second;
    return fallback;
}

}  // namespace pmmf

extern "C" {

/* Profiling hooks (declared in include/pmmf.h). */
pmmf_status pmmf_profile_begin(unsigned family_mask) {
    std::lock_guard<std::mutex> lk(pmmf::g_prof_mu);
    for (auto &r : pmmf::g_prof) {
        pmmf::g_prof_pool.push_back(r.a);
        pmmf::g_prof_pool.push_back(r.b);
    }
    pmmf::g_prof.clear();
    pmmf::g_prof_mask = family_mask;
    return PMMF_OK;
}

pmmf_status pmmf_profile_records(int64_t cap, int32_t *family, double *ms, double *bytes,
                                 double *flops, int64_t *count) {
    if (!count || (cap > 0 && (!family || !ms || !bytes || !flops))) {
        pmmf::set_error("NULL output");
        return PMMF_ERR_INVALID_ARG;
    }
    cudaDeviceSynchronize();
    std::lock_guard<std::mutex> lk(pmmf::g_prof_mu);
    *count = (int64_t)pmmf::g_prof.size();
    for (int64_t i = 0; i < cap && i < *count; ++i) {
        const auto &r = pmmf::g_prof[(size_t)i];
        float t = 0.f;
        cudaEventElapsedTime(&t, r.a, r.b);
        family[i] = r.family;
        ms[i] = t;
        bytes[i] = r.bytes;
        flops[i] = r.flops;
    }
    return PMMF_OK;
}

pmmf_status pmmf_profile_end(double *ms, int64_t *launches, double *bytes, double *flops) {
    cudaDeviceSynchronize();
    std::lock_guard<std::mutex> lk(pmmf::g_prof_mu);
    for (int f = 0; f < pmmf::KF_COUNT; ++f) {
        ms[f] = 0.0;
        launches[f] = 0;
        bytes[f] = 0.0;
        flops[f] = 0.0;
    }
    for (auto &r : pmmf::g_prof) {
        float t = 0.f;
        cudaEventElapsedTime(&t, r.a, r.b);
        ms[r.family] += t;
        launches[r.family] += 1;
        bytes[r.family] += r.bytes;
        flops[r.family] += r.flops;
        pmmf::g_prof_pool.push_back(r.a);
        pmmf::g_prof_pool.push_back(r.b);
    }
    pmmf::g_prof.clear();
    pmmf::g_prof_mask = 0;
    return PMMF_OK;
}

}  // extern "C"

extern "C" {

pmmf_status pmmf_set_tuning(int param, int64_t max_size, int value) {
    using namespace pmmf;
    if (param < 0 || param >= TUNE_COUNT || max_size < 1 || value < 0 ||
        (value == 0 && param != TUNE_MIXED_ACTIVE) ||
        (value > 32 && param != TUNE_REACH_CLUSTERS) ||
        (param == TUNE_SELECT_WARPS && value != 8 && value != 16) ||
        (param == TUNE_ROWS_KERNEL && value != 1 && value != 2) ||
        (param == TUNE_DENSE_TILES && value != 1 && value != 2) ||
        (param == TUNE_SELECT_DSM && value != 1 && value != 2) ||
        (param == TUNE_APPLY_FUSED && value != 1 && value != 2) ||
        (param == TUNE_TC_GRAM && value != 1 && value != 2) ||
        (param == TUNE_SELECT_BLOCKS && (value < 2 || value > 4))) {
        set_error("pmmf_set_tuning: unknown parameter or value out of range");
        return PMMF_ERR_INVALID_ARG;
    }
    TuneTable &t = tune_table();
    std::lock_guard<std::mutex> g(t.mu);
    auto &v = t.b[param];
    for (auto &e : v)
        if (e.first == max_size) {
            e.second = value;
            return PMMF_OK;
        }
    v.emplace_back(max_size, value);
    std::sort(v.begin(), v.end());
    return PMMF_OK;
}

void pmmf_clear_tuning(void) {
    using namespace pmmf;
    TuneTable &t = tune_table();
    std::lock_guard<std::mutex> g(t.mu);
    for (auto &v : t.b) v.clear();
}

}  // extern "C"
