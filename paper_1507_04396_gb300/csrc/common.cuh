// common.cuh -- internal helpers of the pMMF CUDA library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>

#include "pmmf.h"

namespace pmmf {

// ---------------------------------------------------------------- errors

void set_error(const std::string &msg);
extern std::atomic<uint64_t> g_launches;
extern std::atomic<uint64_t> g_allocs;   // device allocations requested (dev_alloc)

struct Err {
    pmmf_status st = PMMF_OK;
    explicit operator bool() const { return st != PMMF_OK; }
};

#define PMMF_CUDA_TRY(expr)                                                              \
    do {                                                                                \
        cudaError_t e__ = (expr);                                                       \
        if (e__ != cudaSuccess) {                                                       \
            ::pmmf::set_error(std::string(#expr) + ": " + cudaGetErrorString(e__));     \
            return e__ == cudaErrorMemoryAllocation ? PMMF_ERR_OOM : PMMF_ERR_CUDA;     \
        }                                                                               \
    } while (0)

#define PMMF_TRY(expr)                          \
    do {                                        \
        pmmf_status s__ = (expr);               \
        if (s__ != PMMF_OK) return s__;         \
    } while (0)

// Count a kernel launch and surface launch-configuration errors.
inline pmmf_status launched(const char *what) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error(std::string(what) + ": " + cudaGetErrorString(e));
        return PMMF_ERR_CUDA;
    }
    return PMMF_OK;
}

inline unsigned grid_for(int64_t items, int per_block, int64_t cap = 152 * 64) {
    int64_t g = (items + per_block - 1) / per_block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (unsigned)g;
}

// ---------------------------------------------------------------- launch tuning

// Launch parameters that an offline sweep may set per cluster-size bucket
// (pmmf_set_tuning); tuned(param, size, fallback) returns the value of the
// smallest bucket whose bound is >= size, else fallback.
// Opt a kernel in to `bytes` of dynamic shared memory.  The default limit of
// 48 KB holds static and dynamic shared memory together, so the opt-in is
// taken from 32 KB on (the kernels' static shared memory is far below 16 KB);
// a kernel whose dynamic size sits just under 48 KB would otherwise fail to
// launch.
template <class K>
inline cudaError_t allow_smem(K kern, size_t bytes) {
    return bytes > 32 * 1024
               ? cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes)
               : cudaSuccess;
}

enum TuneParam : int {
    TUNE_ROWS_WARPS = 0, TUNE_GRAM_WARPS = 1, TUNE_SELECT_WARPS = 2, TUNE_PASS1_ESTIMATE = 3,
    TUNE_REACH_CLUSTERS = 4, TUNE_ROWS_KERNEL = 5, TUNE_DENSE_TILES = 6, TUNE_SELECT_DSM = 7,
    TUNE_APPLY_FUSED = 8, TUNE_SELECT_BLOCKS = 9,
    TUNE_MIXED_ACTIVE = 10, TUNE_TC_GRAM = 11, TUNE_COUNT = 12
};
int tuned(int param, int64_t size, int fallback);

// ---------------------------------------------------------------- profiling

// Kernel families that can be timed with CUDA events on their launch stream.
enum KFamily : int { KF_PARTITION = 0, KF_GRAM = 1, KF_SELECT = 2, KF_ROWS = 3, KF_APPLY = 4,
                     KF_OTHER = 5, KF_COUNT = 6 };

// Bracket one launch: prof_begin before, prof_end after with the launch's
// algorithmic bytes and flops.  Both are no-ops unless the family is enabled.
void prof_begin(int family, cudaStream_t st);
void prof_end(int family, cudaStream_t st, double bytes, double flops);
bool prof_on(int family);

// Device status bits (written by kernels, read by the host after a sync).
enum : unsigned {
    ST_NOT_SYMMETRIC = 1u,
    ST_NONFINITE = 2u,
    ST_BAD_CSR = 4u,
    ST_ROW_TOO_LONG = 8u,
    ST_NOT_SPD = 16u,
    ST_CLUSTER_TOO_BIG = 32u,
    ST_NOT_CONVERGED = 64u,
    ST_BAD_LABEL = 128u,
    ST_TIMEOUT = 256u,        // a kernel's bounded wait ran out
};

// ---------------------------------------------------------------- rotations

// One Givens rotation found by Algorithm 2, stored with cluster-local
// indices: x_li' = c x_li - s x_lj, x_lj' = s x_li + c x_lj.
struct Rot2 {
    int32_t li, lj;
    double c, s;
};

// Step-order record kept for export.
struct RotRec {
    int32_t li, lj, le, lvl;  // tuple, eliminated, dependency level
    double c, s;
};

// ---------------------------------------------------------------- arithmetic

// The canonical rotation of a pair (fixed operation order; no contraction):
//   a' = fma(c, a, -(s b)),  b' = fma(s, a, c b)
__device__ __forceinline__ void rot_pair(double c, double s, double a, double b, double &na,
                                         double &nb) {
    na = __fma_rn(c, a, -__dmul_rn(s, b));
    nb = __fma_rn(s, a, __dmul_rn(c, b));
}

// One output of rot_pair, the same bits: a' when first, else b'.
__device__ __forceinline__ double rot_pair_one(double c, double s, double a, double b, bool first) {
    return first ? __fma_rn(c, a, -__dmul_rn(s, b)) : __fma_rn(s, a, __dmul_rn(c, b));
}

// Transposed rotation: a' = fma(c, a, s b),  b' = fma(-s, a, c b)
__device__ __forceinline__ void rot_pair_t(double c, double s, double a, double b, double &na,
                                           double &nb) {
    na = __fma_rn(c, a, __dmul_rn(s, b));
    nb = __fma_rn(-s, a, __dmul_rn(c, b));
}

// The bits of a double and back, moved by inline PTX.  The move is opaque to
// the compiler, so integer tests on the bits stay integer instructions; an
// equivalent bit test written in C++ may be turned back into an FP64 compare
// or absolute value, and on GB300 every FP64 instruction takes a share of the
// SM's small FP64 pipe (one warp instruction per ~19 cycles per SM).
__device__ __forceinline__ unsigned long long f64_bits(double x) {
    unsigned long long u;
    asm("mov.b64 %0, %1;" : "=l"(u) : "d"(x));
    return u;
}
__device__ __forceinline__ double f64_from_bits(unsigned long long u) {
    double x;
    asm("mov.b64 %0, %1;" : "=d"(x) : "l"(u));
    return x;
}
constexpr unsigned long long F64_ABS = 0x7fffffffffffffffull;

// x != 0.0 tested on the bits (integer pipe).
__device__ __forceinline__ bool nonzero_bits(double x) { return (f64_bits(x) << 1) != 0ull; }

// x > 0.0 on the bits, for x not NaN.
__device__ __forceinline__ bool pos_bits(double x) {
    const unsigned long long u = f64_bits(x);
    return (u >> 63) == 0 && u != 0ull;
}

// x < y on the bits, for x, y not NaN: magnitudes order like their bits, so
// map the sign-magnitude pattern to an unsigned order; +0 and -0 are equal.
__device__ __forceinline__ bool lt_bits(double x, double y) {
    const unsigned long long a = f64_bits(x), b = f64_bits(y);
    if (((a | b) << 1) == 0ull) return false;
    const unsigned long long ka = (a >> 63) ? ~a : (a | 0x8000000000000000ull);
    const unsigned long long kb = (b >> 63) ? ~b : (b | 0x8000000000000000ull);
    return ka < kb;
}

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ int64_t warp_sum_i64(int64_t v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ---------------------------------------------------------------- readbacks

// Page-locked host words mapped into the device's address space (per host
// thread); returns the host view, *dev the device view, NULL on failure.
// Slot ranges: MB_SCHED for the stage schedule, MB_PASS2 for the blocked
// update's sizes.  A kernel writes a range; the host reads it after waiting
// for that kernel's stream or event.
enum : int { MB_SCHED = 0, MB_PASS2 = 8, MAILBOX_SLOTS = 16 };
int64_t *host_mailbox(int64_t **dev);

// ---------------------------------------------------------------- device buffers

struct Arena;  // tracks allocations so an error path frees everything

pmmf_status dev_alloc(void **p, size_t bytes, cudaStream_t st);
void dev_free(void *p, cudaStream_t st);
void set_free_sync(bool on);

template <class T>
struct DBuf {
    T *p = nullptr;
    int64_t n = 0;
    cudaStream_t st = nullptr;
    DBuf() = default;
    DBuf(const DBuf &) = delete;
    DBuf &operator=(const DBuf &) = delete;
    DBuf(DBuf &&o) noexcept { *this = std::move(o); }
    DBuf &operator=(DBuf &&o) noexcept {
        if (this != &o) {
            reset();
            p = o.p; n = o.n; st = o.st;
            o.p = nullptr; o.n = 0;
        }
        return *this;
    }
    ~DBuf() { reset(); }
    void reset() {
        if (p) dev_free(p, st);
        p = nullptr;
        n = 0;
    }
    pmmf_status alloc(int64_t count, cudaStream_t s) {
        reset();
        st = s;
        n = count;
        if (count <= 0) return PMMF_OK;
        return dev_alloc((void **)&p, sizeof(T) * (size_t)count, s);
    }
    pmmf_status zeros(int64_t count, cudaStream_t s) {
        PMMF_TRY(alloc(count, s));
        if (count > 0) PMMF_CUDA_TRY(cudaMemsetAsync(p, 0, sizeof(T) * (size_t)count, s));
        return PMMF_OK;
    }
};

// ---------------------------------------------------------------- primitives (prim.cu)

// Exclusive scan of int64 counts: out[i] = sum_{j<i} in[j], out[n] = total.
// in may alias out (in place, n+1 slots).  tmp is managed internally.
pmmf_status scan_i64(const int64_t *in, int64_t *out, int64_t n, cudaStream_t st);
// The same, the result written to out and to out2 (which must not alias in).
pmmf_status scan_i64_dup(const int64_t *in, int64_t *out, int64_t *out2, int64_t n, cudaStream_t st);
// Same for int32 input, int64 output.
pmmf_status scan_i32_to_i64(const int32_t *in, int64_t *out, int64_t n, cudaStream_t st);

// Stable counting sort: perm receives the positions 0..n-1 of the input
// ordered by key (ascending), equal keys in input order.  key < nbins.
pmmf_status stable_sort_by_key(const uint32_t *key, int64_t n, int64_t nbins, int32_t *perm,
                               cudaStream_t st);

// Stable LSD radix sort of 64-bit keys (keys' low 'bits' bits significant).
pmmf_status radix_sort_u64(const uint64_t *key, int64_t n, int bits, int32_t *perm,
                           cudaStream_t st);

pmmf_status dense_to_csr(const double *a, int64_t n, int64_t ld, DBuf<int64_t> &rowptr,
                         DBuf<int32_t> &col, DBuf<double> &val, cudaStream_t st);
pmmf_status csr_drop_zeros(int64_t n, const int64_t *rp, const int32_t *ci, const double *v,
                           DBuf<int64_t> &rowptr, DBuf<int32_t> &col, DBuf<double> &val,
                           cudaStream_t st);
// Structure (rows monotone, columns in range and ascending) and finiteness;
// with symmetry, also exact symmetry (every (i, j, x) has (j, i, x) stored).
pmmf_status validate_csr(int64_t n, const int64_t *rp, const int32_t *ci, const double *v,
                         unsigned *status, cudaStream_t st, bool symmetry = true);
pmmf_status sum_squares(const double *v, int64_t n, double *out, cudaStream_t st);
pmmf_status iota_i32(int32_t *p, int64_t n, cudaStream_t st);

}  // namespace pmmf
