// tcgram.cu -- the reduced-precision Gram matrices of the shortlist search on
// the fifth-generation tensor cores: tcgen05.mma with the accumulators in
// tensor memory, the operands moved by TMA into 128-byte-swizzled shared
// memory on an mbarrier pipeline.
//
// One CTA per 128 x 64 tile (rows a0.., columns b0.., b0 + 63 >= a0) of one
// cluster's Gram block computes G~ = hi hi^T + hi lo^T + lo hi^T, where hi
// and lo are the TF32 or BF16 split of the cluster's rows (hi = round(x),
// lo = round(x - hi)).  The s terms of every entry are cut into chunks of 16:
// the tensor cores accumulate a chunk's 48 products in FP32 into a buffer of
// its own in tensor memory (6 MMAs of K = 8 for TF32, 3 of K = 16 for BF16),
// and the epilogue warps add the chunk sums into a compensated FP32 pair per
// entry (TwoSum; the cascaded summation Sum2 of Ogita, Rump and Oishi) while
// the tensor cores fill the next buffers.  Chunking and summation are those of
// the warp-level kernel, so the certified error bound of the shortlist holds
// unchanged.
//
// Roles (10 warps): warp 0 allocates tensor memory, its lane 0 issues the TMA
// loads; lane 0 of warp 1 issues the MMAs; warps 2-9 drain the buffers (warp w
// reads tensor-memory lanes 32 (w % 4) .. + 31, i.e. tile rows, and columns
// 32 ((w - 2) / 4) .. + 31, its compensated pairs in registers).  Where the
// rows b0.. lie inside the rows a0.. (the tiles on the diagonal) the B
// operand is read from the A tile.  Every mbarrier wait is bounded: one that runs
// out raises a CTA-wide abort flag, the other roles leave their loops, issued
// copies and MMAs are waited for (bounded) and tensor memory is freed; the
// status word gets ST_TIMEOUT.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <vector>

#include "dense.cuh"
#include "mixed.cuh"

namespace pmmf {
namespace {

constexpr int TC_M = 128;                         // tile rows = MMA M
constexpr int TC_N = 64;                          // tile columns = MMA N
constexpr int TC_ROWB = 128;                      // bytes of K per row and stage (the swizzle span)
constexpr int TC_STAGES = 4;
constexpr int TC_A_BYTES = TC_M * TC_ROWB;        // one operand tile of rows a0..: 16 KB
constexpr int TC_B_BYTES = TC_N * TC_ROWB;        // of rows b0..: 8 KB
constexpr int TC_STAGE_BYTES = 2 * (TC_A_BYTES + TC_B_BYTES);   // hi and lo of both
constexpr int TC_BUFS = 8;                        // chunk buffers of TC_N columns
constexpr int TC_TMEM_COLS = TC_BUFS * TC_N;      // 512: all of the SM's tensor memory
constexpr int TC_CHUNK = 16;                      // terms per FP32 chunk
constexpr int TC_EPI_WARPS = 8;
constexpr int TC_THREADS = 32 * (2 + TC_EPI_WARPS);
constexpr size_t TC_SMEM = (size_t)TC_STAGES * TC_STAGE_BYTES + 1024;   // + alignment slack
constexpr long long TC_WAIT_CYCLES = 1ll << 31;   // ~1 s at the SM clock

__device__ __forceinline__ uint32_t saddr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor of a K-major operand in the 128-byte
// swizzle layout that TMA writes: rows of 128 bytes, groups of 8 rows 1024
// bytes apart (stride byte offset), the leading byte offset unused by this
// layout, descriptor version 1, swizzle mode 2 (128 bytes).  The start address
// of the K step j of a stage is the tile's address + 32 j bytes.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t a) {
    return (uint64_t)((a & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor: FP32 accumulator (bits 4-5 = 1), A and B TF32 (2)
// or BF16 (1) in bits 7-9 and 10-12, both K-major (bits 15, 16 = 0), N >> 3 in
// bits 17-22, M >> 4 in bits 24-28.
template <int PREC>
__host__ __device__ constexpr uint32_t tc_idesc() {
    return (1u << 4) | ((PREC == PMMF_PREC_BF16 ? 1u : 2u) << 7) |
           ((PREC == PMMF_PREC_BF16 ? 1u : 2u) << 10) | ((uint32_t)(TC_N >> 3) << 17) |
           ((uint32_t)(TC_M >> 4) << 24);
}

template <int PREC>
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, int acc) {
    if (PREC == PMMF_PREC_BF16)
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
            "l"(a), "l"(b), "r"(idesc), "r"(acc)
            : "memory");
    else
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
            "l"(a), "l"(b), "r"(idesc), "r"(acc)
            : "memory");
}

// The mbarrier receives one arrival when every tcgen05 operation this thread
// issued before has completed.
__device__ __forceinline__ void tc_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     saddr(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Issue the load of 32 consecutive 32-bit columns of this thread's
// tensor-memory lane; the registers are valid only after tmem_wait32.
__device__ __forceinline__ void tmem_ld32(uint32_t ta, uint32_t (&r)[32]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(ta)
                 : "memory");
}

// Wait for this thread's tensor-memory loads.  The registers pass through
// the statement, so no use of them can be scheduled before it.
__device__ __forceinline__ void tmem_wait32(uint32_t (&r)[32]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
                 :
                 : "memory");
}

// Packed FP32 pairs (Blackwell's f32x2 arithmetic): each half is the IEEE
// FP32 operation rounded to nearest, so two_sum_acc2 computes exactly what
// two_sum_acc computes on each half, with half the instructions.
__device__ __forceinline__ uint64_t f2_add(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t f2_sub(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t f2_pack(uint32_t lo, uint32_t hi) {
    uint64_t d;
    asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "r"(lo), "r"(hi));
    return d;
}
__device__ __forceinline__ void two_sum_acc2(uint64_t &hi, uint64_t &lo, uint64_t x) {
    const uint64_t s = f2_add(hi, x);
    const uint64_t bp = f2_sub(s, hi);
    const uint64_t err = f2_add(f2_sub(hi, f2_sub(s, bp)), f2_sub(x, bp));
    hi = s;
    lo = f2_add(lo, err);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(bar)) : "memory");
}

// Bounded wait for the phase of parity `parity`.  With `abort`, a wait that
// runs out raises the flag and one that sees it raised gives up; without,
// only the time bound applies (the clean-up waits).
__device__ __forceinline__ bool tc_wait(uint64_t *bar, uint32_t parity, volatile int *abort) {
    const uint32_t a = saddr(bar);
    const long long t0 = clock64();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if (abort && *abort) return false;
        if (clock64() - t0 > TC_WAIT_CYCLES) {
            if (abort) *abort = 1;
            return false;
        }
    }
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3}], [%4];" ::"r"(saddr(dst)),
        "l"(map), "r"(x), "r"(y), "r"(saddr(bar))
        : "memory");
}

template <int PREC>
__global__ void __launch_bounds__(TC_THREADS, 1)
k_tc_gram5(const __grid_constant__ CUtensorMap mah, const __grid_constant__ CUtensorMap mal,
           const __grid_constant__ CUtensorMap mbh, const __grid_constant__ CUtensorMap mbl, int64_t sp, const int64_t *coff, const int64_t *goff, const int32_t *tu,
           const int32_t *ta, const int32_t *tb, float *G, unsigned *status) {
    constexpr int EB = PREC == PMMF_PREC_BF16 ? 2 : 4;   // bytes per element
    constexpr int SPC = EB / 2;                          // 32-byte K steps per 16-term chunk
    constexpr int CPB = 8 / EB;                          // chunks per stage (128 bytes of K)
    constexpr int ELEMS = TC_ROWB / EB;                  // elements of K per stage
    extern __shared__ unsigned char tc_raw[];
    __shared__ __align__(8) uint64_t full[TC_STAGES], empty[TC_STAGES], tfull[TC_BUFS],
        tempty[TC_BUFS], drain;
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    unsigned char *sm = (unsigned char *)(((uintptr_t)tc_raw + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int64_t u = tu[blockIdx.x];
    const int64_t base = coff[u];
    const int c = (int)(coff[u + 1] - base);
    const int a0 = ta[blockIdx.x] * TC_M, b0 = tb[blockIdx.x] * TC_N;
    // rows b0.. inside rows a0..: B is read from the A tile (row offset bin)
    const bool inner = b0 >= a0 && b0 + TC_N <= a0 + TC_M;
    const uint32_t bin = (uint32_t)(b0 - a0) * TC_ROWB;
    const int nchunks = (int)((sp + TC_CHUNK - 1) / TC_CHUNK);
    const int nblk = (nchunks + CPB - 1) / CPB;
    volatile int *abort = &s_abort;
    if (tid == 0) {
        for (int q = 0; q < TC_STAGES; ++q) {
            mbar_init(&full[q], 1);
            mbar_init(&empty[q], 1);
        }
        for (int q = 0; q < TC_BUFS; ++q) {
            mbar_init(&tfull[q], 1);
            mbar_init(&tempty[q], TC_EPI_WARPS);
        }
        mbar_init(&drain, 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (wid == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         saddr(&s_tmem)),
                     "r"(TC_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;

    if (wid == 0) {
        if (lane == 0) {
            // ---- producer: stage kb holds K bytes [128 kb, 128 kb + 128) of
            // the operand tiles (those of rows a0.. only when B lies inside)
            const uint32_t bytes = inner ? 2u * TC_A_BYTES : (uint32_t)TC_STAGE_BYTES;
            const int ya = (int)(base + a0), yb = (int)(base + b0);
            int kb = 0;
            for (; kb < nblk; ++kb) {
                const int st = kb % TC_STAGES, n = kb / TC_STAGES;
                if (n > 0 && !tc_wait(&empty[st], (uint32_t)((n - 1) & 1), abort)) break;
                unsigned char *sb = sm + (size_t)st * TC_STAGE_BYTES;
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                                 saddr(&full[st])),
                             "r"(bytes)
                             : "memory");
                const int x = kb * ELEMS;
                tma_load_2d(sb, &mah, x, ya, &full[st]);
                tma_load_2d(sb + TC_A_BYTES, &mal, x, ya, &full[st]);
                if (!inner) {
                    tma_load_2d(sb + 2 * TC_A_BYTES, &mbh, x, yb, &full[st]);
                    tma_load_2d(sb + 2 * TC_A_BYTES + TC_B_BYTES, &mbl, x, yb, &full[st]);
                }
            }
            if (*abort) {
                // the last copies issued may still be landing
                for (int q = max(0, kb - TC_STAGES); q < kb; ++q)
                    tc_wait(&full[q % TC_STAGES], (uint32_t)((q / TC_STAGES) & 1), nullptr);
            }
        }
    } else if (wid == 1) {
        if (lane == 0) {
            // ---- MMA issuer: chunk q goes to buffer q % TC_BUFS once the
            // epilogue has drained that buffer's previous chunk
            constexpr uint32_t idesc = tc_idesc<PREC>();
            int q = 0;
            bool ok = true;
            for (int kb = 0; kb < nblk && ok; ++kb) {
                const int st = kb % TC_STAGES, n = kb / TC_STAGES;
                if (!tc_wait(&full[st], (uint32_t)(n & 1), abort)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t sa = saddr(sm + (size_t)st * TC_STAGE_BYTES);
                const uint32_t ah = sa, al = sa + TC_A_BYTES;
                const uint32_t bh = inner ? ah + bin : sa + 2 * TC_A_BYTES;
                const uint32_t bl = inner ? al + bin : sa + 2 * TC_A_BYTES + TC_B_BYTES;
                const int qend = min(nchunks, (kb + 1) * CPB);
                for (; q < qend; ++q) {
                    const int buf = q % TC_BUFS, nb = q / TC_BUFS;
                    if (nb > 0 && !tc_wait(&tempty[buf], (uint32_t)((nb - 1) & 1), abort)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t d = tmem + (uint32_t)(buf * TC_N);
                    const int k0 = (q % CPB) * SPC;
#pragma unroll
                    for (int ks = 0; ks < SPC; ++ks) {
                        const uint32_t off = (uint32_t)((k0 + ks) * 32);
                        // per K step lo hi^T, hi lo^T, hi hi^T (the warp-level
                        // kernel's order); the chunk's first MMA overwrites
                        tc_mma<PREC>(d, sw128_desc(al + off), sw128_desc(bh + off), idesc, ks > 0);
                        tc_mma<PREC>(d, sw128_desc(ah + off), sw128_desc(bl + off), idesc, 1);
                        tc_mma<PREC>(d, sw128_desc(ah + off), sw128_desc(bh + off), idesc, 1);
                    }
                    tc_commit(&tfull[buf]);
                }
                if (ok) tc_commit(&empty[st]);
            }
            // every MMA issued has completed before tensor memory is freed
            tc_commit(&drain);
            tc_wait(&drain, 0u, nullptr);
        }
    } else {
        // ---- epilogue: compensated sums of the chunk sums of one row
        // (tensor-memory lane) and 32 columns per thread
        constexpr int CW = TC_N / 2;   // columns per thread
        const int quarter = wid & 3;
        const int col0 = ((wid - 2) >> 2) * CW;
        const int r = quarter * 32 + lane;   // tile row
        uint64_t shi[CW / 2], slo[CW / 2];   // columns (2i, 2i + 1) per pair
#pragma unroll
        for (int i = 0; i < CW / 2; ++i) {
            shi[i] = 0ull;
            slo[i] = 0ull;
        }
        const uint32_t tl = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)col0;
        // chunk q: wait for its buffer, issue its load (no wait)
        auto fetch = [&](int q, uint32_t (&v)[32]) -> bool {
            const int buf = q % TC_BUFS, nb = q / TC_BUFS;
            if (!__all_sync(0xffffffffu, tc_wait(&tfull[buf], (uint32_t)(nb & 1), abort))) return false;
            tc_fence_after();
            tmem_ld32(tl + (uint32_t)(buf * TC_N), v);
            return true;
        };
        // chunk q's load has landed: hand its buffer back to the MMA issuer
        auto release = [&](int q, uint32_t (&v)[32]) {
            tmem_wait32(v);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[q % TC_BUFS]);
        };
        auto accumulate = [&](const uint32_t (&v)[32]) {
#pragma unroll
            for (int i = 0; i < CW / 2; ++i) two_sum_acc2(shi[i], slo[i], f2_pack(v[2 * i], v[2 * i + 1]));
        };
        // two register sets: the next chunk's load is in flight while the
        // current one is summed
        uint32_t va[32], vb[32];
        bool ok = true;
        if (nchunks > 0) {
            ok = fetch(0, va);
            if (ok) release(0, va);
        }
        for (int q = 0; ok && q < nchunks; q += 2) {
            const bool h1 = q + 1 < nchunks, h2 = q + 2 < nchunks;
            if (h1) ok = fetch(q + 1, vb);
            accumulate(va);
            if (!ok || !h1) break;
            release(q + 1, vb);
            if (h2) ok = fetch(q + 2, va);
            accumulate(vb);
            if (ok && h2) release(q + 2, va);
        }
        // the tile through shared memory (the stages are free: every load
        // was consumed by an MMA that has completed), then coalesced stores
        // of the entries a <= b and of their mirrors
        float *T = (float *)sm;   // [TC_M][TC_N + 1]
        if (ok) {
#pragma unroll
            for (int i = 0; i < CW; ++i) {
                const int h = (i & 1) * 32;
                const float fh = __uint_as_float((uint32_t)(shi[i / 2] >> h));
                const float fl = __uint_as_float((uint32_t)(slo[i / 2] >> h));
                T[r * (TC_N + 1) + col0 + i] = __double2float_rn(__dadd_rn((double)fh, (double)fl));
            }
        }
        asm volatile("bar.sync 1, %0;" ::"n"(32 * TC_EPI_WARPS) : "memory");
        if (!*abort) {
            float *Gu = G + goff[u];
            const int e = wid - 2;
            for (int rr = e; rr < TC_M; rr += TC_EPI_WARPS) {
                const int a = a0 + rr;
                if (a >= c) continue;
                for (int cc = lane; cc < TC_N; cc += 32) {
                    const int b = b0 + cc;
                    if (b < c && a <= b) Gu[(int64_t)a * c + b] = T[rr * (TC_N + 1) + cc];
                }
            }
            for (int cc = e; cc < TC_N; cc += TC_EPI_WARPS) {
                const int b = b0 + cc;
                if (b >= c) continue;
                for (int rr = lane; rr < TC_M; rr += 32) {
                    const int a = a0 + rr;
                    if (a < c && a <= b) Gu[(int64_t)b * c + a] = T[rr * (TC_N + 1) + cc];
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (wid == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(TC_TMEM_COLS)
                     : "memory");
    }
    if (tid == 0 && *abort) atomicOr(status, ST_TIMEOUT);
}

// rows x sp row-major elements as a tensor map with boxes of 128 bytes x
// box_rows rows in the 128-byte swizzle layout (rows past the end read as
// zeros).
pmmf_status gram_map(CUtensorMap *m, const void *base, int64_t rows, int64_t sp, int prec, int box_rows) {
    auto fn = encode_fn();
    if (!fn) {
        set_error("cuTensorMapEncodeTiled is not available");
        return PMMF_ERR_CUDA;
    }
    const int eb = prec == PMMF_PREC_BF16 ? 2 : 4;
    cuuint64_t dims[2] = {(cuuint64_t)sp, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)sp * (cuuint64_t)eb};
    cuuint32_t box[2] = {(cuuint32_t)(TC_ROWB / eb), (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    CUresult r = fn(m, prec == PMMF_PREC_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                    2, const_cast<void *>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed for the Gram operands");
        return PMMF_ERR_CUDA;
    }
    return PMMF_OK;
}

}  // namespace

pmmf_status tc_gram_tcgen05(int precision, const void *XH, const void *XL, int64_t rows, int64_t sp,
                            const int64_t *coff, const std::vector<int64_t> &hcoff,
                            const int64_t *goff, float *G, unsigned *status, cudaStream_t st) {
    if (sp % 8 != 0 || rows >= ((int64_t)1 << 31) || sp >= ((int64_t)1 << 31)) {
        set_error("tensor-core Gram: row length must be a multiple of 8 and sizes below 2^31");
        return PMMF_ERR_INVALID_ARG;
    }
    const int64_t m = (int64_t)hcoff.size() - 1;
    std::vector<int32_t> tl;   // (u, A, B) per tile: rows 128 A.., columns 64 B.., B >= 2 A
    for (int64_t u = 0; u < m; ++u) {
        const int64_t c = hcoff[u + 1] - hcoff[u];
        const int TA = (int)((c + TC_M - 1) / TC_M), TB = (int)((c + TC_N - 1) / TC_N);
        for (int a = 0; a < TA; ++a)
            for (int b = a * (TC_M / TC_N); b < TB; ++b) {
                tl.push_back((int32_t)u);
                tl.push_back(a);
                tl.push_back(b);
            }
    }
    const int64_t nt = (int64_t)tl.size() / 3;
    if (nt == 0) return PMMF_OK;
    std::vector<int32_t> soa(3 * (size_t)nt);
    for (int64_t t = 0; t < nt; ++t) {
        soa[t] = tl[3 * t];
        soa[nt + t] = tl[3 * t + 1];
        soa[2 * nt + t] = tl[3 * t + 2];
    }
    DBuf<int32_t> dt;
    PMMF_TRY(dt.alloc(3 * nt, st));
    PMMF_CUDA_TRY(cudaMemcpyAsync(dt.p, soa.data(), sizeof(int32_t) * soa.size(), cudaMemcpyHostToDevice, st));
    CUtensorMap mah, mal, mbh, mbl;
    PMMF_TRY(gram_map(&mah, XH, rows, sp, precision, TC_M));
    PMMF_TRY(gram_map(&mal, XL, rows, sp, precision, TC_M));
    PMMF_TRY(gram_map(&mbh, XH, rows, sp, precision, TC_N));
    PMMF_TRY(gram_map(&mbl, XL, rows, sp, precision, TC_N));
    if (precision == PMMF_PREC_BF16) {
        PMMF_CUDA_TRY(allow_smem(k_tc_gram5<PMMF_PREC_BF16>, TC_SMEM));
        k_tc_gram5<PMMF_PREC_BF16><<<(unsigned)nt, TC_THREADS, TC_SMEM, st>>>(
            mah, mal, mbh, mbl, sp, coff, goff, dt.p, dt.p + nt, dt.p + 2 * nt, G, status);
    } else {
        PMMF_CUDA_TRY(allow_smem(k_tc_gram5<PMMF_PREC_TF32>, TC_SMEM));
        k_tc_gram5<PMMF_PREC_TF32><<<(unsigned)nt, TC_THREADS, TC_SMEM, st>>>(
            mah, mal, mbh, mbl, sp, coff, goff, dt.p, dt.p + nt, dt.p + 2 * nt, G, status);
    }
    return launched("tc_gram5");
}

}  // namespace pmmf
