// api.cu -- the C-ABI of include/pmmf.h: input staging and validation, the
// stage loop of Algorithm 1, the factorization handle, matrix-free apply and
// preconditioned CG.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <new>
#include <vector>

#include "apply.cuh"
#include "backward.cuh"
#include "batch.cuh"
#include "dense.cuh"
#include "mixed.cuh"
#include "common.cuh"
#include "stage.cuh"

namespace pmmf {
const char *last_error_cstr();

struct StageData {
    int64_t s = 0, m = 0, nrot = 0, nnz_after = 0, cmax = 0;
    int32_t max_levels = 0;
    double contrib = 0.0;
    StageClusters cls;
    StageRotations rot;
    Csr recorded;               // A_p[S_p, S_p] if params.record_stages
    DBuf<int32_t> recorded_act; // its row -> global id map
    bool has_record = false;
    DBuf<int64_t> nnz_d;        // A_p's exact entry count, read after the loop
};

}  // namespace pmmf

struct pmmf_handle {
    int64_t n = 0, nnz_in = 0;
    int k = 2;
    double norm_a = 0.0, err = 0.0;
    std::vector<pmmf::StageData> st;
    pmmf::DBuf<double> hdiag;
    int64_t ncore = 0;
    pmmf::DBuf<int32_t> core_idx, core_pos;
    pmmf::DBuf<double> core, core_inv;
    int inv_state = 0;  // 0 not formed, 1 formed, 2 not SPD
    pmmf::DBuf<double> core_isqrt;       // core^{-1/2} per block (xi = 1/2)
    int isqrt_state = 0;                 // as inv_state
    pmmf::DBuf<double> hrcp, hisr;       // 1 / h_i, 1 / sqrt(h_i): formed with core_inv, core_isqrt
    int isqrt_iters = 0;                 // Newton-Schulz steps it took
    pmmf::ApplyStages views;
    // core blocks (one for a single factorization, one per matrix of a batch)
    int64_t nblk = 1, bs = 0;
    pmmf::DBuf<int32_t> bdim;            // batch: per-block core size
    // batch: matrix b owns coordinates moff[b] .. moff[b+1]-1
    int64_t nmat = 1;
    std::vector<int64_t> moff;
    std::vector<double> mat_err;
    // reduced-precision shortlist counters: re-scored, fallbacks, steps, max
    unsigned long long prec_stats[4] = {0, 0, 0, 0};
};

namespace pmmf {
namespace {

constexpr int64_t DENSE_MAX_N = 24576;   // rows of 8 * n bytes in shared memory

pmmf_status fail(pmmf_status s, const char *msg) {
    set_error(msg);
    return s;
}

// The loop's results gathered for one readback: out[0] = status bits,
// out[1 + q] = stage q's dependency levels (max over its clusters),
// out[1 + P + q] = its matrix's entry count, out[1 + 2P + q] = the bits of its
// residual contribution, out[1 + 3P] = the bits of ||A||_F^2.  One block per
// stage of a chunk of up to 32.
constexpr int SUMMARY_CHUNK = 32;
struct SummaryChunk {
    const int32_t *nlev[SUMMARY_CHUNK];
    const int64_t *nnz[SUMMARY_CHUNK];
    int64_t m[SUMMARY_CHUNK];
};

__global__ void __launch_bounds__(256) k_stage_summary(SummaryChunk c, int64_t q0, int64_t P,
                                                       const unsigned *status,
                                                       const double *contrib,
                                                       const double *sumsq, int64_t *out) {
    __shared__ int32_t red[8];
    const int b = blockIdx.x;
    const int64_t q = q0 + b;
    if (q0 == 0 && b == 0) {
        if (threadIdx.x == 0) {
            out[0] = (int64_t)*status;
            out[1 + 3 * P] = (int64_t)__double_as_longlong(*sumsq);
        }
        for (int64_t i = threadIdx.x; i < P; i += blockDim.x) {
            out[1 + 2 * P + i] = (int64_t)__double_as_longlong(contrib[i]);
        }
    }
    if (q >= P) return;
    int32_t mx = 0;
    for (int64_t u = threadIdx.x; u < c.m[b]; u += blockDim.x) mx = max(mx, c.nlev[b][u]);
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) mx = max(mx, red[w]);
        out[1 + q] = mx;
        out[1 + P + q] = *c.nnz[b];
    }
}

// Reads the exact entry count of a matrix whose nnz is only a capacity.
pmmf_status exact_nnz(Csr &A, cudaStream_t st) {
    if (A.nnz_exact) return PMMF_OK;
    int64_t v = 0;
    PMMF_CUDA_TRY(cudaMemcpyAsync(&v, A.rowptr.p + A.rows, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    PMMF_CUDA_TRY(cudaStreamSynchronize(st));
    A.nnz = v;
    A.nnz_exact = true;
    return PMMF_OK;
}

// A second stream on which the next stage's clustering and schedule run while
// the current stage's update runs on the caller's stream.  Declare a SideDrain
// after every buffer the stream touches: the drain waits for the stream before
// those are freed.
struct SideDrain {
    cudaStream_t s = nullptr;
    ~SideDrain() {
        if (s) cudaStreamSynchronize(s);
    }
};

struct SideStream {
    cudaStream_t s = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
};

// One side stream (and its two events) per host thread, created on first use
// and kept: creating a stream costs more host time than a small stage.
pmmf_status side_stream(SideStream *&out) {
    thread_local SideStream ss;
    if (!ss.s) {
        SideStream t;
        PMMF_CUDA_TRY(cudaStreamCreateWithFlags(&t.s, cudaStreamNonBlocking));
        PMMF_CUDA_TRY(cudaEventCreateWithFlags(&t.fork, cudaEventDisableTiming));
        PMMF_CUDA_TRY(cudaEventCreateWithFlags(&t.join, cudaEventDisableTiming));
        ss = t;
    }
    out = &ss;
    return PMMF_OK;
}

void set_pool_threshold() {
    static bool done = false;
    if (done) return;
    done = true;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) != cudaSuccess) return;
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
}

template <class T>
pmmf_status to_device(const T *src, int64_t count, int location, DBuf<T> &dst, const T *&out,
                      cudaStream_t st) {
    if (location == PMMF_DEVICE) {
        out = src;
        return PMMF_OK;
    }
    PMMF_TRY(dst.alloc(count, st));
    if (count > 0)
        PMMF_CUDA_TRY(cudaMemcpyAsync(dst.p, src, sizeof(T) * (size_t)count, cudaMemcpyHostToDevice, st));
    out = dst.p;
    return PMMF_OK;
}

// Given stage-1 clusters on the device, checked (one synchronization).
pmmf_status stage1_labels(const pmmf_params *prm, int64_t n, DBuf<int32_t> &tmp,
                          const int32_t *&dl, unsigned *status, cudaStream_t st) {
    dl = nullptr;
    if (!prm->labels) return PMMF_OK;
    PMMF_TRY(to_device(prm->labels, n, prm->labels_location, tmp, dl, st));
    PMMF_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(unsigned), st));
    PMMF_TRY(check_labels(dl, n, prm->num_labels, status, st));
    unsigned hs = 0;
    PMMF_CUDA_TRY(cudaMemcpyAsync(&hs, status, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    PMMF_CUDA_TRY(cudaStreamSynchronize(st));
    if (hs & ST_BAD_LABEL) return fail(PMMF_ERR_INVALID_ARG, "a stage-1 label is outside [0, num_labels)");
    return PMMF_OK;
}

// Device CSR of A with exact zeros dropped, validated (structure, finite,
// exactly symmetric).
pmmf_status stage_input(const pmmf_matrix *A, Csr &out, unsigned *status_d, cudaStream_t st) {
    const int64_t n = A->n;
    if (A->format == PMMF_DENSE) {
        if (!A->val || A->ld < n) return fail(PMMF_ERR_INVALID_ARG, "dense A: val is NULL or ld < n");
        DBuf<double> tmp;
        const double *dv = nullptr;
        int64_t cnt = (n - 1) * A->ld + n;
        PMMF_TRY(to_device(A->val, cnt, A->location, tmp, dv, st));
        PMMF_TRY(dense_to_csr(dv, n, A->ld, out.rowptr, out.col, out.val, st));
    } else if (A->format == PMMF_CSR) {
        if (!A->rowptr || !A->colidx || !A->val) return fail(PMMF_ERR_INVALID_ARG, "CSR A: NULL array");
        int64_t nnz = 0;
        if (A->location == PMMF_HOST) {
            nnz = A->rowptr[n];
            if (A->rowptr[0] != 0 || nnz < 0) return fail(PMMF_ERR_INVALID_ARG, "CSR A: bad rowptr");
            for (int64_t i = 0; i < n; ++i)
                if (A->rowptr[i + 1] < A->rowptr[i]) return fail(PMMF_ERR_INVALID_ARG, "CSR A: rowptr decreases");
        } else {
            int64_t ends[2];
            PMMF_CUDA_TRY(cudaMemcpyAsync(&ends[0], A->rowptr, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
            PMMF_CUDA_TRY(cudaMemcpyAsync(&ends[1], A->rowptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
            PMMF_CUDA_TRY(cudaStreamSynchronize(st));
            if (ends[0] != 0 || ends[1] < 0) return fail(PMMF_ERR_INVALID_ARG, "CSR A: bad rowptr");
            nnz = ends[1];
        }
        DBuf<int64_t> trp;
        DBuf<int32_t> tci;
        DBuf<double> tv;
        const int64_t *rp = nullptr;
        const int32_t *ci = nullptr;
        const double *v = nullptr;
        PMMF_TRY(to_device(A->rowptr, n + 1, A->location, trp, rp, st));
        PMMF_TRY(to_device(A->colidx, nnz, A->location, tci, ci, st));
        PMMF_TRY(to_device(A->val, nnz, A->location, tv, v, st));
        // structure first (monotone rows, columns in range and ascending), on
        // the stored entries; then drop exact zeros and check symmetry
        PMMF_CUDA_TRY(cudaMemsetAsync(status_d, 0, sizeof(unsigned), st));
        PMMF_TRY(validate_csr(n, rp, ci, v, status_d, st, false));
        unsigned hs = 0;
        PMMF_CUDA_TRY(cudaMemcpyAsync(&hs, status_d, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
        PMMF_CUDA_TRY(cudaStreamSynchronize(st));
        if (hs & ST_BAD_CSR) return fail(PMMF_ERR_INVALID_ARG, "CSR A: columns out of range or not ascending");
        PMMF_TRY(csr_drop_zeros(n, rp, ci, v, out.rowptr, out.col, out.val, st));
    } else {
        return fail(PMMF_ERR_INVALID_ARG, "unknown matrix format");
    }
    out.rows = n;
    PMMF_CUDA_TRY(cudaMemcpyAsync(&out.nnz, out.rowptr.p + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    PMMF_CUDA_TRY(cudaMemsetAsync(status_d, 0, sizeof(unsigned), st));
    PMMF_TRY(validate_csr(n, out.rowptr.p, out.col.p, out.val.p, status_d, st));
    unsigned hs = 0;
    PMMF_CUDA_TRY(cudaMemcpyAsync(&hs, status_d, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    PMMF_CUDA_TRY(cudaStreamSynchronize(st));
    if (hs & ST_BAD_CSR) return fail(PMMF_ERR_INVALID_ARG, "CSR A: columns out of range or not ascending");
    if (hs & ST_NONFINITE) return fail(PMMF_ERR_NONFINITE, "A holds NaN or Inf");
    if (hs & ST_NOT_SYMMETRIC) return fail(PMMF_ERR_NOT_SYMMETRIC, "A is not exactly symmetric");
    return PMMF_OK;
}

pmmf_status check_params(const pmmf_matrix *A, const pmmf_params *p) {
    if (!A || !p) return fail(PMMF_ERR_INVALID_ARG, "NULL matrix or params");
    if (A->n < 1) return fail(PMMF_ERR_INVALID_ARG, "n must be >= 1");
    if (A->n >= INT32_MAX) return fail(PMMF_ERR_UNSUPPORTED, "n must be < 2^31");
    if (A->location != PMMF_HOST && A->location != PMMF_DEVICE)
        return fail(PMMF_ERR_INVALID_ARG, "bad matrix location");
    if (p->k < 2 || p->k > 8) return fail(PMMF_ERR_INVALID_ARG, "k must be in [2, 8]");
    if (!(p->eta > 0.0 && p->eta < 1.0)) return fail(PMMF_ERR_INVALID_ARG, "eta must be in (0, 1)");
    if (p->cluster_size < p->k) return fail(PMMF_ERR_INVALID_ARG, "cluster_size must be >= k");
    if (p->core_size < 1 || p->core_size > A->n)
        return fail(PMMF_ERR_INVALID_ARG, "core_size must be in [1, n]");
    if (p->lloyd_iters < 0) return fail(PMMF_ERR_INVALID_ARG, "lloyd_iters must be >= 0");
    if (p->precision < PMMF_PREC_FP64 || p->precision > PMMF_PREC_BF16)
        return fail(PMMF_ERR_INVALID_ARG, "unknown precision mode");
    if (p->coords && (p->coord_dim < 1 || p->coord_dim > 3))
        return fail(PMMF_ERR_INVALID_ARG, "coord_dim must be 1, 2 or 3");
    if (p->coords && p->coords_location != PMMF_HOST && p->coords_location != PMMF_DEVICE)
        return fail(PMMF_ERR_INVALID_ARG, "bad coords location");
    if (p->labels && (p->num_labels < 1 || p->num_labels > INT32_MAX))
        return fail(PMMF_ERR_INVALID_ARG, "num_labels must be in [1, 2^31)");
    if (p->labels && p->labels_location != PMMF_HOST && p->labels_location != PMMF_DEVICE)
        return fail(PMMF_ERR_INVALID_ARG, "bad labels location");
    return PMMF_OK;
}

void build_views(pmmf_handle *h) {
    h->views.clear();
    for (auto &S : h->st) {
        ApplyStage v;
        v.m = S.m;
        v.nrot = S.nrot;
        v.cmax = S.cmax;
        v.s = S.s;
        v.coff = S.cls.coff.p;
        v.members = S.cls.members.p;
        v.roff = S.rot.roff.p;
        v.lvl_off = S.rot.lvl_off.p;
        v.nlev = S.rot.nlev.p;
        v.lvlrot = S.rot.lvl.p;
        v.K = S.rot.K;
        v.kidx = S.rot.kidx.p;
        v.kkv = S.rot.kk.p;
        v.lvlidx = S.rot.lvlidx.p;
        v.kO = S.rot.kO.p;
        h->views.push_back(v);
    }
}

pmmf_status factor_impl(const pmmf_matrix *A, const pmmf_params *prm, pmmf_handle *h,
                        cudaStream_t st) {
    const int64_t n = A->n;
    h->n = n;
    h->k = prm->k;
    DBuf<unsigned> status;
    PMMF_TRY(status.zeros(1, st));

    Csr cur;
    PMMF_TRY(stage_input(A, cur, status.p, st));
    h->nnz_in = cur.nnz;
    // ||A||_F^2, read with the loop's results at the end
    DBuf<double> sumsq;
    PMMF_TRY(sumsq.alloc(1, st));
    PMMF_TRY(sum_squares(cur.val.p, cur.nnz, sumsq.p, st));

    // clustering geometry
    const bool geo = prm->coords != nullptr;
    const int dim = geo ? prm->coord_dim : 0;
    DBuf<int32_t> q, morder;
    if (geo) {
        DBuf<double> tc;
        const double *dc = nullptr;
        PMMF_TRY(to_device(prm->coords, n * dim, prm->coords_location, tc, dc, st));
        DBuf<uint64_t> code;
        PMMF_TRY(q.alloc(n * dim, st));
        PMMF_TRY(code.alloc(n, st));
        PMMF_CUDA_TRY(cudaMemsetAsync(status.p, 0, sizeof(unsigned), st));
        PMMF_TRY(quantize_points(dc, n, dim, q.p, code.p, status.p, st));
        PMMF_TRY(morder.alloc(n, st));
        PMMF_TRY(radix_sort_u64(code.p, n, 15 * dim, morder.p, st));
        unsigned hs = 0;
        PMMF_CUDA_TRY(cudaMemcpyAsync(&hs, status.p, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
        PMMF_CUDA_TRY(cudaStreamSynchronize(st));
        if (hs & ST_NONFINITE) return fail(PMMF_ERR_INVALID_ARG, "coords hold NaN or Inf");
    }
    DBuf<int32_t> tlab;
    const int32_t *dlab = nullptr;
    PMMF_TRY(stage1_labels(prm, n, tlab, dlab, status.p, st));

    DBuf<int32_t> act, pos, cl, loc, elimflag;
    DBuf<double> contribs;
    PMMF_TRY(act.alloc(n, st));
    PMMF_TRY(iota_i32(act.p, n, st));
    PMMF_TRY(pos.alloc(n, st));
    PMMF_TRY(iota_i32(pos.p, n, st));
    PMMF_TRY(cl.alloc(n, st));
    PMMF_TRY(loc.alloc(n, st));
    PMMF_TRY(elimflag.zeros(n, st));
    PMMF_TRY(h->hdiag.zeros(n, st));
    PMMF_TRY(contribs.zeros(n + 1, st));

    const int iters = prm->lloyd_iters > 0 ? prm->lloyd_iters : 10;
    int64_t s = n;
    int64_t p = 0;
    // device status bits of every stage, read once after the loop
    PMMF_CUDA_TRY(cudaMemsetAsync(status.p, 0, sizeof(unsigned), st));
    // clusters of stage pp (active set actp, positions posp) into cls; cl/loc
    // receive each active coordinate's cluster and local index
    auto cluster_stage = [&](int64_t pp, int64_t ss, const int32_t *actp, const int32_t *posp,
                             int32_t *clp, int32_t *locp, StageClusters &cls,
                             cudaStream_t sx) -> pmmf_status {
        int64_t m = (ss + prm->cluster_size / 2) / prm->cluster_size;
        if (m < 1 || !geo) m = 1;
        if (m > 1 || (pp == 1 && dlab)) {
            PartitionIn in;
            in.n = n;
            in.s = ss;
            in.dim = dim;
            in.q = q.p;
            in.morder = morder.p;
            in.pos = posp;
            in.act = actp;
            in.cl = clp;
            in.loc = locp;
            if (pp == 1 && dlab) return partition_from_labels(in, dlab, prm->num_labels, cls, sx);
            return partition_stage(in, m, iters, cls, sx);
        }
        return one_cluster(actp, ss, cls, clp, locp, sx);
    };
    auto more_stages = [&](int64_t ss, int64_t pp) {
        return ss > prm->core_size && (prm->max_stages <= 0 || pp < prm->max_stages);
    };
    SideStream *sidep = nullptr;
    PMMF_TRY(side_stream(sidep));
    const SideStream &side = *sidep;
    // the next stage's positions and cluster maps (swapped in after each stage)
    DBuf<int32_t> posN, clN, locN;
    PMMF_TRY(posN.alloc(n, st));
    PMMF_TRY(clN.alloc(n, st));
    PMMF_TRY(locN.alloc(n, st));
    StageClusters next_cls;
    DBuf<int64_t> next_e, next_roff;
    SideDrain drain{side.s};
    int64_t w_hint = 0;
    if (more_stages(s, p)) {
        PMMF_TRY(cluster_stage(1, s, act.p, pos.p, cl.p, loc.p, next_cls, st));
        PMMF_TRY(schedule_launch(next_cls.coff.p, next_cls.m, next_cls.count_d.p, s, prm->core_size,
                                 prm->eta, next_e, next_roff, st));
    }
    while (more_stages(s, p)) {
        ++p;
        h->st.emplace_back();
        StageData &S = h->st.back();
        S.s = s;
        S.cls = std::move(next_cls);
        // one readback per stage for the schedule (rotations, the one-cluster
        // fallback, the largest cluster and the Gram blocks' total size); from
        // stage 2 on it was computed on the side stream during the previous
        // stage's update, so the wait normally finds it done
        int64_t sched[5] = {0, 0, 0, 0, 0};
        if (p == 1) PMMF_CUDA_TRY(cudaStreamSynchronize(st));
        else PMMF_CUDA_TRY(cudaEventSynchronize(side.join));
        schedule_read(sched);
        DBuf<int64_t> e = std::move(next_e);
        S.rot.roff = std::move(next_roff);
        if (sched[1]) {
            // every cluster too small to rotate: one cluster for this stage
            PMMF_TRY(one_cluster(act.p, s, S.cls, cl.p, loc.p, st));
        } else {
            S.cls.m = sched[4];
        }
        S.m = S.cls.m;
        S.nrot = sched[0];
        S.rot.nrot = sched[0];
        S.cmax = sched[2];
        S.rot.K = prm->k;
        PMMF_TRY(gram_and_select(cur, act.p, pos.p, cl.p, loc.p, S.cls, S.cmax, prm->seed, p, S.rot,
                                 elimflag.p, st, nullptr, nullptr, status.p, sched[3]));
        Survivors sv;
        PMMF_TRY(survivors_stage(act.p, s, S.nrot, elimflag.p, p, sv, st));
        const int64_t s2 = sv.count;
        // the next stage's positions and clusters depend only on the
        // survivors: they run on the side stream while the update runs here
        const bool next = more_stages(s2, p);
        cudaStream_t ns = st;
        if (next) {
            ns = side.s;
            PMMF_CUDA_TRY(cudaEventRecord(side.fork, st));
            PMMF_CUDA_TRY(cudaStreamWaitEvent(ns, side.fork, 0));
        }
        {
            // (on failure, wait for the side stream: it may still read sv)
            pmmf_status ps = cudaMemsetAsync(posN.p, 0xFF, sizeof(int32_t) * (size_t)n, ns) == cudaSuccess
                                 ? PMMF_OK
                                 : fail(PMMF_ERR_CUDA, "position reset failed");
            if (ps == PMMF_OK) ps = set_positions(sv.act.p, s2, posN.p, ns);
            if (ps == PMMF_OK && next)
                ps = cluster_stage(p + 1, s2, sv.act.p, posN.p, clN.p, locN.p, next_cls, ns);
            if (ps == PMMF_OK && next)
                ps = schedule_launch(next_cls.coff.p, next_cls.m, next_cls.count_d.p, s2,
                                     prm->core_size, prm->eta, next_e, next_roff, ns);
            if (ps == PMMF_OK && next && cudaEventRecord(side.join, ns) != cudaSuccess)
                ps = fail(PMMF_ERR_CUDA, "event record failed");
            if (ps != PMMF_OK) {
                cudaStreamSynchronize(side.s);
                return ps;
            }
        }
        UpdateOut up;
        up.w_hint = w_hint;
        pmmf_status us = update_stage(cur, act.p, n, pos.p, cl.p, loc.p, S.cls, S.cmax, S.rot,
                                      elimflag.p, p, sv, h->hdiag.p, contribs.p + (p - 1), up,
                                      status.p, st);
        if (us == PMMF_OK) us = S.nnz_d.alloc(1, st);
        if (us == PMMF_OK &&
            cudaMemcpyAsync(S.nnz_d.p, up.next.rowptr.p + up.next.rows, sizeof(int64_t),
                            cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            us = fail(PMMF_ERR_CUDA, "stage nnz copy failed");
        if (us != PMMF_OK) {
            // the side stream still reads this stage's survivors
            cudaStreamSynchronize(side.s);
            return us;
        }
        if (next) {
            if (cudaStreamWaitEvent(st, side.join, 0) != cudaSuccess) {
                cudaStreamSynchronize(side.s);
                return fail(PMMF_ERR_CUDA, "stream wait failed");
            }
            // made on the side stream, used and freed on this one from here
            next_cls.coff.st = st;
            next_cls.members.st = st;
            next_cls.count_d.st = st;
            next_e.st = st;
            next_roff.st = st;
        }
        // pass 1's output for the next stage, scaled from this one with a 2x margin
        w_hint = (int64_t)(2.0 * (double)up.w_nnz * (double)up.next.nnz /
                           (double)std::max<int64_t>(cur.nnz, 1)) + 1024;
        std::swap(pos, posN);
        std::swap(cl, clN);
        std::swap(loc, locN);
        s = s2;
        cur = std::move(up.next);
        act = std::move(sv.act);
        if (prm->record_stages) {
            PMMF_TRY(exact_nnz(cur, st));
            S.recorded.rows = cur.rows;
            S.recorded.nnz = cur.nnz;
            PMMF_TRY(S.recorded.rowptr.alloc(cur.rows + 1, st));
            PMMF_TRY(S.recorded.col.alloc(cur.nnz, st));
            PMMF_TRY(S.recorded.val.alloc(cur.nnz, st));
            PMMF_TRY(S.recorded_act.alloc(cur.rows, st));
            PMMF_CUDA_TRY(cudaMemcpyAsync(S.recorded.rowptr.p, cur.rowptr.p, sizeof(int64_t) * (size_t)(cur.rows + 1), cudaMemcpyDeviceToDevice, st));
            if (cur.nnz > 0) {
                PMMF_CUDA_TRY(cudaMemcpyAsync(S.recorded.col.p, cur.col.p, sizeof(int32_t) * (size_t)cur.nnz, cudaMemcpyDeviceToDevice, st));
                PMMF_CUDA_TRY(cudaMemcpyAsync(S.recorded.val.p, cur.val.p, sizeof(double) * (size_t)cur.nnz, cudaMemcpyDeviceToDevice, st));
            }
            if (cur.rows > 0)
                PMMF_CUDA_TRY(cudaMemcpyAsync(S.recorded_act.p, act.p, sizeof(int32_t) * (size_t)cur.rows, cudaMemcpyDeviceToDevice, st));
            S.has_record = true;
        }
    }

    // status bits, each stage's dependency levels, entry count and residual
    // contribution: gathered on the device, read with one copy
    const int64_t P = (int64_t)h->st.size();
    std::vector<int64_t> summ((size_t)(2 + 3 * P));
    {
        DBuf<int64_t> summ_d;
        PMMF_TRY(summ_d.alloc(2 + 3 * P, st));
        for (int64_t q0 = 0; q0 == 0 || q0 < P; q0 += SUMMARY_CHUNK) {
            SummaryChunk c{};
            const int64_t nb = std::max<int64_t>(1, std::min<int64_t>(SUMMARY_CHUNK, P - q0));
            for (int64_t b = 0; b < nb && q0 + b < P; ++b) {
                const StageData &S = h->st[(size_t)(q0 + b)];
                c.nlev[b] = S.rot.nlev.p;
                c.nnz[b] = S.nnz_d.p;
                c.m[b] = S.rot.nlev.p ? S.m : 0;
            }
            k_stage_summary<<<(unsigned)nb, 256, 0, st>>>(c, q0, P, status.p, contribs.p, sumsq.p,
                                                          summ_d.p);
            PMMF_TRY(launched("stage_summary"));
        }
        PMMF_CUDA_TRY(cudaMemcpyAsync(summ.data(), summ_d.p, sizeof(int64_t) * summ.size(),
                                      cudaMemcpyDeviceToHost, st));
    }
    // H: core A_L[S_L, S_L] plus the diagonal
    h->ncore = s;
    PMMF_TRY(h->core_idx.alloc(s, st));
    PMMF_CUDA_TRY(cudaMemcpyAsync(h->core_idx.p, act.p, sizeof(int32_t) * (size_t)s, cudaMemcpyDeviceToDevice, st));
    PMMF_TRY(h->core.alloc(s * s, st));
    PMMF_TRY(extract_core(cur, pos.p, s, h->core.p, h->hdiag.p, act.p, st));
    PMMF_TRY(h->core_pos.alloc(n, st));
    PMMF_CUDA_TRY(cudaMemsetAsync(h->core_pos.p, 0xFF, sizeof(int32_t) * (size_t)n, st));
    PMMF_TRY(set_positions(act.p, s, h->core_pos.p, st));
    PMMF_CUDA_TRY(cudaStreamSynchronize(st));
    const unsigned hs = (unsigned)summ[0];
    {
        double a2;
        std::memcpy(&a2, &summ[(size_t)(1 + 3 * P)], sizeof(a2));
        h->norm_a = std::sqrt(a2);
    }
    if (hs & ST_ROW_TOO_LONG) return fail(PMMF_ERR_UNSUPPORTED, "update: output row too long");
    if (hs & ST_NOT_CONVERGED)
        return fail(PMMF_ERR_NOT_CONVERGED, "k x k Jacobi did not converge in 32 sweeps");
    double tot = 0.0;
    for (int64_t i = 0; i < P; ++i) {
        StageData &S = h->st[(size_t)i];
        S.max_levels = (int32_t)summ[(size_t)(1 + i)];
        S.nnz_after = summ[(size_t)(1 + P + i)];
        double c;
        std::memcpy(&c, &summ[(size_t)(1 + 2 * P + i)], sizeof(c));
        S.contrib = c;
        tot += c;
    }
    h->err = h->norm_a > 0.0 ? std::sqrt(tot) / h->norm_a : 0.0;
    h->nblk = 1;
    h->bs = h->ncore;
    h->nmat = 1;
    h->moff = {0, n};
    h->mat_err = {h->err};
    build_views(h);
    return PMMF_OK;
}

// Algorithm 1 on a dense input kept dense (n x n in HBM): the same stage as
// the sparse path (partition, schedule, rotation search) with the dense Gram
// and dense blocked update; the same readings, so the same bits.
pmmf_status factor_dense_impl(const pmmf_matrix *A, const pmmf_params *prm, pmmf_handle *h,
                              cudaStream_t st) {
    const int64_t n = A->n;
    h->n = n;
    h->k = prm->k;
    DBuf<unsigned> status;
    PMMF_TRY(status.zeros(1, st));
    DBuf<double> D;
    {
        DBuf<double> tmp;
        const double *dv = nullptr;
        if (!A->val || A->ld < n) return fail(PMMF_ERR_INVALID_ARG, "dense A: val is NULL or ld < n");
        PMMF_TRY(to_device(A->val, (n - 1) * A->ld + n, A->location, tmp, dv, st));
        PMMF_TRY(dense_load(dv, n, A->ld, D, status.p, st));
        unsigned hs = 0;
        PMMF_CUDA_TRY(cudaMemcpyAsync(&hs, status.p, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
        PMMF_CUDA_TRY(cudaStreamSynchronize(st));
        if (hs & ST_NONFINITE) return fail(PMMF_ERR_NONFINITE, "A holds NaN or Inf");
        if (hs & ST_NOT_SYMMETRIC) return fail(PMMF_ERR_NOT_SYMMETRIC, "A is not exactly symmetric");
    }
    {
        DBuf<double> ss;
        PMMF_TRY(ss.alloc(1, st));
        PMMF_TRY(sum_squares(D.p, n * n, ss.p, st));
        double hs = 0.0;
        PMMF_CUDA_TRY(cudaMemcpyAsync(&hs, ss.p, sizeof(double), cudaMemcpyDeviceToHost, st));
        PMMF_CUDA_TRY(cudaStreamSynchronize(st));
        h->norm_a = std::sqrt(hs);
        // stored entries of the input, as the sparse path counts them
        PMMF_TRY(dense_nonzeros(D.p, n * n, &h->nnz_in, st));
    }
    const bool geo = prm->coords != nullptr;
    const int dim = geo ? prm->coord_dim : 0;
    DBuf<int32_t> q, morder;
    if (geo) {
        DBuf<double> tc;
        const double *dc = nullptr;
        PMMF_TRY(to_device(prm->coords, n * dim, prm->coords_location, tc, dc, st));
        DBuf<uint64_t> code;
        PMMF_TRY(q.alloc(n * dim, st));
        PMMF_TRY(code.alloc(n, st));
        PMMF_CUDA_TRY(cudaMemsetAsync(status.p, 0, sizeof(unsigned), st));
        PMMF_TRY(quantize_points(dc, n, dim, q.p, code.p, status.p, st));
        PMMF_TRY(morder.alloc(n, st));
        PMMF_TRY(radix_sort_u64(code.p, n, 15 * dim, morder.p, st));
        unsigned hs = 0;
        PMMF_CUDA_TRY(cudaMemcpyAsync(&hs, status.p, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
        PMMF_CUDA_TRY(cudaStreamSynchronize(st));
        if (hs & ST_NONFINITE) return fail(PMMF_ERR_INVALID_ARG, "coords hold NaN or Inf");
    }
    DBuf<int32_t> tlab;
    const int32_t *dlab = nullptr;
    PMMF_TRY(stage1_labels(prm, n, tlab, dlab, status.p, st));
    DBuf<int32_t> act, pos, cl, loc, elimflag;
    DBuf<double> contribs;
    PMMF_TRY(act.alloc(n, st));
    PMMF_TRY(iota_i32(act.p, n, st));
    PMMF_TRY(pos.alloc(n, st));
    PMMF_TRY(iota_i32(pos.p, n, st));
    PMMF_TRY(cl.alloc(n, st));
    PMMF_TRY(loc.alloc(n, st));
    PMMF_TRY(elimflag.zeros(n, st));
    PMMF_TRY(h->hdiag.zeros(n, st));
    PMMF_TRY(contribs.zeros(n + 1, st));
    const int iters = prm->lloyd_iters > 0 ? prm->lloyd_iters : 10;
    DBuf<unsigned long long> pstats;
    PMMF_TRY(pstats.zeros(4, st));
    int64_t s = n, p = 0;
    while (s > prm->core_size && (prm->max_stages <= 0 || p < prm->max_stages)) {
        ++p;
        h->st.emplace_back();
        StageData &S = h->st.back();
        S.s = s;
        int64_t m = (s + prm->cluster_size / 2) / prm->cluster_size;
        if (m < 1 || !geo) m = 1;
        if (m > 1 || (p == 1 && dlab)) {
            PartitionIn in;
            in.n = n;
            in.s = s;
            in.dim = dim;
            in.q = q.p;
            in.morder = morder.p;
            in.pos = pos.p;
            in.act = act.p;
            in.cl = cl.p;
            in.loc = loc.p;
            if (p == 1 && dlab) PMMF_TRY(partition_from_labels(in, dlab, prm->num_labels, S.cls, st));
            else PMMF_TRY(partition_stage(in, m, iters, S.cls, st));
        } else {
            PMMF_TRY(one_cluster(act.p, s, S.cls, cl.p, loc.p, st));
        }
        int64_t sched[5] = {0, 0, 0, 0, 0};
        DBuf<int64_t> e;
        PMMF_TRY(schedule_stage(S.cls.coff.p, S.cls.m, S.cls.count_d.p, s, prm->core_size, prm->eta,
                                e, S.rot.roff, sched, st));
        if (sched[1]) PMMF_TRY(one_cluster(act.p, s, S.cls, cl.p, loc.p, st));
        else S.cls.m = sched[4];
        S.m = S.cls.m;
        S.nrot = sched[0];
        S.rot.nrot = sched[0];
        S.rot.K = prm->k;
        std::vector<int64_t> hc((size_t)S.m + 1);
        PMMF_CUDA_TRY(cudaMemcpyAsync(hc.data(), S.cls.coff.p, sizeof(int64_t) * hc.size(), cudaMemcpyDeviceToHost, st));
        PMMF_CUDA_TRY(cudaStreamSynchronize(st));
        for (int64_t u = 0; u < S.m; ++u) S.cmax = std::max(S.cmax, hc[u + 1] - hc[u]);
        PMMF_CUDA_TRY(cudaMemsetAsync(status.p, 0, sizeof(unsigned), st));
        // the reduced-precision Gram and shortlist only while the stage has
        // many clusters (at least PMMF_TUNE_MIXED_ACTIVE, default 12): the FP64
        // Gram costs ~c s^2 = s^2 (s / m), the shortlist search's FP64 rows ~s
        // per step, and with fewer clusters the FP64 Gram and search are the
        // faster pair (dense RBF n = 16,384, clusters of 512, per stage FP64
        // vs TF32: 32 clusters 171 vs 99 ms, 16: 71 vs 58, 8: 39 vs 41, 4: 34
        // vs 44); both choose the same rotations
        const int64_t mixed_min = tuned(TUNE_MIXED_ACTIVE, S.cmax, 12);
        if (prm->precision != PMMF_PREC_FP64 && S.m >= mixed_min) {
            PMMF_TRY(mixed_stage_select(D, s, pos.p, S.cls, hc, S.cmax, prm->precision, prm->seed,
                                        p, S.rot, elimflag.p, pstats.p, status.p, st));
        } else {
            GramBlocks gb;
            PMMF_TRY(gram_blocks(S.cls, gb, st));
            PMMF_TRY(dense_gram(D, s, pos.p, S.cls, hc, gb, st));
            PMMF_TRY(select_stage(S.cls, S.cmax, gb, prm->seed, p, S.rot, elimflag.p, st, nullptr,
                                  nullptr, status.p));
        }
        int32_t nlv = 0;
        {
            unsigned hs = 0;
            std::vector<int32_t> nl((size_t)S.m);
            PMMF_CUDA_TRY(cudaMemcpyAsync(&hs, status.p, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
            PMMF_CUDA_TRY(cudaMemcpyAsync(nl.data(), S.rot.nlev.p, sizeof(int32_t) * nl.size(), cudaMemcpyDeviceToHost, st));
            PMMF_CUDA_TRY(cudaStreamSynchronize(st));
            if (hs & ST_NOT_CONVERGED)
                return fail(PMMF_ERR_NOT_CONVERGED, "k x k Jacobi did not converge in 32 sweeps");
            if (hs & ST_TIMEOUT)
                return fail(PMMF_ERR_TIMEOUT, "a bounded wait of the tensor-core Gram ran out");
            for (int32_t v : nl) nlv = std::max(nlv, v);
            S.max_levels = nlv;
        }
        DenseLevels lv;
        PMMF_TRY(dense_levels(S.cls, S.rot, pos.p, nlv, lv, st));
        DBuf<double> Dn;
        DBuf<int32_t> nact;
        int64_t s2 = 0;
        bool tiled = false;
        // the per-row kernel is the default: measured faster on GB300 (the
        // dense RBF workload n = 16,384: 28.5 against 34.0 ms per factorization)
        if (tuned(TUNE_DENSE_TILES, S.cmax, 2) == 1)
            PMMF_TRY(dense_update_tiles(D, s, S.cls, hc, S.rot, pos.p, act.p, elimflag.p, p,
                                        h->hdiag.p, contribs.p + (p - 1), Dn, nact, s2, status.p, st,
                                        &tiled));
        if (!tiled)
            PMMF_TRY(dense_update(D, s, lv, act.p, elimflag.p, p, h->hdiag.p, contribs.p + (p - 1), Dn,
                                  nact, s2, st));
        PMMF_CUDA_TRY(cudaMemsetAsync(pos.p, 0xFF, sizeof(int32_t) * (size_t)n, st));
        PMMF_TRY(set_positions(nact.p, s2, pos.p, st));
        s = s2;
        D = std::move(Dn);
        act = std::move(nact);
        if (prm->record_stages) {
            PMMF_TRY(dense_record(D.p, s, act.p, S.recorded, st));
            PMMF_TRY(S.recorded_act.alloc(s, st));
            if (s > 0)
                PMMF_CUDA_TRY(cudaMemcpyAsync(S.recorded_act.p, act.p, sizeof(int32_t) * (size_t)s, cudaMemcpyDeviceToDevice, st));
            S.has_record = true;
            S.nnz_after = S.recorded.nnz;
        } else {
            S.nnz_after = s * s;
        }
    }
    h->ncore = s;
    PMMF_TRY(h->core_idx.alloc(s, st));
    if (s > 0)
        PMMF_CUDA_TRY(cudaMemcpyAsync(h->core_idx.p, act.p, sizeof(int32_t) * (size_t)s, cudaMemcpyDeviceToDevice, st));
    PMMF_TRY(h->core.alloc(s * s, st));
    PMMF_TRY(dense_core(D.p, s, act.p, h->core.p, h->hdiag.p, st));
    PMMF_TRY(h->core_pos.alloc(n, st));
    PMMF_CUDA_TRY(cudaMemsetAsync(h->core_pos.p, 0xFF, sizeof(int32_t) * (size_t)n, st));
    PMMF_TRY(set_positions(act.p, s, h->core_pos.p, st));
    std::vector<double> hcb((size_t)p + 1, 0.0);
    if (p > 0)
        PMMF_CUDA_TRY(cudaMemcpyAsync(hcb.data(), contribs.p, sizeof(double) * (size_t)p, cudaMemcpyDeviceToHost, st));
    unsigned hst = 0;
    PMMF_CUDA_TRY(cudaMemcpyAsync(&hst, status.p, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    PMMF_CUDA_TRY(cudaStreamSynchronize(st));
    if (hst & ST_TIMEOUT) return fail(PMMF_ERR_TIMEOUT, "dense update: a tile copy did not complete");
    double tot = 0.0;
    for (int64_t i = 0; i < p; ++i) {
        h->st[i].contrib = hcb[i];
        tot += hcb[i];
    }
    h->err = h->norm_a > 0.0 ? std::sqrt(tot) / h->norm_a : 0.0;
    h->nblk = 1;
    h->bs = h->ncore;
    h->nmat = 1;
    h->moff = {0, n};
    h->mat_err = {h->err};
    PMMF_CUDA_TRY(cudaMemcpy(h->prec_stats, pstats.p, sizeof(h->prec_stats), cudaMemcpyDeviceToHost));
    build_views(h);
    return PMMF_OK;
}

template <class T>
pmmf_status upload(const std::vector<T> &v, DBuf<T> &d, cudaStream_t st) {
    PMMF_TRY(d.alloc((int64_t)std::max<size_t>(v.size(), 1), st));
    if (!v.empty())
        PMMF_CUDA_TRY(cudaMemcpyAsync(d.p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, st));
    return PMMF_OK;
}

// Batched factorization of a block-diagonal matrix: block b (coordinates
// moff[b] .. moff[b+1]-1) is factored exactly as pmmf_factor would factor it
// alone with one cluster per stage and seed + b, i.e. Algorithm 1 per matrix;
// all blocks advance through the stages together.  Per cluster (= matrix),
// e = max(1, min(floor(eta c), c - core_size)) (the single-cluster case of the
// stage schedule); a matrix retires, its active rows becoming its core block,
// once at most core_size coordinates are active.
pmmf_status factor_batch_impl(const pmmf_matrix *A, const std::vector<int64_t> &moff,
                              const pmmf_params *prm, pmmf_handle *h, cudaStream_t st) {
    const int64_t n = A->n, nmat = (int64_t)moff.size() - 1;
    const int64_t delta = prm->core_size;
    h->n = n;
    h->k = prm->k;
    h->nmat = nmat;
    h->moff = moff;
    DBuf<unsigned> status;
    PMMF_TRY(status.zeros(1, st));
    Csr cur;
    PMMF_TRY(stage_input(A, cur, status.p, st));
    h->nnz_in = cur.nnz;
    DBuf<int64_t> moff_d;
    PMMF_TRY(upload(moff, moff_d, st));
    PMMF_CUDA_TRY(cudaMemsetAsync(status.p, 0, sizeof(unsigned), st));
    PMMF_TRY(check_blocks(n, cur.rowptr.p, cur.col.p, moff_d.p, nmat, status.p, st));
    std::vector<double> norm2((size_t)nmat);
    {
        DBuf<double> nd;
        PMMF_TRY(nd.alloc(nmat, st));
        PMMF_TRY(block_sumsq(cur.rowptr.p, cur.val.p, moff_d.p, nmat, nd.p, st));
        unsigned hs = 0;
        PMMF_CUDA_TRY(cudaMemcpyAsync(norm2.data(), nd.p, sizeof(double) * (size_t)nmat, cudaMemcpyDeviceToHost, st));
        PMMF_CUDA_TRY(cudaMemcpyAsync(&hs, status.p, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
        PMMF_CUDA_TRY(cudaStreamSynchronize(st));
        if (hs & ST_BAD_CSR) return fail(PMMF_ERR_INVALID_ARG, "batch: an entry lies outside its diagonal block");
    }
    double tot2 = 0.0;
    for (double v : norm2) tot2 += v;
    h->norm_a = std::sqrt(tot2);

    int64_t nmax = 0;
    for (int64_t b = 0; b < nmat; ++b) nmax = std::max(nmax, moff[b + 1] - moff[b]);
    const int64_t bs = std::max<int64_t>(1, std::min(delta, nmax));
    h->nblk = nmat;
    h->bs = bs;
    PMMF_TRY(h->core.zeros(nmat * bs * bs, st));
    PMMF_TRY(h->core_idx.alloc(nmat * bs, st));
    PMMF_CUDA_TRY(cudaMemsetAsync(h->core_idx.p, 0xFF, sizeof(int32_t) * (size_t)(nmat * bs), st));
    PMMF_TRY(h->core_pos.alloc(n, st));
    PMMF_CUDA_TRY(cudaMemsetAsync(h->core_pos.p, 0xFF, sizeof(int32_t) * (size_t)n, st));
    PMMF_TRY(h->bdim.zeros(nmat, st));

    DBuf<int32_t> act, pos, cl, loc, elimflag, retired_d;
    DBuf<double> contrib1;
    DBuf<int64_t> lo_d, cnt_d;
    PMMF_TRY(act.alloc(n, st));
    PMMF_TRY(iota_i32(act.p, n, st));
    PMMF_TRY(pos.alloc(n, st));
    PMMF_TRY(iota_i32(pos.p, n, st));
    PMMF_TRY(cl.alloc(n, st));
    PMMF_TRY(loc.alloc(n, st));
    PMMF_TRY(elimflag.zeros(n, st));
    PMMF_TRY(h->hdiag.zeros(n, st));
    PMMF_TRY(contrib1.zeros(1, st));
    PMMF_TRY(retired_d.zeros(nmat, st));
    PMMF_TRY(lo_d.alloc(nmat, st));
    PMMF_TRY(cnt_d.alloc(nmat, st));
    std::vector<int32_t> retired((size_t)nmat, 0);
    std::vector<int64_t> lo((size_t)nmat), cnt((size_t)nmat);
    std::vector<double> mat_contrib((size_t)nmat, 0.0);
    int64_t s = n, p = 0, ncore = 0;
    for (;;) {
        PMMF_TRY(batch_ranges(act.p, s, moff_d.p, nmat, lo_d.p, cnt_d.p, st));
        PMMF_CUDA_TRY(cudaMemcpyAsync(lo.data(), lo_d.p, sizeof(int64_t) * (size_t)nmat, cudaMemcpyDeviceToHost, st));
        PMMF_CUDA_TRY(cudaMemcpyAsync(cnt.data(), cnt_d.p, sizeof(int64_t) * (size_t)nmat, cudaMemcpyDeviceToHost, st));
        PMMF_CUDA_TRY(cudaStreamSynchronize(st));
        std::vector<int64_t> rmat, rlo, rcnt, amat;
        for (int64_t b = 0; b < nmat; ++b) {
            if (retired[b]) continue;
            if (cnt[b] <= delta) {
                rmat.push_back(b);
                rlo.push_back(lo[b]);
                rcnt.push_back(cnt[b]);
                retired[b] = 1;
                ncore += cnt[b];
            } else {
                amat.push_back(b);
            }
        }
        if (!rmat.empty()) {
            DBuf<int64_t> rm, rl, rc;
            PMMF_TRY(upload(rmat, rm, st));
            PMMF_TRY(upload(rlo, rl, st));
            PMMF_TRY(upload(rcnt, rc, st));
            PMMF_TRY(batch_core(cur, act.p, pos.p, (int64_t)rmat.size(), rm.p, rl.p, rc.p, bs,
                                h->core.p, h->core_idx.p, h->core_pos.p, h->bdim.p, h->hdiag.p, st));
            PMMF_TRY(upload(retired, retired_d, st));
            PMMF_TRY(batch_drop_rows(cur, act, retired_d.p, moff_d.p, nmat, st));
            s = cur.rows;
            PMMF_CUDA_TRY(cudaMemsetAsync(pos.p, 0xFF, sizeof(int32_t) * (size_t)n, st));
            PMMF_TRY(set_positions(act.p, s, pos.p, st));
        }
        if (amat.empty()) break;
        ++p;
        h->st.emplace_back();
        StageData &S = h->st.back();
        S.s = s;
        const int64_t m = (int64_t)amat.size();
        std::vector<int64_t> coff((size_t)m + 1, 0), roff((size_t)m + 1, 0);
        std::vector<uint64_t> useed((size_t)m);
        std::vector<int32_t> order((size_t)m);
        for (int64_t u = 0; u < m; ++u) {
            const int64_t c = cnt[amat[u]];
            coff[u + 1] = coff[u] + c;
            int64_t e = (int64_t)std::floor(prm->eta * (double)c);
            e = std::max<int64_t>(1, std::min(e, c - delta));
            roff[u + 1] = roff[u] + e;
            S.cmax = std::max(S.cmax, c);
            useed[u] = prm->seed + (uint64_t)amat[u];
            order[u] = (int32_t)u;
        }
        // longest clusters first, so the longest searches start in the first wave
        std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) {
            return roff[x + 1] - roff[x] > roff[y + 1] - roff[y];
        });
        PMMF_TRY(upload(coff, S.cls.coff, st));
        PMMF_TRY(batch_clusters(act.p, s, S.cls.coff.p, m, S.cls, cl.p, loc.p, st));
        PMMF_TRY(upload(roff, S.rot.roff, st));
        DBuf<uint64_t> useed_d;
        DBuf<int32_t> order_d;
        PMMF_TRY(upload(useed, useed_d, st));
        PMMF_TRY(upload(order, order_d, st));
        S.m = m;
        S.nrot = roff[m];
        S.rot.nrot = roff[m];
        S.rot.K = prm->k;
        PMMF_CUDA_TRY(cudaMemsetAsync(status.p, 0, sizeof(unsigned), st));
        PMMF_TRY(gram_and_select(cur, act.p, pos.p, cl.p, loc.p, S.cls, S.cmax, prm->seed, p, S.rot,
                                 elimflag.p, st, order_d.p, useed_d.p, status.p));
        DBuf<double> ccl;
        PMMF_TRY(ccl.zeros(m, st));
        Survivors sv;
        PMMF_TRY(survivors_stage(act.p, s, S.nrot, elimflag.p, p, sv, st));
        UpdateOut up;
        PMMF_TRY(update_stage(cur, act.p, n, pos.p, cl.p, loc.p, S.cls, S.cmax, S.rot, elimflag.p,
                              p, sv, h->hdiag.p, contrib1.p, up, status.p, st, ccl.p));
        {
            unsigned hs = 0;
            std::vector<int32_t> nl((size_t)m);
            std::vector<double> cc((size_t)m);
            PMMF_CUDA_TRY(cudaMemcpyAsync(&hs, status.p, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
            PMMF_CUDA_TRY(cudaMemcpyAsync(nl.data(), S.rot.nlev.p, sizeof(int32_t) * nl.size(), cudaMemcpyDeviceToHost, st));
            PMMF_CUDA_TRY(cudaMemcpyAsync(cc.data(), ccl.p, sizeof(double) * cc.size(), cudaMemcpyDeviceToHost, st));
            PMMF_CUDA_TRY(cudaMemcpyAsync(&up.next.nnz, up.next.rowptr.p + up.next.rows, sizeof(int64_t),
                                          cudaMemcpyDeviceToHost, st));
            PMMF_CUDA_TRY(cudaStreamSynchronize(st));
            up.next.nnz_exact = true;
            if (hs & ST_ROW_TOO_LONG) return fail(PMMF_ERR_UNSUPPORTED, "update: output row too long");
            if (hs & ST_NOT_CONVERGED)
                return fail(PMMF_ERR_NOT_CONVERGED, "k x k Jacobi did not converge in 32 sweeps");
            int32_t ml = 0;
            for (int32_t v : nl) ml = std::max(ml, v);
            S.max_levels = ml;
            for (int64_t u = 0; u < m; ++u) {
                mat_contrib[amat[u]] += cc[u];
                S.contrib += cc[u];
            }
        }
        S.nnz_after = up.next.nnz;
        PMMF_CUDA_TRY(cudaMemsetAsync(pos.p, 0xFF, sizeof(int32_t) * (size_t)n, st));
        PMMF_TRY(set_positions(sv.act.p, up.next.rows, pos.p, st));
        s = up.next.rows;
        cur = std::move(up.next);
        act = std::move(sv.act);
    }
    h->ncore = ncore;
    double tot = 0.0;
    h->mat_err.assign((size_t)nmat, 0.0);
    for (int64_t b = 0; b < nmat; ++b) {
        tot += mat_contrib[b];
        h->mat_err[b] = norm2[b] > 0.0 ? std::sqrt(mat_contrib[b]) / std::sqrt(norm2[b]) : 0.0;
    }
    h->err = h->norm_a > 0.0 ? std::sqrt(tot) / h->norm_a : 0.0;
    build_views(h);
    return PMMF_OK;
}

}  // namespace
}  // namespace pmmf

using namespace pmmf;

extern "C" {

const char *pmmf_last_error(void) { return last_error_cstr(); }

uint64_t pmmf_launch_count(void) { return g_launches.load(); }
uint64_t pmmf_alloc_count(void) { return g_allocs.load(); }

pmmf_status pmmf_factor(const pmmf_matrix *A, const pmmf_params *p, pmmf_handle **out,
                        void *stream) {
    set_error("");
    if (!out) return fail(PMMF_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    PMMF_TRY(check_params(A, p));
    set_pool_threshold();
    cudaStream_t st = (cudaStream_t)stream;
    pmmf_handle *h = new (std::nothrow) pmmf_handle();
    if (!h) return fail(PMMF_ERR_OOM, "host allocation failed");
    pmmf_status s;
    try {
        // a dense input stays dense when its rows fit one CTA's shared memory
        const bool dense = A->format == PMMF_DENSE && A->n <= DENSE_MAX_N;
        if (p->precision != PMMF_PREC_FP64 && !dense)
            s = fail(PMMF_ERR_UNSUPPORTED, "reduced-precision Gram needs a dense input with n <= 24576");
        else if (dense)
            s = factor_dense_impl(A, p, h, st);
        else
            s = factor_impl(A, p, h, st);
    } catch (const std::bad_alloc &) {
        s = fail(PMMF_ERR_OOM, "host allocation failed");
    }
    if (s != PMMF_OK) {
        cudaStreamSynchronize(st);
        delete h;
        return s;
    }
    *out = h;
    return PMMF_OK;
}

pmmf_status pmmf_factor_blockdiag(const pmmf_matrix *A, int64_t nmat, const int64_t *block_off,
                                  const pmmf_params *p, pmmf_handle **out, void *stream) {
    set_error("");
    if (!out) return fail(PMMF_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    PMMF_TRY(check_params(A, p));
    if (nmat < 1 || !block_off) return fail(PMMF_ERR_INVALID_ARG, "need nmat >= 1 and block_off");
    if (p->coords) return fail(PMMF_ERR_INVALID_ARG, "batch: one cluster per matrix, coords must be NULL");
    if (p->max_stages > 0) return fail(PMMF_ERR_INVALID_ARG, "batch: max_stages must be 0");
    std::vector<int64_t> moff(block_off, block_off + nmat + 1);
    if (moff[0] != 0 || moff[nmat] != A->n) return fail(PMMF_ERR_INVALID_ARG, "block_off must run from 0 to n");
    for (int64_t b = 0; b < nmat; ++b)
        if (moff[b + 1] <= moff[b]) return fail(PMMF_ERR_INVALID_ARG, "block_off must increase strictly");
    set_pool_threshold();
    cudaStream_t st = (cudaStream_t)stream;
    pmmf_handle *h = new (std::nothrow) pmmf_handle();
    if (!h) return fail(PMMF_ERR_OOM, "host allocation failed");
    pmmf_status s;
    try {
        s = factor_batch_impl(A, moff, p, h, st);
    } catch (const std::bad_alloc &) {
        s = fail(PMMF_ERR_OOM, "host allocation failed");
    }
    if (s != PMMF_OK) {
        cudaStreamSynchronize(st);
        delete h;
        return s;
    }
    *out = h;
    return PMMF_OK;
}

pmmf_status pmmf_factor_batched(int64_t nmat, const pmmf_matrix *A, const pmmf_params *p,
                                pmmf_handle **out, void *stream) {
    set_error("");
    if (!out) return fail(PMMF_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (nmat < 1 || !A) return fail(PMMF_ERR_INVALID_ARG, "need nmat >= 1 matrices");
    std::vector<int64_t> moff((size_t)nmat + 1, 0);
    int64_t nnz = 0;
    for (int64_t b = 0; b < nmat; ++b) {
        if (A[b].format != PMMF_CSR || A[b].location != PMMF_HOST || !A[b].rowptr || A[b].n < 1)
            return fail(PMMF_ERR_INVALID_ARG, "batch: every matrix must be a HOST CSR matrix with n >= 1");
        moff[b + 1] = moff[b] + A[b].n;
        nnz += A[b].rowptr[A[b].n] - A[b].rowptr[0];
    }
    if (moff[nmat] >= INT32_MAX) return fail(PMMF_ERR_UNSUPPORTED, "batch: total size must be < 2^31");
    std::vector<int64_t> rp((size_t)moff[nmat] + 1, 0);
    std::vector<int32_t> ci((size_t)std::max<int64_t>(nnz, 1));
    std::vector<double> v((size_t)std::max<int64_t>(nnz, 1));
    int64_t q = 0;
    for (int64_t b = 0; b < nmat; ++b) {
        const pmmf_matrix &M = A[b];
        if (!M.colidx || !M.val) return fail(PMMF_ERR_INVALID_ARG, "batch: NULL CSR array");
        for (int64_t i = 0; i < M.n; ++i) {
            for (int64_t e = M.rowptr[i]; e < M.rowptr[i + 1]; ++e) {
                if (M.colidx[e] < 0 || M.colidx[e] >= M.n)
                    return fail(PMMF_ERR_INVALID_ARG, "batch: column index out of range");
                ci[(size_t)q] = (int32_t)(M.colidx[e] + moff[b]);
                v[(size_t)q] = M.val[e];
                ++q;
            }
            rp[(size_t)(moff[b] + i + 1)] = q;
        }
    }
    pmmf_matrix big{};
    big.n = moff[nmat];
    big.format = PMMF_CSR;
    big.location = PMMF_HOST;
    big.rowptr = rp.data();
    big.colidx = ci.data();
    big.val = v.data();
    return pmmf_factor_blockdiag(&big, nmat, moff.data(), p, out, stream);
}

pmmf_status pmmf_get_precision_stats(const pmmf_handle *f, int64_t *rescored, int64_t *fallbacks,
                                     int64_t *steps, int64_t *max_shortlist) {
    if (!f) return fail(PMMF_ERR_INVALID_ARG, "NULL handle");
    if (rescored) *rescored = (int64_t)f->prec_stats[0];
    if (fallbacks) *fallbacks = (int64_t)f->prec_stats[1];
    if (steps) *steps = (int64_t)f->prec_stats[2];
    if (max_shortlist) *max_shortlist = (int64_t)f->prec_stats[3];
    return PMMF_OK;
}

pmmf_status pmmf_get_batch(const pmmf_handle *f, int64_t *nmat, int64_t *core_stride,
                           int64_t *block_off, double *errors, int32_t *core_dim) {
    if (!f) return fail(PMMF_ERR_INVALID_ARG, "NULL handle");
    if (nmat) *nmat = f->nmat;
    if (core_stride) *core_stride = f->bs;
    if (block_off) std::copy(f->moff.begin(), f->moff.end(), block_off);
    if (errors) std::copy(f->mat_err.begin(), f->mat_err.end(), errors);
    if (core_dim) {
        if (f->nblk > 1)
            PMMF_CUDA_TRY(cudaMemcpy(core_dim, f->bdim.p, sizeof(int32_t) * (size_t)f->nmat, cudaMemcpyDeviceToHost));
        else
            core_dim[0] = (int32_t)f->ncore;
    }
    return PMMF_OK;
}

void pmmf_free(pmmf_handle *f) {
    if (!f) return;
    cudaDeviceSynchronize();
    set_free_sync(true);
    delete f;
    set_free_sync(false);
}

pmmf_status pmmf_get_info(const pmmf_handle *f, pmmf_info *info) {
    if (!f || !info) return fail(PMMF_ERR_INVALID_ARG, "NULL handle or info");
    info->n = f->n;
    info->stages = (int32_t)f->st.size();
    info->core_size = f->ncore;
    int64_t r = 0;
    for (auto &s : f->st) r += s.nrot;
    info->rotations = r;
    info->nnz_input = f->nnz_in;
    info->norm_a = f->norm_a;
    info->error = f->err;
    return PMMF_OK;
}

pmmf_status pmmf_get_stage_info(const pmmf_handle *f, int p, pmmf_stage_info *info) {
    if (!f || !info || p < 0 || p >= (int)f->st.size()) return fail(PMMF_ERR_INVALID_ARG, "bad stage");
    const StageData &s = f->st[p];
    info->active = s.s;
    info->clusters = s.m;
    info->rotations = s.nrot;
    info->nnz_after = s.nnz_after;
    info->max_levels = s.max_levels;
    info->contrib = s.contrib;
    return PMMF_OK;
}

pmmf_status pmmf_get_stage_clusters(const pmmf_handle *f, int p, int64_t *offsets, int32_t *members) {
    if (!f || p < 0 || p >= (int)f->st.size() || !offsets || !members)
        return fail(PMMF_ERR_INVALID_ARG, "bad stage or NULL buffer");
    const StageData &s = f->st[p];
    PMMF_CUDA_TRY(cudaMemcpy(offsets, s.cls.coff.p, sizeof(int64_t) * (size_t)(s.m + 1), cudaMemcpyDeviceToHost));
    PMMF_CUDA_TRY(cudaMemcpy(members, s.cls.members.p, sizeof(int32_t) * (size_t)s.s, cudaMemcpyDeviceToHost));
    return PMMF_OK;
}

pmmf_status pmmf_get_stage_rotations(const pmmf_handle *f, int p, int32_t *cluster, int32_t *kk,
                                     int32_t *idx, double *O, int32_t *elim) {
    if (!f || p < 0 || p >= (int)f->st.size()) return fail(PMMF_ERR_INVALID_ARG, "bad stage");
    const StageData &s = f->st[p];
    const int K = f->k;
    std::vector<int64_t> coff((size_t)s.m + 1), roff((size_t)s.m + 1);
    std::vector<int32_t> mem((size_t)s.s);
    PMMF_CUDA_TRY(cudaMemcpy(coff.data(), s.cls.coff.p, sizeof(int64_t) * coff.size(), cudaMemcpyDeviceToHost));
    PMMF_CUDA_TRY(cudaMemcpy(roff.data(), s.rot.roff.p, sizeof(int64_t) * roff.size(), cudaMemcpyDeviceToHost));
    PMMF_CUDA_TRY(cudaMemcpy(mem.data(), s.cls.members.p, sizeof(int32_t) * mem.size(), cudaMemcpyDeviceToHost));
    if (K > 2) {
        const size_t nr = (size_t)std::max<int64_t>(s.nrot, 1);
        std::vector<int32_t> ki(nr * K), kv(nr), ke(nr);
        std::vector<double> ko(nr * K * K);
        if (s.nrot > 0) {
            PMMF_CUDA_TRY(cudaMemcpy(ki.data(), s.rot.kidx.p, sizeof(int32_t) * (size_t)(s.nrot * K), cudaMemcpyDeviceToHost));
            PMMF_CUDA_TRY(cudaMemcpy(kv.data(), s.rot.kk.p, sizeof(int32_t) * (size_t)s.nrot, cudaMemcpyDeviceToHost));
            PMMF_CUDA_TRY(cudaMemcpy(ke.data(), s.rot.kel.p, sizeof(int32_t) * (size_t)s.nrot, cudaMemcpyDeviceToHost));
            PMMF_CUDA_TRY(cudaMemcpy(ko.data(), s.rot.kO.p, sizeof(double) * (size_t)(s.nrot * K * K), cudaMemcpyDeviceToHost));
        }
        for (int64_t u = 0; u < s.m; ++u)
            for (int64_t r = roff[u]; r < roff[u + 1]; ++r) {
                if (cluster) cluster[r] = (int32_t)u;
                if (kk) kk[r] = kv[r];
                if (idx)
                    for (int a = 0; a < K; ++a)
                        idx[r * K + a] = ki[r * K + a] >= 0 ? mem[coff[u] + ki[r * K + a]] : -1;
                if (O)
                    for (int a = 0; a < K * K; ++a) O[r * K * K + a] = ko[r * K * K + a];
                if (elim) elim[r] = mem[coff[u] + ke[r]];
            }
        return PMMF_OK;
    }
    std::vector<RotRec> rec((size_t)std::max<int64_t>(s.nrot, 1));
    if (s.nrot > 0)
        PMMF_CUDA_TRY(cudaMemcpy(rec.data(), s.rot.rec.p, sizeof(RotRec) * (size_t)s.nrot, cudaMemcpyDeviceToHost));
    for (int64_t u = 0; u < s.m; ++u) {
        for (int64_t r = roff[u]; r < roff[u + 1]; ++r) {
            const RotRec &q = rec[r];
            if (cluster) cluster[r] = (int32_t)u;
            if (kk) kk[r] = 2;
            if (idx) {
                for (int a = 0; a < K; ++a) idx[r * K + a] = -1;
                idx[r * K + 0] = mem[coff[u] + q.li];
                idx[r * K + 1] = mem[coff[u] + q.lj];
            }
            if (O) {
                for (int a = 0; a < K * K; ++a) O[r * K * K + a] = 0.0;
                O[r * K * K + 0] = q.c;
                O[r * K * K + 1] = -q.s;
                O[r * K * K + 2] = q.s;
                O[r * K * K + 3] = q.c;
            }
            if (elim) elim[r] = mem[coff[u] + q.le];
        }
    }
    return PMMF_OK;
}

pmmf_status pmmf_get_h(const pmmf_handle *f, double *hdiag, int32_t *core_idx, double *core) {
    if (!f) return fail(PMMF_ERR_INVALID_ARG, "NULL handle");
    if (hdiag) PMMF_CUDA_TRY(cudaMemcpy(hdiag, f->hdiag.p, sizeof(double) * (size_t)f->n, cudaMemcpyDeviceToHost));
    const int64_t slots = f->nblk * f->bs;
    if (core_idx && slots > 0)
        PMMF_CUDA_TRY(cudaMemcpy(core_idx, f->core_idx.p, sizeof(int32_t) * (size_t)slots, cudaMemcpyDeviceToHost));
    if (core && slots > 0)
        PMMF_CUDA_TRY(cudaMemcpy(core, f->core.p, sizeof(double) * (size_t)(slots * f->bs), cudaMemcpyDeviceToHost));
    return PMMF_OK;
}

}  // extern "C"

namespace pmmf {
namespace {

pmmf_status ensure_inverse(pmmf_handle *f, cudaStream_t st) {
    if (f->inv_state == 1) return PMMF_OK;
    if (f->inv_state == 2) return fail(PMMF_ERR_NOT_SPD, "H is not positive definite");
    DBuf<unsigned> status;
    PMMF_TRY(status.zeros(1, st));
    PMMF_TRY(f->core_inv.alloc(f->nblk * f->bs * f->bs, st));
    if (f->nblk > 1)
        PMMF_TRY(invert_core_blocks(f->core.p, f->nblk, f->bs, f->bdim.p, f->hdiag.p, f->core_pos.p,
                                    f->n, f->core_inv.p, status.p, st));
    else
        PMMF_TRY(invert_core(f->core.p, f->ncore, f->hdiag.p, f->core_pos.p, f->n, f->core_inv.p,
                             status.p, st));
    // The reciprocals are formed before the status readback, so the one
    // synchronization below also finishes them: once the state says "formed",
    // any stream or host thread may read them without further ordering.
    PMMF_TRY(f->hrcp.alloc(f->n, st));
    PMMF_TRY(h_reciprocals(f->hdiag.p, f->n, false, f->hrcp.p, st));
    unsigned hs = 0;
    PMMF_CUDA_TRY(cudaMemcpyAsync(&hs, status.p, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    PMMF_CUDA_TRY(cudaStreamSynchronize(st));
    if (hs & ST_NOT_SPD) {
        f->hrcp.reset();
        f->inv_state = 2;
        return fail(PMMF_ERR_NOT_SPD, "H is not positive definite");
    }
    f->inv_state = 1;
    return PMMF_OK;
}

pmmf_status ensure_isqrt(pmmf_handle *f, cudaStream_t st) {
    if (f->isqrt_state == 1) return PMMF_OK;
    if (f->isqrt_state == 2) return fail(PMMF_ERR_NOT_SPD, "H is not positive definite");
    DBuf<unsigned> status;
    PMMF_TRY(status.zeros(1, st));
    PMMF_TRY(f->core_isqrt.alloc(f->nblk * f->bs * f->bs, st));
    const pmmf_status cs = core_inverse_sqrt(f->core.p, f->nblk, f->bs, f->nblk > 1 ? f->bdim.p : nullptr,
                                             f->hdiag.p, f->core_pos.p, f->n, f->core_isqrt.p,
                                             status.p, &f->isqrt_iters, st);
    if (cs == PMMF_ERR_NOT_SPD) {
        f->isqrt_state = 2;
        return cs;
    }
    PMMF_TRY(cs);
    // Formed before the readback, as in ensure_inverse: the synchronization
    // below orders them before every later use on any stream.
    PMMF_TRY(f->hisr.alloc(f->n, st));
    PMMF_TRY(h_reciprocals(f->hdiag.p, f->n, true, f->hisr.p, st));
    unsigned hs = 0;
    PMMF_CUDA_TRY(cudaMemcpyAsync(&hs, status.p, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    PMMF_CUDA_TRY(cudaStreamSynchronize(st));
    if (hs & ST_NOT_SPD) {
        f->hisr.reset();
        f->isqrt_state = 2;
        return fail(PMMF_ERR_NOT_SPD, "H is not positive definite");
    }
    f->isqrt_state = 1;
    return PMMF_OK;
}

HData hdata(const pmmf_handle *f) {
    HData H;
    H.n = f->n;
    H.m = f->nblk * f->bs;
    H.nblk = f->nblk;
    H.bs = f->bs;
    H.bdim = f->nblk > 1 ? f->bdim.p : nullptr;
    H.hdiag = f->hdiag.p;
    H.core_pos = f->core_pos.p;
    H.core_idx = f->core_idx.p;
    H.core = f->core.p;
    H.core_inv = f->core_inv.p;
    H.core_isqrt = f->core_isqrt.p;
    H.hrcp = f->inv_state == 1 ? f->hrcp.p : nullptr;
    H.hisr = f->isqrt_state == 1 ? f->hisr.p : nullptr;
    return H;
}

// y <- op(x) with y already holding a copy of x.
pmmf_status apply_inplace(pmmf_handle *f, int op, double *y, int64_t nrhs, int64_t ld,
                          cudaStream_t st) {
    const int mode = op == PMMF_OP_A_INV || op == PMMF_OP_H_INV ? 1
                   : op == PMMF_OP_A_INV_SQRT || op == PMMF_OP_H_INV_SQRT ? 2 : 0;
    if (mode == 1) PMMF_TRY(ensure_inverse(f, st));
    if (mode == 2) PMMF_TRY(ensure_isqrt(f, st));
    switch (op) {
    case PMMF_OP_U: return apply_rotations(f->views, false, y, ld, nrhs, st);
    case PMMF_OP_UT: return apply_rotations(f->views, true, y, ld, nrhs, st);
    case PMMF_OP_H:
    case PMMF_OP_H_INV:
    case PMMF_OP_H_INV_SQRT: return apply_h(hdata(f), mode, y, ld, nrhs, st);
    case PMMF_OP_A:
    case PMMF_OP_A_INV:
    case PMMF_OP_A_INV_SQRT:
        PMMF_TRY(apply_rotations(f->views, false, y, ld, nrhs, st));
        PMMF_TRY(apply_h(hdata(f), mode, y, ld, nrhs, st));
        return apply_rotations(f->views, true, y, ld, nrhs, st);
    default: return fail(PMMF_ERR_INVALID_ARG, "unknown op");
    }
}

}  // namespace
}  // namespace pmmf

extern "C" {

pmmf_status pmmf_get_stage_matrix(const pmmf_handle *f, int p, int64_t *rowptr_n1, int32_t *col,
                                  double *val, int64_t *nnz) {
    if (!f || p < 0 || p >= (int)f->st.size()) return fail(PMMF_ERR_INVALID_ARG, "bad stage");
    const StageData &s = f->st[p];
    if (!s.has_record) return fail(PMMF_ERR_INVALID_ARG, "stage not recorded (set record_stages)");
    if (nnz) *nnz = s.recorded.nnz;
    if (!rowptr_n1 && !col && !val) return PMMF_OK;
    if (!rowptr_n1 || !col || !val) return fail(PMMF_ERR_INVALID_ARG, "NULL buffer");
    std::vector<int64_t> rp((size_t)s.recorded.rows + 1);
    std::vector<int32_t> act((size_t)s.recorded.rows);
    PMMF_CUDA_TRY(cudaMemcpy(rp.data(), s.recorded.rowptr.p, sizeof(int64_t) * rp.size(), cudaMemcpyDeviceToHost));
    if (!act.empty())
        PMMF_CUDA_TRY(cudaMemcpy(act.data(), s.recorded_act.p, sizeof(int32_t) * act.size(), cudaMemcpyDeviceToHost));
    if (s.recorded.nnz > 0) {
        PMMF_CUDA_TRY(cudaMemcpy(col, s.recorded.col.p, sizeof(int32_t) * (size_t)s.recorded.nnz, cudaMemcpyDeviceToHost));
        PMMF_CUDA_TRY(cudaMemcpy(val, s.recorded.val.p, sizeof(double) * (size_t)s.recorded.nnz, cudaMemcpyDeviceToHost));
    }
    // rows by global id: rows outside S_p are empty
    std::vector<int64_t> len((size_t)f->n, 0);
    for (size_t r = 0; r < act.size(); ++r) len[act[r]] = rp[r + 1] - rp[r];
    rowptr_n1[0] = 0;
    for (int64_t i = 0; i < f->n; ++i) rowptr_n1[i + 1] = rowptr_n1[i] + len[i];
    return PMMF_OK;
}

pmmf_status pmmf_apply(const pmmf_handle *fc, int op, const double *x, double *y, int64_t nrhs,
                       int64_t ld, void *stream) {
    set_error("");
    pmmf_handle *f = const_cast<pmmf_handle *>(fc);
    if (!f || !x || !y) return fail(PMMF_ERR_INVALID_ARG, "NULL handle or vector");
    if (nrhs < 1 || ld < nrhs) return fail(PMMF_ERR_INVALID_ARG, "need nrhs >= 1 and ld >= nrhs");
    if (op < PMMF_OP_A || op > PMMF_OP_H_INV_SQRT) return fail(PMMF_ERR_INVALID_ARG, "unknown op");
    cudaStream_t st = (cudaStream_t)stream;
    if (x != y) PMMF_TRY(copy_block(x, ld, y, ld, f->n, nrhs, st));
    return apply_inplace(f, op, y, nrhs, ld, st);
}

}  // extern "C"

namespace pmmf {
namespace {

// Conjugate gradients with the factorization as preconditioner (Sec. 4):
// sym = false: PCG with M^{-1} = A~^{-1} (xi = 1); sym = true: plain CG on the
// split system W A W y = W b, W = A~^{-1/2}, x = W y (xi = 1/2).
pmmf_status solve_impl(const pmmf_handle *fc, const pmmf_matrix *A, const double *b, double *x,
                       int64_t nrhs, double rtol, int maxit, int32_t *iters, double *relres,
                       void *stream, bool sym) {
    set_error("");
    pmmf_handle *f = const_cast<pmmf_handle *>(fc);
    if (!f || !A || !b || !x || !iters || !relres) return fail(PMMF_ERR_INVALID_ARG, "NULL argument");
    if (A->n != f->n) return fail(PMMF_ERR_INVALID_ARG, "A and the factorization differ in size");
    if (nrhs < 1 || nrhs > 8) return fail(PMMF_ERR_UNSUPPORTED, "nrhs must be in [1, 8]");
    if (!(rtol > 0.0) || maxit < 0) return fail(PMMF_ERR_INVALID_ARG, "need rtol > 0 and maxit >= 0");
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = f->n;
    const int nr = (int)nrhs;
    DBuf<unsigned> status;
    PMMF_TRY(status.zeros(1, st));
    Csr M;
    PMMF_TRY(stage_input(A, M, status.p, st));
    DevCsr dA;
    dA.n = n;
    dA.rp = M.rowptr.p;
    dA.ci = M.col.p;
    dA.v = M.val.p;
    PMMF_TRY(sym ? ensure_isqrt(f, st) : ensure_inverse(f, st));

    DBuf<double> r, z, pv, qv, sc, part, zc;
    DBuf<int32_t> done, itd;
    PMMF_TRY(r.alloc(n * nr, st));
    PMMF_TRY(z.alloc(n * nr, st));
    PMMF_TRY(pv.alloc(n * nr, st));
    PMMF_TRY(qv.alloc(n * nr, st));
    PMMF_TRY(sc.zeros(8 * 8, st));          // rz, pq, rr, rznew, bb, bnorm, alpha, beta
    PMMF_TRY(part.alloc(dot_partial_size(nr), st));
    PMMF_TRY(done.zeros(8, st));
    PMMF_TRY(itd.zeros(9, st));             // iterations per column, then the counter
    PMMF_TRY(zc.alloc(std::max<int64_t>(f->nblk * f->bs * nr, 1), st));
    double *rz = sc.p, *pq = sc.p + 8, *rr = sc.p + 16, *rzn = sc.p + 24, *bb = sc.p + 32;
    double *bnorm = sc.p + 40, *alpha = sc.p + 48, *beta = sc.p + 56;
    const HData H = hdata(f);
    // W v in place (W = U^T H^{-1/2} U)
    auto apply_w = [&](double *v, cudaStream_t s) -> pmmf_status {
        PMMF_TRY(apply_rotations(f->views, false, v, nr, nr, s));
        PMMF_TRY(apply_h_scratch(H, 2, v, nr, nr, zc.p, s));
        return apply_rotations(f->views, true, v, nr, nr, s);
    };
    // one CG iteration on the split system: q = W A W p, x holds y; the
    // residual is the split one, and p <- r + beta p
    auto body_sym = [&](cudaStream_t s) -> pmmf_status {
        PMMF_CUDA_TRY(cudaMemcpyAsync(z.p, pv.p, sizeof(double) * (size_t)(n * nr), cudaMemcpyDeviceToDevice, s));
        PMMF_TRY(apply_w(z.p, s));
        PMMF_TRY(spmv(dA, z.p, qv.p, nr, s));
        PMMF_TRY(apply_w(qv.p, s));
        PMMF_TRY(dots(pv.p, qv.p, n, nr, pq, part.p, s));
        PMMF_TRY(cg_update_xr(x, r.p, pv.p, qv.p, n, nr, rz, pq, done.p, alpha, s));
        PMMF_TRY(dots(r.p, r.p, n, nr, rr, part.p, s));
        PMMF_TRY(cg_check(rr, bnorm, rtol, nr, done.p, itd.p, itd.p + 8, s));
        return cg_update_p(pv.p, r.p, n, nr, rr, rz, done.p, beta, s);
    };
    // one PCG iteration (Sec. 4 with M^{-1} = U^T H^{-1} U applied matrix-free)
    auto body_pcg = [&](cudaStream_t s) -> pmmf_status {
        PMMF_TRY(spmv(dA, pv.p, qv.p, nr, s));
        PMMF_TRY(dots(pv.p, qv.p, n, nr, pq, part.p, s));
        PMMF_TRY(cg_update_xr(x, r.p, pv.p, qv.p, n, nr, rz, pq, done.p, alpha, s));
        PMMF_TRY(dots(r.p, r.p, n, nr, rr, part.p, s));
        PMMF_TRY(cg_check(rr, bnorm, rtol, nr, done.p, itd.p, itd.p + 8, s));
        PMMF_CUDA_TRY(cudaMemcpyAsync(z.p, r.p, sizeof(double) * (size_t)(n * nr), cudaMemcpyDeviceToDevice, s));
        PMMF_TRY(apply_rotations(f->views, false, z.p, nr, nr, s));
        PMMF_TRY(apply_h_scratch(H, true, z.p, nr, nr, zc.p, s));
        PMMF_TRY(apply_rotations(f->views, true, z.p, nr, nr, s));
        PMMF_TRY(dots(r.p, z.p, n, nr, rzn, part.p, s));
        return cg_update_p(pv.p, z.p, n, nr, rzn, rz, done.p, beta, s);
    };
    auto body = [&](cudaStream_t s) -> pmmf_status { return sym ? body_sym(s) : body_pcg(s); };
    PMMF_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(double) * (size_t)(n * nr), st));
    PMMF_CUDA_TRY(cudaMemcpyAsync(r.p, b, sizeof(double) * (size_t)(n * nr), cudaMemcpyDeviceToDevice, st));
    if (sym) {
        // r = W b, p = r, rz = r.r, and the split right-hand side's norm
        PMMF_TRY(apply_w(r.p, st));
        PMMF_CUDA_TRY(cudaMemcpyAsync(pv.p, r.p, sizeof(double) * (size_t)(n * nr), cudaMemcpyDeviceToDevice, st));
        PMMF_TRY(dots(r.p, r.p, n, nr, rz, part.p, st));
        PMMF_TRY(dots(r.p, r.p, n, nr, bb, part.p, st));
    } else {
        PMMF_CUDA_TRY(cudaMemcpyAsync(z.p, b, sizeof(double) * (size_t)(n * nr), cudaMemcpyDeviceToDevice, st));
        PMMF_TRY(apply_inplace(f, PMMF_OP_A_INV, z.p, nr, nr, st));
        PMMF_CUDA_TRY(cudaMemcpyAsync(pv.p, z.p, sizeof(double) * (size_t)(n * nr), cudaMemcpyDeviceToDevice, st));
        PMMF_TRY(dots(r.p, z.p, n, nr, rz, part.p, st));
        PMMF_TRY(dots(b, b, n, nr, bb, part.p, st));
    }
    double hb[8], hr[8];
    int32_t hdone[8];
    PMMF_CUDA_TRY(cudaMemcpyAsync(hb, bb, sizeof(double) * nr, cudaMemcpyDeviceToHost, st));
    PMMF_CUDA_TRY(cudaStreamSynchronize(st));
    for (int c = 0; c < nr; ++c) {
        hb[c] = std::sqrt(hb[c]);
        hdone[c] = hb[c] == 0.0;
        iters[c] = 0;
    }
    PMMF_CUDA_TRY(cudaMemcpyAsync(done.p, hdone, sizeof(int32_t) * nr, cudaMemcpyHostToDevice, st));
    PMMF_CUDA_TRY(cudaMemcpyAsync(bnorm, hb, sizeof(double) * nr, cudaMemcpyHostToDevice, st));
    // Iteration 1 runs directly (it also sets the kernels' shared-memory
    // attributes); the iteration is then captured once as a CUDA graph and
    // replayed in batches, the convergence flags read back after each batch.
    // Iterations after a column has converged leave that column unchanged.
    auto all_done = [&]() -> pmmf_status {
        PMMF_CUDA_TRY(cudaMemcpyAsync(hdone, done.p, sizeof(int32_t) * nr, cudaMemcpyDeviceToHost, st));
        PMMF_CUDA_TRY(cudaStreamSynchronize(st));
        return PMMF_OK;
    };
    auto finished = [&]() {
        for (int c = 0; c < nr; ++c)
            if (!hdone[c]) return false;
        return true;
    };
    int it = 0;
    if (maxit > 0 && !finished()) {
        PMMF_TRY(body(st));
        it = 1;
        PMMF_TRY(all_done());
    }
    if (it < maxit && !finished()) {
        cudaStream_t cs = nullptr;
        PMMF_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        pmmf_status bs = PMMF_OK;
        cudaError_t ce = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
        if (ce == cudaSuccess) {
            bs = body(cs);
            ce = cudaStreamEndCapture(cs, &graph);
        }
        if (ce == cudaSuccess && bs == PMMF_OK) ce = cudaGraphInstantiate(&exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        cudaStreamDestroy(cs);
        if (bs != PMMF_OK) return bs;
        if (ce != cudaSuccess) {
            if (exec) cudaGraphExecDestroy(exec);
            return fail(PMMF_ERR_CUDA, (std::string("PCG graph capture: ") + cudaGetErrorString(ce)).c_str());
        }
        pmmf_status ls = PMMF_OK;
        while (it < maxit && !finished()) {
            const int batch = std::min(8, maxit - it);
            for (int q = 0; q < batch && ls == PMMF_OK; ++q) {
                const cudaError_t le = cudaGraphLaunch(exec, st);
                if (le != cudaSuccess) ls = fail(PMMF_ERR_CUDA, (std::string("PCG graph launch: ") + cudaGetErrorString(le)).c_str());
                g_launches.fetch_add(1, std::memory_order_relaxed);
            }
            it += batch;
            if (ls == PMMF_OK) ls = all_done();
            if (ls != PMMF_OK) break;
        }
        cudaGraphExecDestroy(exec);
        PMMF_TRY(ls);
    }
    PMMF_CUDA_TRY(cudaMemcpyAsync(iters, itd.p, sizeof(int32_t) * nr, cudaMemcpyDeviceToHost, st));
    if (sym) {
        PMMF_TRY(apply_w(x, st));                       // x = W y
        PMMF_TRY(dots(b, b, n, nr, bb, part.p, st));    // ||b|| for relres
    }
    // true residual at exit
    PMMF_TRY(spmv(dA, x, qv.p, nr, st));
    PMMF_TRY(vec_sub(b, qv.p, r.p, n * nr, st));
    PMMF_TRY(dots(r.p, r.p, n, nr, rr, part.p, st));
    double hbb[8];
    PMMF_CUDA_TRY(cudaMemcpyAsync(hr, rr, sizeof(double) * nr, cudaMemcpyDeviceToHost, st));
    PMMF_CUDA_TRY(cudaMemcpyAsync(hbb, bb, sizeof(double) * nr, cudaMemcpyDeviceToHost, st));
    PMMF_CUDA_TRY(cudaStreamSynchronize(st));
    bool conv = true;
    for (int c = 0; c < nr; ++c) {
        relres[c] = hbb[c] > 0.0 ? std::sqrt(hr[c] / hbb[c]) : 0.0;
        conv = conv && hdone[c];
    }
    if (!conv) return fail(PMMF_ERR_NOT_CONVERGED, "PCG did not converge within maxit");
    return PMMF_OK;
}

}  // namespace
}  // namespace pmmf

extern "C" {

pmmf_status pmmf_solve_precond(const pmmf_handle *f, const pmmf_matrix *A, const double *b,
                               double *x, int64_t nrhs, double rtol, int maxit, int32_t *iters,
                               double *relres, void *stream) {
    return pmmf::solve_impl(f, A, b, x, nrhs, rtol, maxit, iters, relres, stream, false);
}

pmmf_status pmmf_solve_precond_sym(const pmmf_handle *f, const pmmf_matrix *A, const double *b,
                                   double *x, int64_t nrhs, double rtol, int maxit,
                                   int32_t *iters, double *relres, void *stream) {
    return pmmf::solve_impl(f, A, b, x, nrhs, rtol, maxit, iters, relres, stream, true);
}

pmmf_status pmmf_apply_backward(const pmmf_handle *fc, int op, const double *x, const double *g,
                                int64_t nrhs, int64_t ld, double *dx, double *dtheta,
                                double *dhdiag, double *dcore, void *stream) {
    set_error("");
    pmmf_handle *f = const_cast<pmmf_handle *>(fc);
    if (!f || !x || !g) return fail(PMMF_ERR_INVALID_ARG, "NULL handle or vector");
    if (nrhs < 1 || ld < nrhs) return fail(PMMF_ERR_INVALID_ARG, "need nrhs >= 1 and ld >= nrhs");
    if (op != PMMF_OP_A && op != PMMF_OP_A_INV)
        return fail(PMMF_ERR_INVALID_ARG, "backward is defined for PMMF_OP_A and PMMF_OP_A_INV");
    if (f->nblk > 1) return fail(PMMF_ERR_UNSUPPORTED, "backward of a batch handle is not built");
    cudaStream_t st = (cudaStream_t)stream;
    const bool inv = op == PMMF_OP_A_INV;
    if (inv) PMMF_TRY(ensure_inverse(f, st));
    std::vector<const RotRec *> recs;
    std::vector<const int32_t *> klvls;
    for (auto &S : f->st) {
        recs.push_back(S.rot.rec.p);
        klvls.push_back(S.rot.klvl.p);
    }
    return apply_backward(f->views, recs, klvls, hdata(f), inv, x, g, nrhs, ld, dx, dtheta, dhdiag,
                          dcore, st);
}

}  // extern "C"

namespace pmmf {
namespace {

// The Givens signs of every k-point block, formed once from the blocks as
// they are (theta_scratch receives their angles).
pmmf_status ensure_block_signs(pmmf_handle *f, StageData &S, double *theta_scratch,
                               cudaStream_t st) {
    if (S.rot.kD_ready) return block_angles(S.nrot, f->k, S.rot.kk.p, S.rot.kO.p, theta_scratch,
                                            nullptr, st);
    PMMF_TRY(S.rot.kD.alloc(std::max<int64_t>(S.nrot * f->k, 1), st));
    PMMF_TRY(block_angles(S.nrot, f->k, S.rot.kk.p, S.rot.kO.p, theta_scratch, S.rot.kD.p, st));
    S.rot.kD_ready = true;
    return PMMF_OK;
}

}  // namespace
}  // namespace pmmf

extern "C" {

pmmf_status pmmf_get_angles(const pmmf_handle *fc, double *theta, void *stream) {
    set_error("");
    pmmf_handle *f = const_cast<pmmf_handle *>(fc);
    if (!f || !theta) return fail(PMMF_ERR_INVALID_ARG, "NULL handle or output");
    if (f->nblk > 1) return fail(PMMF_ERR_UNSUPPORTED, "angles of a batch handle are not built");
    cudaStream_t st = (cudaStream_t)stream;
    int64_t off = 0;
    const int64_t per = f->k > 2 ? (int64_t)f->k * (f->k - 1) / 2 : 1;
    for (auto &S : f->st) {
        if (f->k > 2) PMMF_TRY(ensure_block_signs(f, S, theta + off * per, st));
        else PMMF_TRY(get_angles(S.rot.rec.p, S.nrot, theta + off, st));
        off += S.nrot;
    }
    return PMMF_OK;
}

pmmf_status pmmf_set_angles(pmmf_handle *f, const double *theta, void *stream) {
    set_error("");
    if (!f || !theta) return fail(PMMF_ERR_INVALID_ARG, "NULL handle or input");
    if (f->nblk > 1) return fail(PMMF_ERR_UNSUPPORTED, "angles of a batch handle are not built");
    cudaStream_t st = (cudaStream_t)stream;
    int64_t off = 0;
    const int64_t per = f->k > 2 ? (int64_t)f->k * (f->k - 1) / 2 : 1;
    for (size_t p = 0; p < f->st.size(); ++p) {
        StageData &S = f->st[p];
        if (f->k > 2) {
            if (!S.rot.kD_ready) {
                DBuf<double> scratch;
                PMMF_TRY(scratch.alloc(std::max<int64_t>(S.nrot * per, 1), st));
                PMMF_TRY(ensure_block_signs(f, S, scratch.p, st));
            }
            PMMF_TRY(block_from_angles(S.nrot, f->k, S.rot.kk.p, theta + off * per, S.rot.kD.p,
                                       S.rot.kO.p, st));
        } else {
            PMMF_TRY(set_angles(f->views[p], S.rot.rec.p, S.rot.lvl.p, theta + off, st));
        }
        off += S.nrot;
    }
    return PMMF_OK;
}

pmmf_status pmmf_block_angle_grad(const pmmf_handle *fc, const double *dO, double *dtheta,
                                  void *stream) {
    set_error("");
    pmmf_handle *f = const_cast<pmmf_handle *>(fc);
    if (!f || !dO || !dtheta) return fail(PMMF_ERR_INVALID_ARG, "NULL handle or array");
    if (f->k < 3) return fail(PMMF_ERR_UNSUPPORTED, "k = 2 rotations are angles already");
    if (f->nblk > 1) return fail(PMMF_ERR_UNSUPPORTED, "angles of a batch handle are not built");
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t per = (int64_t)f->k * (f->k - 1) / 2, kk2 = (int64_t)f->k * f->k;
    int64_t off = 0;
    for (auto &S : f->st) {
        DBuf<double> th;
        PMMF_TRY(th.alloc(std::max<int64_t>(S.nrot * per, 1), st));
        PMMF_TRY(ensure_block_signs(f, S, th.p, st));
        PMMF_TRY(block_angle_grad(S.nrot, f->k, S.rot.kk.p, th.p, S.rot.kD.p, dO + off * kk2,
                                  dtheta + off * per, st));
        off += S.nrot;
    }
    return PMMF_OK;
}

pmmf_status pmmf_set_h(pmmf_handle *f, const double *hdiag, const double *core, void *stream) {
    set_error("");
    if (!f) return fail(PMMF_ERR_INVALID_ARG, "NULL handle");
    cudaStream_t st = (cudaStream_t)stream;
    if (hdiag)
        PMMF_CUDA_TRY(cudaMemcpyAsync(f->hdiag.p, hdiag, sizeof(double) * (size_t)f->n,
                                      cudaMemcpyDeviceToDevice, st));
    if (core && f->nblk * f->bs > 0)
        PMMF_CUDA_TRY(cudaMemcpyAsync(f->core.p, core, sizeof(double) * (size_t)(f->nblk * f->bs * f->bs),
                                      cudaMemcpyDeviceToDevice, st));
    if (hdiag || core) f->inv_state = f->isqrt_state = 0;
    return PMMF_OK;
}

}  // extern "C"

namespace pmmf {

// Read-only view of a handle for the allocation-free apply.
pmmf_status handle_views(const pmmf_handle *f, const ApplyStages **views, HData *H, int64_t *n,
                         bool *inverse_ready, bool *isqrt_ready) {
    if (!f) return fail(PMMF_ERR_INVALID_ARG, "NULL handle");
    *views = &f->views;
    *H = hdata(f);
    *n = f->n;
    *inverse_ready = f->inv_state == 1;
    *isqrt_ready = f->isqrt_state == 1;
    return PMMF_OK;
}

}  // namespace pmmf
