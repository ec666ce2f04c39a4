// shard.cu -- the steps of one pMMF stage as separate calls, for a stage split
// over several GPUs (Sec. 2.3: the clusters' searches are independent; the
// blocked update needs every cluster's rotations, and the matrix is
// redistributed between stages).  The host side that routes rows and
// rotations between ranks is paper_1507_04396_gb300/shard.py; every
// floating-point step runs here, in the same kernels as pmmf_factor, so a
// stage split over ranks gives pmmf_factor's rotations and H bit for bit.
#include <algorithm>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "stage.cuh"

struct pmmf_shard {
    int64_t n = 0;
    pmmf_params prm{};
    int dim = 0;
    pmmf::DBuf<int32_t> q, morder;     // quantized points and their Morton order
    pmmf::DBuf<int32_t> labels;        // stage-1 clusters, if given
    pmmf::DBuf<int32_t> elimflag;      // n: stage of a coordinate's elimination
    pmmf::DBuf<unsigned> status;
    // the last transform's rows
    pmmf::Csr out;
    pmmf::DBuf<int32_t> out_ids;
};

namespace pmmf {
namespace {

pmmf_status fail(pmmf_status s, const char *msg) {
    set_error(msg);
    return s;
}

// A DBuf that views caller memory for the duration of a call (never frees it).
template <class T>
struct View {
    DBuf<T> &b;
    View(DBuf<T> &buf, const T *p, int64_t n) : b(buf) {
        b.p = const_cast<T *>(p);
        b.n = n;
    }
    ~View() {
        b.p = nullptr;
        b.n = 0;
    }
};

// Global id -> cluster ordinal and index inside it, for the clusters of coff /
// members (one CTA per cluster); other entries of cl / loc are left as set.
__global__ void k_cluster_maps(const int64_t *coff, const int32_t *members, int32_t *cl,
                               int32_t *loc) {
    const int64_t u = blockIdx.x;
    for (int64_t j = coff[u] + threadIdx.x; j < coff[u + 1]; j += blockDim.x) {
        cl[members[j]] = (int32_t)u;
        loc[members[j]] = (int32_t)(j - coff[u]);
    }
}

template <class T>
pmmf_status to_host(std::vector<T> &h, const T *d, int64_t n, cudaStream_t st) {
    h.resize((size_t)std::max<int64_t>(n, 0));
    if (n > 0) PMMF_CUDA_TRY(cudaMemcpyAsync(h.data(), d, sizeof(T) * (size_t)n, cudaMemcpyDeviceToHost, st));
    return PMMF_OK;
}

template <class T>
pmmf_status to_dev(DBuf<T> &d, const std::vector<T> &h, cudaStream_t st) {
    PMMF_TRY(d.alloc(std::max<int64_t>((int64_t)h.size(), 1), st));
    if (!h.empty())
        PMMF_CUDA_TRY(cudaMemcpyAsync(d.p, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice, st));
    return PMMF_OK;
}

// A stage's rotations given with global ids (clusters in ordinal order, step
// order inside) as the internal tables of the row passes: local indices,
// dependency levels (1 + the largest level of the tuple's coordinates) and
// the level-grouped order with its per-cluster offsets.  Host-side: the
// tables are O(rotations).
pmmf_status import_rotations(int64_t n, int64_t m, const std::vector<int64_t> &coff,
                             const std::vector<int32_t> &members, int K, int64_t T,
                             const int32_t *dkk, const int32_t *didx, const double *dO,
                             const int32_t *delim, const int32_t *dcl, StageRotations &rot,
                             cudaStream_t st) {
    std::vector<int32_t> kk, idx, el, rc;
    std::vector<double> O;
    PMMF_TRY(to_host(kk, dkk, T, st));
    PMMF_TRY(to_host(idx, didx, T * K, st));
    PMMF_TRY(to_host(O, dO, T * K * K, st));
    PMMF_TRY(to_host(el, delim, T, st));
    PMMF_TRY(to_host(rc, dcl, T, st));
    PMMF_CUDA_TRY(cudaStreamSynchronize(st));
    std::vector<int32_t> loc((size_t)n, -1), lvl((size_t)n, 0);
    for (int64_t u = 0; u < m; ++u)
        for (int64_t j = coff[u]; j < coff[u + 1]; ++j) loc[members[j]] = (int32_t)(j - coff[u]);
    std::vector<int64_t> roff((size_t)m + 1, 0);
    for (int64_t t = 0; t < T; ++t) {
        if (rc[t] < 0 || rc[t] >= m || (t > 0 && rc[t] < rc[t - 1]))
            return fail(PMMF_ERR_INVALID_ARG, "rotations must be ordered by cluster ordinal");
        roff[(size_t)rc[t] + 1]++;
    }
    for (int64_t u = 0; u < m; ++u) roff[u + 1] += roff[u];
    std::vector<int32_t> rl((size_t)std::max<int64_t>(T, 1));   // each rotation's level
    std::vector<int32_t> lvl_off((size_t)(T + m + 1), 0), nlev((size_t)std::max<int64_t>(m, 1), 0);
    std::vector<int32_t> order((size_t)std::max<int64_t>(T, 1));  // level slot -> rotation
    for (int64_t u = 0; u < m; ++u) {
        const int64_t r0 = roff[u], e = roff[u + 1] - r0;
        int nl = 0;
        for (int64_t t = r0; t < r0 + e; ++t) {
            int L = 0;
            for (int a = 0; a < kk[t]; ++a) L = std::max(L, lvl[idx[t * K + a]]);
            ++L;
            for (int a = 0; a < kk[t]; ++a) lvl[idx[t * K + a]] = L;
            rl[t] = L;
            nl = std::max(nl, L);
        }
        std::vector<int32_t> cnt((size_t)nl + 2, 0);
        for (int64_t t = r0; t < r0 + e; ++t) cnt[rl[t]]++;
        int acc = 0;
        for (int L = 1; L <= nl; ++L) {
            lvl_off[r0 + u + L - 1] = (int32_t)(r0 + acc);
            const int c = cnt[L];
            cnt[L] = acc;
            acc += c;
        }
        lvl_off[r0 + u + nl] = (int32_t)(r0 + acc);
        nlev[u] = nl;
        for (int64_t t = r0; t < r0 + e; ++t) order[r0 + cnt[rl[t]]++] = (int32_t)t;
        for (int64_t t = r0; t < r0 + e; ++t)
            for (int a = 0; a < kk[t]; ++a) lvl[idx[t * K + a]] = 0;   // levels restart per stage
    }
    rot.nrot = T;
    rot.K = K;
    PMMF_TRY(to_dev(rot.roff, roff, st));
    PMMF_TRY(to_dev(rot.lvl_off, lvl_off, st));
    PMMF_TRY(to_dev(rot.nlev, nlev, st));
    if (K <= 2) {
        std::vector<RotRec> rec((size_t)std::max<int64_t>(T, 1));
        std::vector<Rot2> lr((size_t)std::max<int64_t>(T, 1));
        for (int64_t t = 0; t < T; ++t) {
            const int32_t li = loc[idx[t * K]], lj = loc[idx[t * K + 1]];
            // the block [[c, -s], [s, c]]
            rec[t] = RotRec{li, lj, loc[el[t]], rl[t], O[t * 4 + 0], O[t * 4 + 2]};
        }
        for (int64_t q = 0; q < T; ++q) {
            const RotRec &r = rec[order[q]];
            lr[q] = Rot2{r.li, r.lj, r.c, r.s};
        }
        if (T == 0) {
            rec.clear();
            lr.clear();
        }
        PMMF_TRY(to_dev(rot.rec, rec, st));
        PMMF_TRY(to_dev(rot.lvl, lr, st));
    } else {
        std::vector<int32_t> li((size_t)(T * K)), kel((size_t)T), lidx((size_t)T);
        for (int64_t t = 0; t < T; ++t) {
            for (int a = 0; a < K; ++a) li[t * K + a] = a < kk[t] ? loc[idx[t * K + a]] : -1;
            kel[t] = loc[el[t]];
            lidx[t] = order[t];
        }
        PMMF_TRY(to_dev(rot.kidx, li, st));
        PMMF_TRY(to_dev(rot.kk, kk, st));
        PMMF_TRY(to_dev(rot.kel, kel, st));
        PMMF_TRY(to_dev(rot.klvl, rl, st));
        PMMF_TRY(to_dev(rot.lvlidx, lidx, st));
        PMMF_TRY(to_dev(rot.kO, O, st));
    }
    // the host vectors are copied before they go out of scope
    PMMF_CUDA_TRY(cudaStreamSynchronize(st));
    return PMMF_OK;
}

}  // namespace
}  // namespace pmmf

using namespace pmmf;

extern "C" {

pmmf_status pmmf_shard_create(int64_t n, const pmmf_params *p, pmmf_shard **out, void *stream) {
    set_error("");
    if (!out || !p) return fail(PMMF_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    if (n < 1 || n >= INT32_MAX) return fail(PMMF_ERR_INVALID_ARG, "n must be in [1, 2^31)");
    if (p->k < 2 || p->k > 8 || !(p->eta > 0.0 && p->eta < 1.0) || p->cluster_size < p->k ||
        p->core_size < 1 || p->core_size > n)
        return fail(PMMF_ERR_INVALID_ARG, "parameter out of range");
    if (p->coords && (p->coord_dim < 1 || p->coord_dim > 3))
        return fail(PMMF_ERR_INVALID_ARG, "coord_dim must be 1, 2 or 3");
    cudaStream_t st = (cudaStream_t)stream;
    pmmf_shard *h = new (std::nothrow) pmmf_shard();
    if (!h) return fail(PMMF_ERR_OOM, "host allocation failed");
    h->n = n;
    h->prm = *p;
    h->prm.coords = nullptr;
    h->prm.labels = nullptr;
    auto bad = [&](pmmf_status s) {
        set_free_sync(true);
        delete h;
        set_free_sync(false);
        return s;
    };
    pmmf_status s = h->status.zeros(1, st);
    if (s == PMMF_OK) s = h->elimflag.zeros(n, st);
    if (s == PMMF_OK && p->coords) {
        h->dim = p->coord_dim;
        DBuf<double> dc;
        DBuf<uint64_t> code;
        const double *cp = p->coords;
        if (p->coords_location != PMMF_DEVICE) {
            s = dc.alloc(n * h->dim, st);
            if (s == PMMF_OK &&
                cudaMemcpyAsync(dc.p, p->coords, sizeof(double) * (size_t)(n * h->dim),
                                cudaMemcpyHostToDevice, st) != cudaSuccess)
                s = fail(PMMF_ERR_CUDA, "copying coords failed");
            cp = dc.p;
        }
        if (s == PMMF_OK) s = h->q.alloc(n * h->dim, st);
        if (s == PMMF_OK) s = code.alloc(n, st);
        if (s == PMMF_OK) s = quantize_points(cp, n, h->dim, h->q.p, code.p, h->status.p, st);
        if (s == PMMF_OK) s = h->morder.alloc(n, st);
        if (s == PMMF_OK) s = radix_sort_u64(code.p, n, 15 * h->dim, h->morder.p, st);
        if (s == PMMF_OK && cudaStreamSynchronize(st) != cudaSuccess)
            s = fail(PMMF_ERR_CUDA, "synchronize failed");
    }
    if (s == PMMF_OK && p->labels) {
        s = h->labels.alloc(n, st);
        if (s == PMMF_OK &&
            cudaMemcpyAsync(h->labels.p, p->labels, sizeof(int32_t) * (size_t)n,
                            p->labels_location == PMMF_DEVICE ? cudaMemcpyDeviceToDevice
                                                              : cudaMemcpyHostToDevice,
                            st) != cudaSuccess)
            s = fail(PMMF_ERR_CUDA, "copying labels failed");
        h->prm.num_labels = p->num_labels;
    }
    if (s != PMMF_OK) return bad(s);
    *out = h;
    return PMMF_OK;
}

void pmmf_shard_free(pmmf_shard *sh) {
    if (!sh) return;
    cudaDeviceSynchronize();
    set_free_sync(true);
    delete sh;
    set_free_sync(false);
}

pmmf_status pmmf_shard_clusters(pmmf_shard *sh, int64_t stage, int64_t s, const int32_t *act,
                                int64_t *m_out, int64_t *coff, int32_t *members, int64_t *e,
                                void *stream) {
    set_error("");
    if (!sh || !act || !m_out || !coff || !members || !e || s < 1 || s > sh->n || stage < 1)
        return fail(PMMF_ERR_INVALID_ARG, "bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = sh->n;
    const pmmf_params &prm = sh->prm;
    DBuf<int32_t> pos, cl, loc;
    PMMF_TRY(pos.alloc(n, st));
    PMMF_TRY(cl.alloc(n, st));
    PMMF_TRY(loc.alloc(n, st));
    PMMF_CUDA_TRY(cudaMemsetAsync(pos.p, 0xFF, sizeof(int32_t) * (size_t)n, st));
    PMMF_TRY(set_positions(act, s, pos.p, st));
    StageClusters cls;
    int64_t m = (s + prm.cluster_size / 2) / prm.cluster_size;
    if (m < 1 || !sh->q.p) m = 1;
    const bool given = stage == 1 && sh->labels.p;
    if (m > 1 || given) {
        PartitionIn in;
        in.n = n;
        in.s = s;
        in.dim = sh->dim;
        in.q = sh->q.p;
        in.morder = sh->morder.p;
        in.pos = pos.p;
        in.act = act;
        in.cl = cl.p;
        in.loc = loc.p;
        if (given) PMMF_TRY(partition_from_labels(in, sh->labels.p, prm.num_labels, cls, st));
        else PMMF_TRY(partition_stage(in, m, prm.lloyd_iters > 0 ? prm.lloyd_iters : 10, cls, st));
    } else {
        PMMF_TRY(one_cluster(act, s, cls, cl.p, loc.p, st));
    }
    DBuf<int64_t> de, droff;
    int64_t sched[5] = {0, 0, 0, 0, 0};
    PMMF_TRY(schedule_stage(cls.coff.p, cls.m, cls.count_d.p, s, prm.core_size, prm.eta, de, droff,
                            sched, st));
    if (sched[1]) PMMF_TRY(one_cluster(act, s, cls, cl.p, loc.p, st));
    const int64_t mm = sched[1] ? 1 : sched[4];
    *m_out = mm;
    PMMF_CUDA_TRY(cudaMemcpyAsync(coff, cls.coff.p, sizeof(int64_t) * (size_t)(mm + 1), cudaMemcpyDeviceToDevice, st));
    PMMF_CUDA_TRY(cudaMemcpyAsync(members, cls.members.p, sizeof(int32_t) * (size_t)s, cudaMemcpyDeviceToDevice, st));
    PMMF_CUDA_TRY(cudaMemcpyAsync(e, de.p, sizeof(int64_t) * (size_t)mm, cudaMemcpyDeviceToDevice, st));
    PMMF_CUDA_TRY(cudaStreamSynchronize(st));
    return PMMF_OK;
}

pmmf_status pmmf_shard_search(pmmf_shard *sh, int64_t stage, int64_t s, const int32_t *act,
                              const int64_t *rowptr, const int32_t *col, const double *val,
                              int64_t m, const int64_t *coff, const int32_t *members,
                              const int64_t *e, int64_t nown, const int32_t *own,
                              int32_t *rcluster, int32_t *rkk, int32_t *ridx, double *rO,
                              int32_t *relim, void *stream) {
    set_error("");
    if (!sh || !act || !rowptr || !coff || !members || !e || s < 1 || m < 1 || nown < 0 ||
        (nown > 0 && !own) || stage < 1)
        return fail(PMMF_ERR_INVALID_ARG, "bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = sh->n;
    const int K = sh->prm.k;
    std::vector<int64_t> hcoff, he;
    std::vector<int32_t> hown;
    PMMF_TRY(to_host(hcoff, coff, m + 1, st));
    PMMF_TRY(to_host(he, e, m, st));
    PMMF_TRY(to_host(hown, own, nown, st));
    int64_t nnz = 0;
    PMMF_CUDA_TRY(cudaMemcpyAsync(&nnz, rowptr + s, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    PMMF_CUDA_TRY(cudaStreamSynchronize(st));
    // the owned clusters, numbered 0..nown-1, and their members
    std::vector<int64_t> lcoff((size_t)nown + 1, 0), lroff((size_t)nown + 1, 0);
    int64_t cmax = 0, g2 = 0;
    for (int64_t b = 0; b < nown; ++b) {
        const int64_t u = hown[b];
        if (u < 0 || u >= m || (b > 0 && u <= hown[b - 1]))
            return fail(PMMF_ERR_INVALID_ARG, "owned clusters must be ascending ordinals");
        const int64_t c = hcoff[u + 1] - hcoff[u];
        lcoff[b + 1] = lcoff[b] + c;
        lroff[b + 1] = lroff[b] + he[u];
        cmax = std::max(cmax, c);
        g2 += c * c;
    }
    const int64_t T = lroff[nown], nmem = lcoff[nown];
    if (T == 0) return PMMF_OK;
    StageClusters cls;
    cls.m = nown;
    PMMF_TRY(to_dev(cls.coff, lcoff, st));
    PMMF_TRY(cls.members.alloc(std::max<int64_t>(nmem, 1), st));
    for (int64_t b = 0; b < nown; ++b) {
        const int64_t u = hown[b];
        const int64_t c = hcoff[u + 1] - hcoff[u];
        if (c > 0)
            PMMF_CUDA_TRY(cudaMemcpyAsync(cls.members.p + lcoff[b], members + hcoff[u],
                                          sizeof(int32_t) * (size_t)c, cudaMemcpyDeviceToDevice, st));
    }
    DBuf<int32_t> ords, pos, cl, loc;
    PMMF_TRY(to_dev(ords, hown, st));
    PMMF_TRY(pos.alloc(n, st));
    PMMF_TRY(cl.alloc(n, st));
    PMMF_TRY(loc.alloc(n, st));
    PMMF_CUDA_TRY(cudaMemsetAsync(pos.p, 0xFF, sizeof(int32_t) * (size_t)n, st));
    PMMF_CUDA_TRY(cudaMemsetAsync(cl.p, 0xFF, sizeof(int32_t) * (size_t)n, st));
    PMMF_CUDA_TRY(cudaMemsetAsync(loc.p, 0xFF, sizeof(int32_t) * (size_t)n, st));
    PMMF_TRY(set_positions(act, s, pos.p, st));
    k_cluster_maps<<<(unsigned)nown, 128, 0, st>>>(cls.coff.p, cls.members.p, cl.p, loc.p);
    PMMF_TRY(launched("cluster_maps"));
    StageRotations rot;
    rot.K = K;
    rot.nrot = T;
    PMMF_TRY(to_dev(rot.roff, lroff, st));
    // the rows as a CSR over the whole active set (rows of other clusters empty)
    Csr A;
    A.rows = s;
    A.nnz = nnz;
    View<int64_t> vr(A.rowptr, rowptr, s + 1);
    View<int32_t> vc(A.col, col, nnz);
    View<double> vv(A.val, val, nnz);
    PMMF_CUDA_TRY(cudaMemsetAsync(sh->status.p, 0, sizeof(unsigned), st));
    PMMF_TRY(gram_and_select(A, act, pos.p, cl.p, loc.p, cls, cmax, sh->prm.seed, stage, rot,
                             sh->elimflag.p, st, nullptr, nullptr, sh->status.p, g2, ords.p, nmem));
    // the rotations with global ids, owned clusters in order
    std::vector<int32_t> mem, okk((size_t)T), oidx((size_t)(T * K)), oel((size_t)T), ocl((size_t)T);
    std::vector<double> oO((size_t)(T * K * K));
    PMMF_TRY(to_host(mem, cls.members.p, nmem, st));
    unsigned hs = 0;
    PMMF_CUDA_TRY(cudaMemcpyAsync(&hs, sh->status.p, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    if (K <= 2) {
        std::vector<RotRec> rec;
        PMMF_TRY(to_host(rec, rot.rec.p, T, st));
        PMMF_CUDA_TRY(cudaStreamSynchronize(st));
        for (int64_t b = 0; b < nown; ++b)
            for (int64_t t = lroff[b]; t < lroff[b + 1]; ++t) {
                const RotRec &r = rec[t];
                const int64_t base = lcoff[b];
                ocl[t] = hown[b];
                okk[t] = 2;
                oidx[t * 2] = mem[base + r.li];
                oidx[t * 2 + 1] = mem[base + r.lj];
                oO[t * 4 + 0] = r.c;
                oO[t * 4 + 1] = -r.s;
                oO[t * 4 + 2] = r.s;
                oO[t * 4 + 3] = r.c;
                oel[t] = mem[base + r.le];
            }
    } else {
        std::vector<int32_t> ki, kk, ke;
        std::vector<double> ko;
        PMMF_TRY(to_host(ki, rot.kidx.p, T * K, st));
        PMMF_TRY(to_host(kk, rot.kk.p, T, st));
        PMMF_TRY(to_host(ke, rot.kel.p, T, st));
        PMMF_TRY(to_host(ko, rot.kO.p, T * K * K, st));
        PMMF_CUDA_TRY(cudaStreamSynchronize(st));
        for (int64_t b = 0; b < nown; ++b)
            for (int64_t t = lroff[b]; t < lroff[b + 1]; ++t) {
                const int64_t base = lcoff[b];
                ocl[t] = hown[b];
                okk[t] = kk[t];
                for (int a = 0; a < K; ++a) oidx[t * K + a] = ki[t * K + a] >= 0 ? mem[base + ki[t * K + a]] : -1;
                for (int a = 0; a < K * K; ++a) oO[t * K * K + a] = ko[t * K * K + a];
                oel[t] = mem[base + ke[t]];
            }
    }
    if (hs & ST_NOT_CONVERGED) return fail(PMMF_ERR_NOT_CONVERGED, "k x k Jacobi did not converge in 32 sweeps");
    PMMF_CUDA_TRY(cudaMemcpyAsync(rcluster, ocl.data(), sizeof(int32_t) * (size_t)T, cudaMemcpyHostToDevice, st));
    PMMF_CUDA_TRY(cudaMemcpyAsync(rkk, okk.data(), sizeof(int32_t) * (size_t)T, cudaMemcpyHostToDevice, st));
    PMMF_CUDA_TRY(cudaMemcpyAsync(ridx, oidx.data(), sizeof(int32_t) * (size_t)(T * K), cudaMemcpyHostToDevice, st));
    PMMF_CUDA_TRY(cudaMemcpyAsync(rO, oO.data(), sizeof(double) * (size_t)(T * K * K), cudaMemcpyHostToDevice, st));
    PMMF_CUDA_TRY(cudaMemcpyAsync(relim, oel.data(), sizeof(int32_t) * (size_t)T, cudaMemcpyHostToDevice, st));
    PMMF_CUDA_TRY(cudaStreamSynchronize(st));
    return PMMF_OK;
}

pmmf_status pmmf_shard_transform(pmmf_shard *sh, int64_t stage, int account, int64_t nrows,
                                 const int32_t *ids, const int64_t *rowptr, const int32_t *col,
                                 const double *val, int64_t s, int64_t m, const int64_t *coff,
                                 const int32_t *members, int64_t nrot, const int32_t *rcluster,
                                 const int32_t *rkk, const int32_t *ridx, const double *rO,
                                 const int32_t *relim, double *hdiag, double *contrib,
                                 int64_t *out_rows, int64_t *out_nnz, void *stream) {
    set_error("");
    if (!sh || nrows < 0 || (nrows > 0 && (!ids || !rowptr)) || !coff || !members || m < 1 ||
        s < 1 || nrot < 0 || !out_rows || !out_nnz || (account && (!hdiag || !contrib)) ||
        stage < 1)
        return fail(PMMF_ERR_INVALID_ARG, "bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = sh->n;
    const int K = sh->prm.k;
    std::vector<int64_t> hcoff;
    std::vector<int32_t> hmem;
    PMMF_TRY(to_host(hcoff, coff, m + 1, st));
    PMMF_TRY(to_host(hmem, members, s, st));
    PMMF_CUDA_TRY(cudaStreamSynchronize(st));
    int64_t cmax = 1;
    for (int64_t u = 0; u < m; ++u) cmax = std::max(cmax, hcoff[u + 1] - hcoff[u]);
    StageRotations rot;
    PMMF_TRY(import_rotations(n, m, hcoff, hmem, K, nrot, rkk, ridx, rO, relim, rcluster, rot, st));
    StageClusters cls;
    cls.m = m;
    View<int64_t> vco(cls.coff, coff, m + 1);
    View<int32_t> vme(cls.members, members, s);
    DBuf<int32_t> cl, loc;
    PMMF_TRY(cl.alloc(n, st));
    PMMF_TRY(loc.alloc(n, st));
    PMMF_CUDA_TRY(cudaMemsetAsync(cl.p, 0xFF, sizeof(int32_t) * (size_t)n, st));
    PMMF_CUDA_TRY(cudaMemsetAsync(loc.p, 0xFF, sizeof(int32_t) * (size_t)n, st));
    k_cluster_maps<<<(unsigned)m, 128, 0, st>>>(coff, members, cl.p, loc.p);
    PMMF_TRY(launched("cluster_maps"));
    // this stage's eliminations (accounting only)
    DBuf<double> dummy;
    if (account) {
        std::vector<int32_t> hel;
        PMMF_TRY(to_host(hel, relim, nrot, st));
        PMMF_CUDA_TRY(cudaStreamSynchronize(st));
        std::vector<int32_t> flag((size_t)n, 0);
        for (int32_t x : hel) flag[x] = 1;
        PMMF_CUDA_TRY(cudaMemcpyAsync(sh->elimflag.p, flag.data(), sizeof(int32_t) * (size_t)n,
                                      cudaMemcpyHostToDevice, st));
    } else {
        PMMF_TRY(dummy.zeros(2, st));
    }
    int64_t nnz = 0;
    if (nrows > 0) {
        PMMF_CUDA_TRY(cudaMemcpyAsync(&nnz, rowptr + nrows, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        PMMF_CUDA_TRY(cudaStreamSynchronize(st));
    }
    Csr R;
    R.rows = nrows;
    R.nnz = nnz;
    DBuf<int64_t> rp0;
    if (nrows == 0) PMMF_TRY(rp0.zeros(1, st));
    View<int64_t> vr(R.rowptr, nrows > 0 ? rowptr : rp0.p, nrows + 1);
    View<int32_t> vc(R.col, col, nnz);
    View<double> vv(R.val, val, nnz);
    PMMF_CUDA_TRY(cudaMemsetAsync(sh->status.p, 0, sizeof(unsigned), st));
    // accounting marks with 1: stage 1 selects them; plain passes never match (-1)
    PMMF_TRY(transform_stage(R, ids, cl.p, loc.p, cls, cmax, rot, sh->elimflag.p, account ? 1 : -1,
                             account ? hdiag : dummy.p, account ? contrib : dummy.p + 1, sh->out,
                             sh->out_ids, sh->status.p, st));
    unsigned hs = 0;
    PMMF_CUDA_TRY(cudaMemcpyAsync(&hs, sh->status.p, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    PMMF_CUDA_TRY(cudaStreamSynchronize(st));
    if (hs & ST_ROW_TOO_LONG) return fail(PMMF_ERR_UNSUPPORTED, "transform: output row too long");
    *out_rows = sh->out.rows;
    *out_nnz = sh->out.nnz;
    return PMMF_OK;
}

pmmf_status pmmf_shard_result(const pmmf_shard *sh, int32_t *ids, int64_t *rowptr, int32_t *col,
                              double *val, void *stream) {
    if (!sh) return fail(PMMF_ERR_INVALID_ARG, "NULL shard");
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t r = sh->out.rows, z = sh->out.nnz;
    if (ids && r > 0)
        PMMF_CUDA_TRY(cudaMemcpyAsync(ids, sh->out_ids.p, sizeof(int32_t) * (size_t)r, cudaMemcpyDeviceToDevice, st));
    if (rowptr)
        PMMF_CUDA_TRY(cudaMemcpyAsync(rowptr, sh->out.rowptr.p, sizeof(int64_t) * (size_t)(r + 1), cudaMemcpyDeviceToDevice, st));
    if (col && z > 0)
        PMMF_CUDA_TRY(cudaMemcpyAsync(col, sh->out.col.p, sizeof(int32_t) * (size_t)z, cudaMemcpyDeviceToDevice, st));
    if (val && z > 0)
        PMMF_CUDA_TRY(cudaMemcpyAsync(val, sh->out.val.p, sizeof(double) * (size_t)z, cudaMemcpyDeviceToDevice, st));
    return PMMF_OK;
}

pmmf_status pmmf_shard_sumsq(const double *val, int64_t nnz, double *out, void *stream) {
    set_error("");
    if (!out || nnz < 0 || (nnz > 0 && !val)) return fail(PMMF_ERR_INVALID_ARG, "bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    DBuf<double> d;
    PMMF_TRY(d.zeros(1, st));
    if (nnz > 0) PMMF_TRY(sum_squares(val, nnz, d.p, st));
    PMMF_CUDA_TRY(cudaMemcpyAsync(out, d.p, sizeof(double), cudaMemcpyDeviceToHost, st));
    PMMF_CUDA_TRY(cudaStreamSynchronize(st));
    return PMMF_OK;
}

}  // extern "C"
