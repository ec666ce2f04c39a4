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
#include <vector>

#include "common.cuh"
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

// Smaller-angle Jacobi rotation zeroing the off-diagonal of q [[a,b],[b,d]] q^T.
__device__ void jacobi2(double a, double b, double d, double &c, double &s) {
    if (b == 0.0) {
        c = 1.0;
        s = 0.0;
        return;
    }
    double zeta = __ddiv_rn(__dsub_rn(d, a), __dmul_rn(2.0, b));
    double t;
    if (fabs(zeta) > 1e150) {
        t = __ddiv_rn(1.0, __dmul_rn(2.0, zeta));
    } else {
        double r = __dsqrt_rn(__dadd_rn(1.0, __dmul_rn(zeta, zeta)));
        t = __ddiv_rn(zeta >= 0.0 ? 1.0 : -1.0, __dadd_rn(fabs(zeta), r));
    }
    c = __ddiv_rn(1.0, __dsqrt_rn(__dadd_rn(1.0, __dmul_rn(t, t))));
    s = __dmul_rn(t, c);
}

// New 2x2 block of q X q^T for symmetric X with X_ii = a, X_ij = X_ji = b,
// X_jj = d: row step R = q X_TT, then column step R q^T (upper half, mirrored).
__device__ void rot_block(double c, double s, double a, double b, double d, double &na, double &nb,
                          double &nd) {
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

// One warp per Gram row (cluster u, local a); lanes walk b >= a.  Each entry
// is a sequential fma chain over the common columns of rows x_a and x_b in
// ascending column order (terms where either entry is zero leave the chain
// unchanged, so only common stored columns matter).
__global__ void k_gram(const int64_t *rp, const int32_t *ci, const double *v, const int32_t *pos,
                       const int32_t *cl, const int64_t *coff, const int32_t *members, int64_t s,
                       const int64_t *goff, double *G, double *M) {
    int lane = threadIdx.x & 31;
    int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t j = w; j < s; j += nw) {
        int32_t xa = members[j];
        int64_t u = cl[xa];
        int64_t base = coff[u];
        int64_t c = coff[u + 1] - base;
        int64_t a = j - base;
        int64_t ra = pos[xa];
        int64_t a0 = rp[ra], a1 = rp[ra + 1];
        double *Gu = G + goff[u];
        double *Mu = M + goff[u];
        for (int64_t b = a + lane; b < c; b += 32) {
            int32_t xb = members[base + b];
            int64_t rb = pos[xb];
            int64_t pa = a0, pb = rp[rb], eb = rp[rb + 1];
            double acc = 0.0;
            while (pa < a1 && pb < eb) {
                int32_t ca = ci[pa], cb = ci[pb];
                if (ca < cb) {
                    ++pa;
                } else if (ca > cb) {
                    ++pb;
                } else {
                    acc = __fma_rn(v[pa], v[pb], acc);
                    ++pa;
                    ++pb;
                }
            }
            // M_ab = A[x_a][x_b] (x_a < x_b since members ascend)
            double mv = 0.0;
            int64_t lo = a0, hi = a1;
            while (lo < hi) {
                int64_t mid = (lo + hi) >> 1;
                int32_t cm = ci[mid];
                if (cm < xb) lo = mid + 1;
                else if (cm > xb) hi = mid;
                else { mv = v[mid]; break; }
            }
            Gu[a * c + b] = acc;
            Gu[b * c + a] = acc;
            Mu[a * c + b] = mv;
            Mu[b * c + a] = mv;
        }
    }
}

constexpr int SEL_THREADS = 256;

struct Best {
    double sc;
    int32_t idx;
};

__device__ __forceinline__ bool better(double s1, int32_t i1, double s2, int32_t i2) {
    return s1 > s2 || (s1 == s2 && i1 < i2);
}

// i = position 'pos' among the set bits of mask[0..nw) (one thread).
__device__ int select_bit(const uint32_t *mask, int nwords, int64_t pos) {
    int64_t rem = pos;
    for (int wi = 0; wi < nwords; ++wi) {
        uint32_t m = mask[wi];
        int pc = __popc(m);
        if (rem < pc) {
            for (int b = 0; b < 32; ++b) {
                if (m & (1u << b)) {
                    if (rem == 0) return wi * 32 + b;
                    --rem;
                }
            }
        }
        rem -= pc;
    }
    return -1;
}

// One CTA per cluster.  Shared memory: G and M diagonals, w, the active mask,
// per-coordinate dependency levels and level counters.
__global__ void __launch_bounds__(SEL_THREADS)
k_select(const int64_t *coff, const int32_t *members, const int64_t *goff, double *Gall,
         double *Mall, const int64_t *roff, uint64_t seed, int64_t stage, RotRec *rec, Rot2 *lvlrot,
         int32_t *lvl_off, int32_t *nlev, int32_t *elimflag) {
    extern __shared__ double sh[];
    const int64_t u = blockIdx.x;
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
    __shared__ Best wbest[SEL_THREADS / 32];
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
        if (e > 0) s_i = select_bit(mask, nwords, (int64_t)__umul64hi(draw(seed, stage, u, 0), (uint64_t)c));
    }
    __syncthreads();

    for (int t = 0; t < e; ++t) {
        // partner search over the active coordinates
        const int i = s_i < 0 ? 0 : s_i;
        const double *Gi = G + (int64_t)i * c;
        double bs = -1.0;
        int32_t bi = 0x7fffffff;
        for (int y = tid; y < c; y += SEL_THREADS) {
            if (y == i || !(mask[y >> 5] & (1u << (y & 31)))) continue;
            double sc = __dmul_rn(fabs(Gi[y]), w[y]);
            if (better(sc, y, bs, bi)) { bs = sc; bi = y; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            double os = __shfl_xor_sync(0xffffffffu, bs, o);
            int32_t oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (better(os, oi, bs, bi)) { bs = os; bi = oi; }
        }
        if (lane == 0) wbest[wid] = Best{bs, bi};
        __syncthreads();
        if (tid == 0) {
            for (int q = 1; q < SEL_THREADS / 32; ++q)
                if (better(wbest[q].sc, wbest[q].idx, bs, bi)) { bs = wbest[q].sc; bi = wbest[q].idx; }
            // at least two coordinates are active at every step (e_u <= c_u - 1);
            // the clamp only keeps a corrupted state from indexing out of bounds
            const int j = (bi >= 0 && bi < c && bi != i) ? bi : (i == 0 ? 1 : 0);
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
            elimflag[members[base + le]] = (int32_t)stage;
            mask[le >> 5] &= ~(1u << (le & 31));
            s_j = j;
            s_c = cc;
            s_s = ss;
            if (t + 1 < e)
                s_i = select_bit(mask, nwords,
                                 (int64_t)__umul64hi(draw(seed, stage, u, t + 1), (uint64_t)(c - t - 1)));
        }
        __syncthreads();
        // rows/columns i and j of G and M for every other active coordinate
        {
            const int j = s_j;
            const double cc = s_c, ss = s_s;
            double *Gj = G + (int64_t)j * c;
            double *Mi = M + (int64_t)i * c;
            double *Mj = M + (int64_t)j * c;
            double *Gw = G + (int64_t)i * c;
            for (int y = tid; y < c; y += SEL_THREADS) {
                if (y == i || y == j || !(mask[y >> 5] & (1u << (y & 31)))) continue;
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

    // group the rotations by dependency level (rotations of one level touch
    // disjoint coordinates, so any order inside a level gives the same bits)
    const int nl = s_maxlev;
    for (int t = tid; t < e; t += SEL_THREADS) atomicAdd(&lcnt[rec[r0 + t].lvl], 1);
    __syncthreads();
    if (tid == 0) {
        int acc = 0;
        for (int L = 1; L <= nl; ++L) {
            int cnt = lcnt[L];
            lcnt[L] = acc;
            lvl_off[r0 + u + L - 1] = (int32_t)(r0 + acc);
            acc += cnt;
        }
        lvl_off[r0 + u + nl] = (int32_t)(r0 + acc);
        nlev[u] = nl;
    }
    __syncthreads();
    for (int t = tid; t < e; t += SEL_THREADS) {
        RotRec rr = rec[r0 + t];
        int slot = atomicAdd(&lcnt[rr.lvl], 1);
        lvlrot[r0 + slot] = Rot2{rr.li, rr.lj, rr.c, rr.s};
    }
}

}  // namespace

pmmf_status gram_and_select(const Csr &A, const int32_t *pos, const int32_t *cl,
                            const StageClusters &cls, int64_t cmax, uint64_t seed, int64_t stage,
                            StageRotations &rot, int32_t *elimflag, cudaStream_t st) {
    const int64_t m = cls.m;
    DBuf<int64_t> goff;
    PMMF_TRY(goff.alloc(m + 1, st));
    k_square_sizes<<<grid_for(m, 256), 256, 0, st>>>(cls.coff.p, m, goff.p);
    PMMF_TRY(launched("square_sizes"));
    PMMF_TRY(scan_i64(goff.p, goff.p, m, st));
    int64_t gtot = 0;
    PMMF_CUDA_TRY(cudaMemcpyAsync(&gtot, goff.p + m, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    PMMF_CUDA_TRY(cudaStreamSynchronize(st));
    DBuf<double> G, M;
    PMMF_TRY(G.alloc(gtot, st));   // k_gram writes every entry of every cluster block
    PMMF_TRY(M.alloc(gtot, st));
    int64_t s = A.rows;
    prof_begin(KF_GRAM, st);
    k_gram<<<grid_for(s * 32, 256), 256, 0, st>>>(A.rowptr.p, A.col.p, A.val.p, pos, cl,
                                                   cls.coff.p, cls.members.p, s, goff.p, G.p, M.p);
    // compulsory traffic: the cluster rows once (12 B per entry, 8 B per row
    // pointer) and both c_u x c_u outputs
    prof_end(KF_GRAM, st, 12.0 * (double)A.nnz + 8.0 * (double)s + 16.0 * (double)gtot, 0.0);
    PMMF_TRY(launched("gram"));

    PMMF_TRY(rot.rec.alloc(rot.nrot > 0 ? rot.nrot : 1, st));
    PMMF_TRY(rot.lvl.alloc(rot.nrot > 0 ? rot.nrot : 1, st));
    PMMF_TRY(rot.lvl_off.alloc(rot.nrot + m + 1, st));
    PMMF_TRY(rot.nlev.zeros(m, st));
    size_t shb = sizeof(double) * 3 * (size_t)cmax + sizeof(uint32_t) * (size_t)((cmax + 31) / 32) +
                 sizeof(int32_t) * (size_t)(2 * cmax + 4);
    if (shb > 220 * 1024) {
        set_error("cluster too large for the selection kernel");
        return PMMF_ERR_UNSUPPORTED;
    }
    if (shb > 48 * 1024)
        PMMF_CUDA_TRY(cudaFuncSetAttribute(k_select, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shb));
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
    k_select<<<(unsigned)m, SEL_THREADS, shb, st>>>(cls.coff.p, cls.members.p, goff.p, G.p, M.p,
                                                    rot.roff.p, seed, stage, rot.rec.p, rot.lvl.p,
                                                    rot.lvl_off.p, rot.nlev.p, elimflag);
    prof_end(KF_SELECT, st, 0.0, sel_flops);
    PMMF_TRY(launched("select"));
    return PMMF_OK;
}

}  // namespace pmmf
