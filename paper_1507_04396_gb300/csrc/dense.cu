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
                }
            }
        }
    }
}

// One CTA per row: the row in shared memory, every level's rotations applied
// in turn (rotations of one level touch disjoint positions).
__global__ void __launch_bounds__(256)
k_dense_rows(double *D, int64_t s, const int64_t *goffL, int nlv, DenseRotList L) {
    extern __shared__ double row[];
    const int64_t r = blockIdx.x;
    double *Dr = D + r * s;
    for (int64_t q = threadIdx.x; q < s; q += blockDim.x) row[q] = Dr[q];
    __syncthreads();
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
                double in[8];
                bool nz = false;
                for (int a = 0; a < kk; ++a) {
                    in[a] = row[P[a]];
                    nz |= nonzero_bits(in[a]);
                }
                if (nz) {
                    const double *O = L.kO + t * L.K * L.K;
                    double out[8];
                    for (int a = 0; a < kk; ++a) out[a] = rot_row(O, kk, a, in);
                    for (int a = 0; a < kk; ++a) row[P[a]] = out[a];
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
    if (sh > 48 * 1024)
        PMMF_CUDA_TRY(cudaFuncSetAttribute(k_dense_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh));
    DBuf<double> T;
    PMMF_TRY(T.alloc(s * s, st));
    // every pass reads and writes the s x s block once
    prof_begin(KF_ROWS, st);
    k_dense_rows<<<(unsigned)s, 256, sh, st>>>(D.p, s, lv.goffL.p, lv.nlv, lv.L);
    prof_end(KF_ROWS, st, 16.0 * (double)s * (double)s, 0.0);
    PMMF_TRY(launched("dense_rows"));
    dim3 tg((unsigned)((s + 31) / 32), (unsigned)((s + 31) / 32)), tb(32, 8);
    k_dense_transpose<<<tg, tb, 0, st>>>(D.p, s, T.p);
    PMMF_TRY(launched("dense_transpose"));
    prof_begin(KF_ROWS, st);
    k_dense_rows<<<(unsigned)s, 256, sh, st>>>(T.p, s, lv.goffL.p, lv.nlv, lv.L);
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
