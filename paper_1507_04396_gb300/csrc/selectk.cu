// selectk.cu -- the rotation search of Algorithm 2 with k-point rotations
// (k >= 3; Sec. 2.2), one CTA per cluster.  Per step t:
//   pick      i = the r * |I| / 2^64-th active index, r from splitmix64
//   partners  the kk - 1 active j != i of largest |G_ij| * w_j (w_j =
//             1 / sqrt(G_jj), 0 if G_jj <= 0), in decreasing score order,
//             ties to the smaller index; kk = min(k, |I|)
//   rotation  O diagonalizing the kk x kk Gram sub-block: the smaller-angle
//             Jacobi rotation for kk = 2, cyclic Jacobi otherwise (R7)
//   update    G <- O G O^T and M <- O M O^T on the tuple (rows recomputed and
//             mirrored, the tuple block as (O X_TT) O^T)
//   eliminate the tuple member of smallest G_xx - M_xx^2, ties to the later
//             tuple position
// The arithmetic is that of a sequential FP64 evaluation in this order, so
// the rotations equal it bit for bit.
#include "common.cuh"
#include "rotmath.cuh"
#include "stage.cuh"

namespace pmmf {
namespace {

constexpr int KS_THREADS = 256;
constexpr int KS_WARPS = KS_THREADS / 32;
constexpr unsigned long long EXCL = ~0ull;   // not a candidate

__device__ __forceinline__ uint64_t mixk(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t drawk(uint64_t seed, uint64_t p, uint64_t u, uint64_t t) {
    uint64_t h = mixk(seed);
    h = mixk(h ^ p);
    h = mixk(h ^ u);
    return mixk(h ^ t);
}

__device__ __forceinline__ bool active_bit(const uint32_t *mask, int y) {
    return (mask[y >> 5] >> (y & 31)) & 1u;
}

// The pos-th set bit of mask (one thread).
__device__ int nth_active(const uint32_t *mask, int nwords, int64_t pos) {
    int rem = (int)pos;
    for (int wi = 0; wi < nwords; ++wi) {
        const uint32_t m = mask[wi];
        const int pc = __popc(m);
        if (rem < pc) {
            for (int b = 0; b < 32; ++b)
                if ((m >> b) & 1u) {
                    if (rem == 0) return wi * 32 + b;
                    --rem;
                }
        }
        rem -= pc;
    }
    return -1;
}

__device__ __forceinline__ bool better(unsigned long long k1, int i1, unsigned long long k2, int i2) {
    return k1 > k2 || (k1 == k2 && i1 < i2);
}

// KM: the largest tuple (3 for k = 3, 8 otherwise); the tuple's arrays are
// sized by it and their loops unrolled.
template <int KM>
__global__ void __launch_bounds__(KS_THREADS)
k_select_k(const int64_t *coff, const int32_t *members, const int64_t *goff, double *Gall,
           double *Mall, const int64_t *roff, uint64_t seed, int64_t stage, int K, int32_t *kidx,
           int32_t *kkv, int32_t *kel, int32_t *klvl, double *kO, int32_t *lvlidx,
           int32_t *lvl_off, int32_t *nlev, int32_t *elimflag, const int32_t *order,
           const uint64_t *useed, unsigned *status, const int32_t *ords) {
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
    unsigned long long *key = (unsigned long long *)(w + c);
    const int nwords = (c + 31) / 32;
    uint32_t *mask = (uint32_t *)(key + c);
    int32_t *lvl = (int32_t *)(mask + nwords);
    int32_t *lcnt = lvl + c;   // e + 2
    __shared__ int s_T[8], s_kk, s_maxlev;
    __shared__ double s_O[64], s_g[64], s_J[4], s_R[4], s_RT[2][64];
    __shared__ unsigned long long s_bk[KS_WARPS];
    __shared__ int s_bi[KS_WARPS];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const uint64_t sd = useed ? useed[u] : seed;
    const uint64_t uu = useed ? 0 : (uint64_t)(ords ? ords[u] : u);

    for (int a = tid; a < c; a += KS_THREADS) {
        const double g = G[(int64_t)a * c + a];
        gd[a] = g;
        md[a] = M[(int64_t)a * c + a];
        w[a] = g > 0.0 ? __ddiv_rn(1.0, __dsqrt_rn(g)) : 0.0;
        lvl[a] = 0;
    }
    for (int wi = tid; wi < nwords; wi += KS_THREADS) {
        const int rem = c - wi * 32;
        mask[wi] = rem >= 32 ? 0xffffffffu : ((1u << rem) - 1u);
    }
    for (int q = tid; q < e + 2; q += KS_THREADS) lcnt[q] = 0;
    if (tid == 0) s_maxlev = 0;
    __syncthreads();

    int na = c;
    for (int t = 0; t < e; ++t, --na) {
        if (tid == 0) {
            const uint64_t r = drawk(sd, (uint64_t)stage, uu, (uint64_t)t);
            s_T[0] = nth_active(mask, nwords, (int64_t)__umul64hi(r, (uint64_t)na));
            s_kk = K < na ? K : na;
        }
        __syncthreads();
        const int i = s_T[0], kk = s_kk;
        for (int y = tid; y < c; y += KS_THREADS) {
            unsigned long long kv = EXCL;
            if (y != i && active_bit(mask, y)) {
                const double g = G[(int64_t)i * c + y];
                // |g| * w = |g * w| bit for bit (round to nearest is symmetric)
                kv = f64_bits(__dmul_rn(g, w[y])) & F64_ABS;
            }
            key[y] = kv;
        }
        __syncthreads();
        for (int a = 1; a < kk; ++a) {
            unsigned long long bk = 0;
            int bi = 0x7fffffff;
            for (int y = tid; y < c; y += KS_THREADS) {
                const unsigned long long kv = key[y];
                if (kv != EXCL && (bi == 0x7fffffff || better(kv, y, bk, bi))) {
                    bk = kv;
                    bi = y;
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long ok = __shfl_xor_sync(0xffffffffu, bk, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (oi != 0x7fffffff && (bi == 0x7fffffff || better(ok, oi, bk, bi))) {
                    bk = ok;
                    bi = oi;
                }
            }
            if (lane == 0) {
                s_bk[wid] = bk;
                s_bi[wid] = bi;
            }
            __syncthreads();
            if (tid == 0) {
                unsigned long long fk = s_bk[0];
                int fi = s_bi[0];
                for (int q = 1; q < KS_WARPS; ++q)
                    if (s_bi[q] != 0x7fffffff && (fi == 0x7fffffff || better(s_bk[q], s_bi[q], fk, fi))) {
                        fk = s_bk[q];
                        fi = s_bi[q];
                    }
                s_T[a] = fi;
                key[fi] = EXCL;
            }
            __syncthreads();
        }
        int T[KM];
#pragma unroll
        for (int a = 0; a < KM; ++a) T[a] = a < kk ? s_T[a] : -1;
        if (wid == 0) {
            if (kk == 2) {
                if (lane == 0) {
                    double cc, ss;
                    jacobi2(G[(int64_t)T[0] * c + T[0]], G[(int64_t)T[0] * c + T[1]],
                            G[(int64_t)T[1] * c + T[1]], cc, ss);
                    s_O[0] = cc;
                    s_O[1] = -ss;
                    s_O[2] = ss;
                    s_O[3] = cc;
                }
            } else {
                // the k x k block diagonalised by the warp
                for (int a = lane; a < kk * kk; a += 32) s_g[a] = G[(int64_t)T[a / kk] * c + T[a % kk]];
                __syncwarp();
                const bool ok = jacobi_k_warp(kk, s_g, s_O, s_J, s_R);
                if (lane == 0 && !ok) atomicOr(status, ST_NOT_CONVERGED);
            }
        }
        __syncthreads();
        // the tuple block of G and M, R = O X_TT then R O^T (upper half,
        // mirrored), by warp 0 one entry per lane; its inputs are not among
        // the entries the other warps rotate
        if (wid == 0) {
            const int nR = 2 * kk * kk;
            for (int q = lane; q < nR; q += 32) {
                const int mat = q / (kk * kk), t = q - mat * kk * kk;
                const int a = t / kk, cc = t - a * kk;
                const double *X = mat ? M : G;
                double in[KM];
#pragma unroll
                for (int b = 0; b < KM; ++b) in[b] = b < kk ? X[(int64_t)s_T[b] * c + s_T[cc]] : 0.0;
                s_RT[mat][a * kk + cc] = rot_row_u<KM>(s_O, kk, a, in);
            }
            __syncwarp();
            const int nup = kk * (kk + 1) / 2;
            for (int q = lane; q < 2 * nup; q += 32) {
                const int mat = q / nup;
                int t = q - mat * nup, a = 0;
                while (t >= kk - a) {   // (a, b), a <= b, in row order
                    t -= kk - a;
                    ++a;
                }
                const int b = a + t;
                const double *R = s_RT[mat];
                double acc = __dmul_rn(R[a * kk + kk - 1], s_O[b * kk + kk - 1]);
                for (int cc = kk - 2; cc >= 0; --cc) acc = __fma_rn(R[a * kk + cc], s_O[b * kk + cc], acc);
                double *X = mat ? M : G;
                X[(int64_t)s_T[a] * c + s_T[b]] = acc;
                X[(int64_t)s_T[b] * c + s_T[a]] = acc;
                if (a == b) (mat ? md : gd)[s_T[a]] = acc;
            }
        }
        // rows and mirrored columns of the tuple, every other active column
        for (int y = tid; y < c; y += KS_THREADS) {
            bool inT = false;
#pragma unroll
            for (int a = 0; a < KM; ++a) inT |= a < kk && T[a] == y;
            if (inT || !active_bit(mask, y)) continue;
            double gi[KM], mi[KM], go[KM], mo[KM];
#pragma unroll
            for (int a = 0; a < KM; ++a) {
                gi[a] = a < kk ? G[(int64_t)T[a] * c + y] : 0.0;
                mi[a] = a < kk ? M[(int64_t)T[a] * c + y] : 0.0;
            }
#pragma unroll
            for (int a = 0; a < KM; ++a) {
                go[a] = a < kk ? rot_row_u<KM>(s_O, kk, a, gi) : 0.0;
                mo[a] = a < kk ? rot_row_u<KM>(s_O, kk, a, mi) : 0.0;
            }
#pragma unroll
            for (int a = 0; a < KM; ++a)
                if (a < kk) {
                    G[(int64_t)T[a] * c + y] = go[a];
                    G[(int64_t)y * c + T[a]] = go[a];
                    M[(int64_t)T[a] * c + y] = mo[a];
                    M[(int64_t)y * c + T[a]] = mo[a];
                }
        }
        __syncthreads();
        if (tid < kk) {
            const int x = s_T[tid];
            const double g = gd[x];
            w[x] = g > 0.0 ? __ddiv_rn(1.0, __dsqrt_rn(g)) : 0.0;
        }
        if (tid == 0) {
            int bi = 0;
            double dbest = __dsub_rn(gd[s_T[0]], __dmul_rn(md[s_T[0]], md[s_T[0]]));
            for (int a = 1; a < kk; ++a) {
                const int x = s_T[a];
                const double d = __dsub_rn(gd[x], __dmul_rn(md[x], md[x]));
                if (d <= dbest) {
                    dbest = d;
                    bi = a;
                }
            }
            const int le = s_T[bi];
            int L = 0;
            for (int a = 0; a < kk; ++a) L = max(L, lvl[s_T[a]]);
            ++L;
            for (int a = 0; a < kk; ++a) lvl[s_T[a]] = L;
            s_maxlev = max(s_maxlev, L);
            mask[le >> 5] &= ~(1u << (le & 31));
            const int64_t rr = r0 + t;
            for (int a = 0; a < K; ++a) kidx[rr * K + a] = a < kk ? s_T[a] : -1;
            for (int a = 0; a < K * K; ++a) kO[rr * K * K + a] = a < kk * kk ? s_O[a] : 0.0;
            kkv[rr] = kk;
            kel[rr] = le;
            klvl[rr] = L;
        }
        __syncthreads();
    }
    // group by dependency level; flag the eliminated coordinates
    const int nl = s_maxlev;
    for (int t = tid; t < e; t += KS_THREADS) {
        atomicAdd(&lcnt[klvl[r0 + t]], 1);
        elimflag[members[base + kel[r0 + t]]] = (int32_t)stage;
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
    for (int t = tid; t < e; t += KS_THREADS) {
        const int slot = atomicAdd(&lcnt[klvl[r0 + t]], 1);
        lvlidx[r0 + slot] = (int32_t)(r0 + t);
    }
}

}  // namespace

pmmf_status select_kpoint(const StageClusters &cls, int64_t cmax, const int64_t *goff, double *G,
                          double *M, uint64_t seed, int64_t stage, StageRotations &rot,
                          int32_t *elimflag, cudaStream_t st, const int32_t *order,
                          const uint64_t *useed, unsigned *status, const int32_t *ords) {
    const int64_t m = cls.m, nr = rot.nrot > 0 ? rot.nrot : 1;
    const int K = rot.K;
    PMMF_TRY(rot.kidx.alloc(nr * K, st));
    PMMF_TRY(rot.kO.alloc(nr * K * K, st));
    PMMF_TRY(rot.kk.alloc(nr, st));
    PMMF_TRY(rot.kel.alloc(nr, st));
    PMMF_TRY(rot.klvl.alloc(nr, st));
    PMMF_TRY(rot.lvlidx.alloc(nr, st));
    PMMF_TRY(rot.lvl_off.alloc(rot.nrot + m + 1, st));
    PMMF_TRY(rot.nlev.zeros(m, st));
    const size_t sh = sizeof(double) * 3 * (size_t)cmax + sizeof(uint64_t) * (size_t)cmax +
                      sizeof(uint32_t) * (size_t)((cmax + 31) / 32) +
                      sizeof(int32_t) * (size_t)(2 * cmax + 4);
    if (sh > 220 * 1024) {
        set_error("cluster too large for the k-point rotation search");
        return PMMF_ERR_UNSUPPORTED;
    }
    auto kern = K == 3 ? k_select_k<3> : k_select_k<8>;
    PMMF_CUDA_TRY(allow_smem(kern, sh));
    prof_begin(KF_SELECT, st);
    kern<<<(unsigned)m, KS_THREADS, sh, st>>>(cls.coff.p, cls.members.p, goff, G, M,
                                                   rot.roff.p, seed, stage, K, rot.kidx.p, rot.kk.p,
                                                   rot.kel.p, rot.klvl.p, rot.kO.p, rot.lvlidx.p,
                                                   rot.lvl_off.p, rot.nlev.p, elimflag, order,
                                                   useed, status, ords);
    prof_end(KF_SELECT, st, 0.0, 0.0);
    return launched("select_k");
}

}  // namespace pmmf
