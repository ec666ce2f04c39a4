// backward.cu -- gradient of the factorized operator y = U^T M U x
// (M = H or H^{-1}; Sec. 2.4's matrix-free product) with the greedy
// selections held fixed, and the parameter get/set kernels it needs.
//
// For L = sum(g * y):
//   z = U x, w = U g                      forward through the stages, the
//                                         stage-start slices of [x | g] kept
//                                         (stage-level checkpoints)
//   dL/dM = w z^T on H's structure        (M = H^{-1}: dL/dH = -(M w)(M z)^T,
//                                         the core's part folded onto the lower
//                                         triangle the inverse is formed from)
//   u = M z, h = M w                      (M treated as symmetric)
//   backward through the stages, last first: per cluster, the stage's
//   rotations are replayed forward from the checkpoint to recover every
//   rotation's output (v_t, q_t), then undone in reverse on [p | r]
//   (p_T = u, r_T = h).  For the rotation t on (i, j) with angle theta_t
//   ((c, s) = (cos, sin)), the U occurrence contributes r_j v_i - r_i v_j and
//   the U^T occurrence q_i p_j - q_j p_i (a 2-D cross product, invariant under
//   the rotation itself, so both are taken at the same point), summed over the
//   right-hand sides.  What remains in r after the last stage is dL/dx.
// k-point rotations are parameterised by their block O (x_T' = O x_T): the U
// occurrence adds r_a v_b and the U^T occurrence p_a q_b to dL/dO_ab, with
// r, p at the rotation's output and v, q at its input, over the right-hand
// sides.
#include <cmath>

#include "apply.cuh"
#include "backward.cuh"
#include "rotmath.cuh"

namespace pmmf {
namespace {

constexpr int BW_THREADS = 256;

// out[l * w + r] = v[members[l] * w + r]: the stage's coordinates in cluster order.
__global__ void k_gather_members(const int32_t *members, int64_t s, const double *v, int w,
                                 double *out) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < s * w;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t l = q / w, r = q - l * w;
        out[q] = v[(int64_t)members[l] * w + r];
    }
}

// [x | g] columns c0 .. c0+nr of the caller's blocks -> one n x 2nr block.
__global__ void k_pack2(const double *x, const double *g, int64_t ld, int64_t n, int nr,
                        int64_t c0, double *out) {
    const int w = 2 * nr;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n * w;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = q / w;
        const int r = (int)(q - i * w);
        out[q] = r < nr ? x[i * ld + c0 + r] : g[i * ld + c0 + r - nr];
    }
}

// Columns nr .. 2nr of a packed block -> the caller's columns c0 .. c0+nr.
__global__ void k_unpack_hi(const double *in, int64_t n, int nr, double *y, int64_t ld,
                            int64_t c0) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n * nr;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = q / nr;
        const int r = (int)(q - i * nr);
        y[i * ld + c0 + r] = in[i * 2 * nr + nr + r];
    }
}

// Wavelet diagonal of dL/dH: sign * sum_r a_ir b_ir with a = columns nr.., b =
// columns ..nr of a packed block; 0 on core coordinates.
__global__ void k_dh_diag(const double *blk, int64_t n, int nr, const int32_t *core_pos,
                          double sign, int accumulate, double *dh) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double acc = accumulate ? dh[i] : 0.0;
        if (core_pos[i] < 0) {
            const double *row = blk + i * 2 * nr;
            for (int r = 0; r < nr; ++r) acc = __fma_rn(sign * row[nr + r], row[r], acc);
        }
        dh[i] = acc;
    }
}

// Core block of dL/dH: G[a][b] = sign * sum_r A[core_idx[a]][r] B[core_idx[b]][r]
// with A = columns nr.., B = columns ..nr.  fold (the inverse, which reads
// only the core's lower triangle): G[a][b] + G[b][a] below the diagonal, 0
// above it.
__global__ void k_dcore(const double *blk, int64_t m, int nr, const int32_t *core_idx,
                        double sign, int fold, int accumulate, double *dcore) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < m * m;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = q / m, b = q - a * m;
        double acc = accumulate ? dcore[q] : 0.0;
        if (!fold || a >= b) {
            const double *ra = blk + (int64_t)core_idx[a] * 2 * nr + nr;
            const double *rb = blk + (int64_t)core_idx[b] * 2 * nr;
            for (int r = 0; r < nr; ++r) acc = __fma_rn(sign * ra[r], rb[r], acc);
        }
        if (fold && a > b) {
            const double *ra = blk + (int64_t)core_idx[b] * 2 * nr + nr;
            const double *rb = blk + (int64_t)core_idx[a] * 2 * nr;
            for (int r = 0; r < nr; ++r) acc = __fma_rn(sign * ra[r], rb[r], acc);
        }
        dcore[q] = acc;
    }
}

// One stage of the backward sweep, one CTA per cluster.  ck holds the
// stage-start slice [v | q] (cluster order, 2nr per coordinate); pr is the
// global [p | r] block, updated in place from the stage's end state to its
// start state.  dtheta gets the stage's angle gradients in (cluster, step)
// order.  Shared memory: V, Q, P, R (c x nr each), every rotation's outputs
// (e x nr x 4), per-(rotation, column) terms (e x nr) and the rotation records.
__global__ void __launch_bounds__(BW_THREADS)
k_backward_stage(const int64_t *coff, const int32_t *members, const int64_t *roff,
                 const RotRec *rec, const int32_t *nlev, const double *ck, double *pr, int nr,
                 int accumulate, double *dtheta) {
    extern __shared__ double sm[];
    const int64_t u = blockIdx.x;
    const int64_t base = coff[u];
    const int c = (int)(coff[u + 1] - base);
    const int64_t r0 = roff[u];
    const int e = (int)(roff[u + 1] - r0);
    if (e == 0) return;
    const int nl = nlev[u];
    const int w2 = 2 * nr;
    const int tid = threadIdx.x;
    double *V = sm;
    double *Q = V + (int64_t)c * nr;
    double *P = Q + (int64_t)c * nr;
    double *R = P + (int64_t)c * nr;
    double *SV = R + (int64_t)c * nr;
    double *part = SV + (int64_t)e * nr * 4;
    RotRec *rr = (RotRec *)(part + (int64_t)e * nr);
    for (int64_t q = tid; q < (int64_t)c * nr; q += BW_THREADS) {
        const int64_t l = q / nr, r = q - l * nr;
        const double *cq = ck + (base + l) * w2;
        const double *pq = pr + (int64_t)members[base + l] * w2;
        V[q] = cq[r];
        Q[q] = cq[nr + r];
        P[q] = pq[r];
        R[q] = pq[nr + r];
    }
    for (int t = tid; t < e; t += BW_THREADS) rr[t] = rec[r0 + t];
    __syncthreads();
    const int en = e * nr;
    // replay: every rotation's outputs of v and q, level by level
    for (int L = 1; L <= nl; ++L) {
        for (int q = tid; q < en; q += BW_THREADS) {
            const int t = q / nr, r = q - t * nr;
            const RotRec x = rr[t];
            if (x.lvl != L) continue;
            double a, b;
            rot_pair(x.c, x.s, V[x.li * nr + r], V[x.lj * nr + r], a, b);
            V[x.li * nr + r] = a;
            V[x.lj * nr + r] = b;
            double *sv = SV + (int64_t)q * 4;
            sv[0] = a;
            sv[1] = b;
            rot_pair(x.c, x.s, Q[x.li * nr + r], Q[x.lj * nr + r], a, b);
            Q[x.li * nr + r] = a;
            Q[x.lj * nr + r] = b;
            sv[2] = a;
            sv[3] = b;
        }
        __syncthreads();
    }
    // undo in reverse level order, taking each rotation's terms first
    for (int L = nl; L >= 1; --L) {
        for (int q = tid; q < en; q += BW_THREADS) {
            const int t = q / nr, r = q - t * nr;
            const RotRec x = rr[t];
            if (x.lvl != L) continue;
            const double pi = P[x.li * nr + r], pj = P[x.lj * nr + r];
            const double ri = R[x.li * nr + r], rj = R[x.lj * nr + r];
            const double *sv = SV + (int64_t)q * 4;
            double d = __dmul_rn(rj, sv[0]);
            d = __fma_rn(-ri, sv[1], d);
            d = __fma_rn(sv[2], pj, d);
            d = __fma_rn(-sv[3], pi, d);
            part[q] = d;
            double a, b;
            rot_pair_t(x.c, x.s, pi, pj, a, b);
            P[x.li * nr + r] = a;
            P[x.lj * nr + r] = b;
            rot_pair_t(x.c, x.s, ri, rj, a, b);
            R[x.li * nr + r] = a;
            R[x.lj * nr + r] = b;
        }
        __syncthreads();
    }
    for (int t = tid; t < e; t += BW_THREADS) {
        double acc = accumulate ? dtheta[r0 + t] : 0.0;
        for (int r = 0; r < nr; ++r) acc = __dadd_rn(acc, part[t * nr + r]);
        dtheta[r0 + t] = acc;
    }
    for (int64_t q = tid; q < (int64_t)c * nr; q += BW_THREADS) {
        const int64_t l = q / nr, r = q - l * nr;
        double *pq = pr + (int64_t)members[base + l] * w2;
        pq[r] = P[q];
        pq[nr + r] = R[q];
    }
}

size_t backward_smem(int64_t c, int64_t e, int nr) {
    return sizeof(double) * (size_t)(4 * c * nr + 5 * e * nr) + sizeof(RotRec) * (size_t)e;
}

// One stage of the backward sweep for k-point rotations (one CTA per
// cluster).  The replay keeps each rotation's inputs of v and q (SIN: per
// rotation and right-hand side, K entries of each); the undo runs one thread
// per rotation of a level, which forms the rotation's dL/dO block over all
// right-hand sides and then applies O^T to its coordinates of p and r.  dO
// gets K*K slots per rotation (stride kk inside, unused slots 0) in step
// order.
__global__ void __launch_bounds__(BW_THREADS)
k_backward_stage_k(const int64_t *coff, const int32_t *members, const int64_t *roff, int K,
                   const int32_t *kidx, const int32_t *kkv, const int32_t *klvl, const double *kO,
                   const int32_t *nlev, const double *ck, double *pr, int nr, int accumulate,
                   double *dO) {
    extern __shared__ double sm[];
    const int64_t u = blockIdx.x;
    const int64_t base = coff[u];
    const int c = (int)(coff[u + 1] - base);
    const int64_t r0 = roff[u];
    const int e = (int)(roff[u + 1] - r0);
    if (e == 0) return;
    const int nl = nlev[u];
    const int w2 = 2 * nr;
    const int tid = threadIdx.x;
    double *V = sm;
    double *Q = V + (int64_t)c * nr;
    double *P = Q + (int64_t)c * nr;
    double *R = P + (int64_t)c * nr;
    double *SIN = R + (int64_t)c * nr;
    for (int64_t q = tid; q < (int64_t)c * nr; q += BW_THREADS) {
        const int64_t l = q / nr, r = q - l * nr;
        const double *cq = ck + (base + l) * w2;
        const double *pq = pr + (int64_t)members[base + l] * w2;
        V[q] = cq[r];
        Q[q] = cq[nr + r];
        P[q] = pq[r];
        R[q] = pq[nr + r];
    }
    __syncthreads();
    const int en = e * nr;
    for (int L = 1; L <= nl; ++L) {
        for (int q = tid; q < en; q += BW_THREADS) {
            const int t = q / nr, r = q - t * nr;
            const int64_t tt = r0 + t;
            if (klvl[tt] != L) continue;
            const int kk = kkv[tt];
            const int32_t *T = kidx + tt * K;
            const double *O = kO + tt * K * K;
            double *sin = SIN + (int64_t)q * 2 * K;
            double vin[8], qin[8];
            for (int a = 0; a < kk; ++a) {
                vin[a] = V[T[a] * nr + r];
                qin[a] = Q[T[a] * nr + r];
                sin[a] = vin[a];
                sin[K + a] = qin[a];
            }
            for (int a = 0; a < kk; ++a) {
                V[T[a] * nr + r] = rot_row(O, kk, a, vin);
                Q[T[a] * nr + r] = rot_row(O, kk, a, qin);
            }
        }
        __syncthreads();
    }
    for (int L = nl; L >= 1; --L) {
        for (int t = tid; t < e; t += BW_THREADS) {
            const int64_t tt = r0 + t;
            if (klvl[tt] != L) continue;
            const int kk = kkv[tt];
            const int32_t *T = kidx + tt * K;
            const double *O = kO + tt * K * K;
            double *d = dO + tt * K * K;
            for (int a = 0; a < kk; ++a)
                for (int b = 0; b < kk; ++b) {
                    double acc = accumulate ? d[a * kk + b] : 0.0;
                    for (int r = 0; r < nr; ++r) {
                        const double *sin = SIN + ((int64_t)t * nr + r) * 2 * K;
                        acc = __fma_rn(R[T[a] * nr + r], sin[b], acc);
                        acc = __fma_rn(P[T[a] * nr + r], sin[K + b], acc);
                    }
                    d[a * kk + b] = acc;
                }
            if (!accumulate)
                for (int z = kk * kk; z < K * K; ++z) d[z] = 0.0;
            for (int r = 0; r < nr; ++r) {
                double pin[8], rin[8];
                for (int a = 0; a < kk; ++a) {
                    pin[a] = P[T[a] * nr + r];
                    rin[a] = R[T[a] * nr + r];
                }
                for (int a = 0; a < kk; ++a) {
                    P[T[a] * nr + r] = rot_row_t(O, kk, a, pin);
                    R[T[a] * nr + r] = rot_row_t(O, kk, a, rin);
                }
            }
        }
        __syncthreads();
    }
    for (int64_t q = tid; q < (int64_t)c * nr; q += BW_THREADS) {
        const int64_t l = q / nr, r = q - l * nr;
        double *pq = pr + (int64_t)members[base + l] * w2;
        pq[r] = P[q];
        pq[nr + r] = R[q];
    }
}

size_t backward_smem_k(int64_t c, int64_t e, int K, int nr) {
    return sizeof(double) * (size_t)(4 * c * nr + 2 * e * nr * K);
}

__global__ void k_get_angles(const RotRec *rec, int64_t nrot, double *theta) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nrot;
         t += (int64_t)gridDim.x * blockDim.x)
        theta[t] = atan2(rec[t].s, rec[t].c);
}

__global__ void k_set_angles(RotRec *rec, int64_t nrot, const double *theta) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nrot;
         t += (int64_t)gridDim.x * blockDim.x) {
        double s, c;
        sincos(theta[t], &s, &c);
        rec[t].c = c;
        rec[t].s = s;
    }
}

// ---- angle parameterisation of k-point blocks --------------------------------
// Givens elimination of the kk x kk block column by column (j = 0..kk-2,
// l = j+1..kk-1): theta_i = atan2(A_lj, A_jj), rows (j, l) <- G (c row j + s
// row l, -s row j + c row l), leaving D = diag(+-1); O = G_1^T .. G_P^T D.
// One thread per rotation; P = K (K - 1) / 2 angle slots and K sign slots per
// rotation (unused slots 0).
__device__ __forceinline__ void bl_rows(double *A, int kk, int j, int l, double c, double s) {
    for (int b = 0; b < kk; ++b) {
        const double aj = A[j * kk + b], al = A[l * kk + b];
        A[j * kk + b] = __dadd_rn(__dmul_rn(c, aj), __dmul_rn(s, al));
        A[l * kk + b] = __dadd_rn(__dmul_rn(-s, aj), __dmul_rn(c, al));
    }
}
__device__ __forceinline__ void bl_rows_t(double *A, int kk, int j, int l, double c, double s) {
    for (int b = 0; b < kk; ++b) {
        const double aj = A[j * kk + b], al = A[l * kk + b];
        A[j * kk + b] = __dsub_rn(__dmul_rn(c, aj), __dmul_rn(s, al));
        A[l * kk + b] = __dadd_rn(__dmul_rn(s, aj), __dmul_rn(c, al));
    }
}

__global__ void k_block_angles(int64_t nrot, int K, const int32_t *kkv, const double *kO,
                               double *theta, double *D) {
    const int P = K * (K - 1) / 2;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nrot;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int kk = kkv[t];
        double A[64];
        for (int q = 0; q < kk * kk; ++q) A[q] = kO[t * K * K + q];
        double *th = theta + t * P;
        int i = 0;
        for (int j = 0; j + 1 < kk; ++j)
            for (int l = j + 1; l < kk; ++l) {
                const double a = atan2(A[l * kk + j], A[j * kk + j]);
                double s, c;
                sincos(a, &s, &c);
                th[i++] = a;
                bl_rows(A, kk, j, l, c, s);
            }
        for (; i < P; ++i) th[i] = 0.0;
        if (D)
            for (int a = 0; a < K; ++a)
                D[t * K + a] = a < kk ? ((f64_bits(A[a * kk + a]) >> 63) && (f64_bits(A[a * kk + a]) << 1) ? -1.0 : 1.0) : 0.0;
    }
}

__global__ void k_block_from_angles(int64_t nrot, int K, const int32_t *kkv, const double *theta,
                                    const double *D, double *kO) {
    const int P = K * (K - 1) / 2;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nrot;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int kk = kkv[t];
        double O[64];
        for (int a = 0; a < kk; ++a)
            for (int b = 0; b < kk; ++b) O[a * kk + b] = a == b ? D[t * K + a] : 0.0;
        const double *th = theta + t * P;
        int i = kk * (kk - 1) / 2;
        for (int j = kk - 2; j >= 0; --j)
            for (int l = kk - 1; l > j; --l) {
                --i;
                double s, c;
                sincos(th[i], &s, &c);
                bl_rows_t(O, kk, j, l, c, s);
            }
        for (int q = 0; q < K * K; ++q) kO[t * K * K + q] = q < kk * kk ? O[q] : 0.0;
    }
}

// dL/dtheta_i = < Lam_i, dG_i^T/dtheta B_i > with Lam_i = G_{i-1} .. G_1 dO and
// B_i = G_{i+1}^T .. G_P^T D; dG^T/dtheta on rows (j, l) = [[-s, -c], [c, -s]].
// Lam is carried to the last rotation and walked back with G_i^T (G is
// orthogonal) while B grows from D, so each thread holds two kk x kk blocks.
__global__ void k_block_angle_grad(int64_t nrot, int K, const int32_t *kkv, const double *theta,
                                   const double *D, const double *dO, double *dtheta) {
    const int P = K * (K - 1) / 2;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nrot;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int kk = kkv[t];
        const int pk = kk * (kk - 1) / 2;
        const double *th = theta + t * P;
        double Lam[64], B[64];
        for (int q = 0; q < kk * kk; ++q) Lam[q] = dO[t * K * K + q];
        {
            int i = 0;
            for (int j = 0; j + 1 < kk; ++j)
                for (int l = j + 1; l < kk; ++l) {
                    double s, c;
                    sincos(th[i++], &s, &c);
                    bl_rows(Lam, kk, j, l, c, s);
                }
        }
        for (int a = 0; a < kk; ++a)
            for (int b = 0; b < kk; ++b) B[a * kk + b] = a == b ? D[t * K + a] : 0.0;
        double *out = dtheta + t * P;
        int i = pk;
        for (int j = kk - 2; j >= 0; --j)
            for (int l = kk - 1; l > j; --l) {
                --i;
                double s, c;
                sincos(th[i], &s, &c);
                bl_rows_t(Lam, kk, j, l, c, s);        // Lam_i = G_i^T Lam_{i+1}
                double acc = 0.0;
                for (int b = 0; b < kk; ++b) {
                    const double bj = B[j * kk + b], bl = B[l * kk + b];
                    acc = __dadd_rn(acc, __dmul_rn(Lam[j * kk + b], __dsub_rn(__dmul_rn(-s, bj), __dmul_rn(c, bl))));
                    acc = __dadd_rn(acc, __dmul_rn(Lam[l * kk + b], __dsub_rn(__dmul_rn(c, bj), __dmul_rn(s, bl))));
                }
                out[i] = acc;
                bl_rows_t(B, kk, j, l, c, s);          // B_{i-1} = G_i^T B_i
            }
        for (int q = pk; q < P; ++q) out[q] = 0.0;
    }
}

// Rebuild the level-grouped copies from the step-order records (one CTA per
// cluster; the level offsets are unchanged).  Thread 0 walks the cluster's
// rotations in step order, so the order inside a level is deterministic.
__global__ void k_regroup_levels(const int64_t *roff, const RotRec *rec, const int32_t *lvl_off,
                                 const int32_t *nlev, Rot2 *lvlrot, int32_t *cnt_scratch) {
    const int64_t u = blockIdx.x;
    if (threadIdx.x != 0) return;
    const int64_t r0 = roff[u];
    const int e = (int)(roff[u + 1] - r0);
    const int nl = nlev[u];
    const int32_t *lo = lvl_off + r0 + u;
    int32_t *cnt = cnt_scratch + r0 + u;  // nl + 1 <= e + 1 slots
    for (int L = 0; L <= nl; ++L) cnt[L] = 0;
    for (int t = 0; t < e; ++t) {
        const RotRec x = rec[r0 + t];
        const int L = x.lvl - 1;
        lvlrot[lo[L] + cnt[L]++] = Rot2{x.li, x.lj, x.c, x.s};
    }
}

}  // namespace

pmmf_status apply_backward(const ApplyStages &S, const std::vector<const RotRec *> &recs,
                           const std::vector<const int32_t *> &klvls, const HData &H,
                           bool inverse, const double *x, const double *g, int64_t nrhs,
                           int64_t ld, double *dx, double *dtheta, double *dhdiag, double *dcore,
                           cudaStream_t st) {
    const int64_t n = H.n;
    const int nst = (int)S.size();
    int64_t totrot = 0;
    std::vector<int64_t> toff((size_t)nst + 1, 0);
    int nr = 8;
    const int K = nst > 0 ? S[0].K : 2;
    auto smem = [&](int64_t c, int w) {
        return K > 2 ? backward_smem_k(c, c, K, w) : backward_smem(c, c, w);
    };
    for (int p = 0; p < nst; ++p) {
        toff[p + 1] = toff[p] + S[p].nrot;
        // a cluster never rotates more coordinates than it holds
        while (nr > 1 && smem(S[p].cmax, nr) > 220 * 1024) --nr;
        if (smem(S[p].cmax, nr) > 220 * 1024) {
            set_error("backward: cluster too large for shared memory");
            return PMMF_ERR_UNSUPPORTED;
        }
    }
    totrot = toff[nst];
    const int64_t per_rot = K > 2 ? (int64_t)K * K : 1;   // dtheta slots per rotation
    nr = (int)std::min<int64_t>(nr, nrhs);
    const int w2 = 2 * nr;
    // checkpoint offsets: stage p's slice holds its active coordinates x 2nr
    std::vector<int64_t> coff_ck((size_t)nst + 1, 0);
    for (int p = 0; p < nst; ++p) coff_ck[p + 1] = coff_ck[p] + S[p].s * w2;
    DBuf<double> vq, prb, ck, dth;
    PMMF_TRY(vq.alloc(n * w2, st));
    PMMF_TRY(prb.alloc(n * w2, st));
    PMMF_TRY(ck.alloc(std::max<int64_t>(coff_ck[nst], 1), st));
    double *dt = dtheta;
    if (!dt && totrot > 0) {
        PMMF_TRY(dth.alloc(totrot * per_rot, st));
        dt = dth.p;
    }

    for (int64_t c0 = 0; c0 < nrhs; c0 += nr) {
        const int cur = (int)std::min<int64_t>(nr, nrhs - c0);
        const int cw = 2 * cur;
        const int acc = c0 > 0 ? 1 : 0;
        k_pack2<<<grid_for(n * cw, 256), 256, 0, st>>>(x, g, ld, n, cur, c0, vq.p);
        PMMF_TRY(launched("bw_pack"));
        for (int p = 0; p < nst; ++p) {
            if (S[p].nrot == 0) continue;
            k_gather_members<<<grid_for(S[p].s * cw, 256), 256, 0, st>>>(
                S[p].members, S[p].s, vq.p, cw, ck.p + coff_ck[p]);
            PMMF_TRY(launched("bw_gather"));
            ApplyStages one(1, S[p]);
            PMMF_TRY(apply_rotations(one, false, vq.p, cw, cw, st));
        }
        // vq = [z | w]
        if (!inverse) {
            if (dhdiag) {
                k_dh_diag<<<grid_for(n, 256), 256, 0, st>>>(vq.p, n, cur, H.core_pos, 1.0, acc, dhdiag);
                PMMF_TRY(launched("bw_dh_diag"));
            }
            if (dcore && H.m > 0) {
                k_dcore<<<grid_for(H.m * H.m, 256), 256, 0, st>>>(vq.p, H.m, cur, H.core_idx, 1.0, 0, acc, dcore);
                PMMF_TRY(launched("bw_dcore"));
            }
        }
        PMMF_TRY(copy_block(vq.p, cw, prb.p, cw, n, cw, st));
        PMMF_TRY(apply_h(H, inverse, prb.p, cw, cw, st));
        // prb = [u | h] = M [z | w]
        if (inverse) {
            if (dhdiag) {
                k_dh_diag<<<grid_for(n, 256), 256, 0, st>>>(prb.p, n, cur, H.core_pos, -1.0, acc, dhdiag);
                PMMF_TRY(launched("bw_dh_diag"));
            }
            if (dcore && H.m > 0) {
                k_dcore<<<grid_for(H.m * H.m, 256), 256, 0, st>>>(prb.p, H.m, cur, H.core_idx, -1.0, 1, acc, dcore);
                PMMF_TRY(launched("bw_dcore"));
            }
        }
        for (int p = nst - 1; p >= 0; --p) {
            const ApplyStage &a = S[p];
            if (a.nrot == 0) continue;
            if (K > 2) {
                const size_t shk = backward_smem_k(a.cmax, a.cmax, K, cur);
                PMMF_CUDA_TRY(allow_smem(k_backward_stage_k, shk));
                k_backward_stage_k<<<(unsigned)a.m, BW_THREADS, shk, st>>>(
                    a.coff, a.members, a.roff, K, a.kidx, a.kkv, klvls[p], a.kO, a.nlev,
                    ck.p + coff_ck[p], prb.p, cur, acc, dt + toff[p] * per_rot);
                PMMF_TRY(launched("bw_stage_k"));
                continue;
            }
            const size_t sh = backward_smem(a.cmax, a.cmax, cur);
            PMMF_CUDA_TRY(allow_smem(k_backward_stage, sh));
            k_backward_stage<<<(unsigned)a.m, BW_THREADS, sh, st>>>(
                a.coff, a.members, a.roff, recs[p], a.nlev, ck.p + coff_ck[p], prb.p, cur, acc,
                dt + toff[p]);
            PMMF_TRY(launched("bw_stage"));
        }
        if (dx) {
            k_unpack_hi<<<grid_for(n * cur, 256), 256, 0, st>>>(prb.p, n, cur, dx, ld, c0);
            PMMF_TRY(launched("bw_unpack"));
        }
    }
    return PMMF_OK;
}

pmmf_status block_angles(int64_t nrot, int K, const int32_t *kkv, const double *kO,
                         double *theta, double *D, cudaStream_t st) {
    if (nrot == 0) return PMMF_OK;
    k_block_angles<<<grid_for(nrot, 128), 128, 0, st>>>(nrot, K, kkv, kO, theta, D);
    return launched("block_angles");
}

pmmf_status block_from_angles(int64_t nrot, int K, const int32_t *kkv, const double *theta,
                              const double *D, double *kO, cudaStream_t st) {
    if (nrot == 0) return PMMF_OK;
    k_block_from_angles<<<grid_for(nrot, 128), 128, 0, st>>>(nrot, K, kkv, theta, D, kO);
    return launched("block_from_angles");
}

pmmf_status block_angle_grad(int64_t nrot, int K, const int32_t *kkv, const double *theta,
                             const double *D, const double *dO, double *dtheta, cudaStream_t st) {
    if (nrot == 0) return PMMF_OK;
    k_block_angle_grad<<<grid_for(nrot, 64), 64, 0, st>>>(nrot, K, kkv, theta, D, dO, dtheta);
    return launched("block_angle_grad");
}

pmmf_status get_angles(const RotRec *rec, int64_t nrot, double *theta, cudaStream_t st) {
    if (nrot == 0) return PMMF_OK;
    k_get_angles<<<grid_for(nrot, 256), 256, 0, st>>>(rec, nrot, theta);
    return launched("get_angles");
}

pmmf_status set_angles(const ApplyStage &a, RotRec *rec, Rot2 *lvlrot, const double *theta,
                       cudaStream_t st) {
    if (a.nrot == 0) return PMMF_OK;
    k_set_angles<<<grid_for(a.nrot, 256), 256, 0, st>>>(rec, a.nrot, theta);
    PMMF_TRY(launched("set_angles"));
    DBuf<int32_t> cnt;
    PMMF_TRY(cnt.alloc(a.nrot + a.m + 1, st));
    k_regroup_levels<<<(unsigned)a.m, 32, 0, st>>>(a.roff, rec, a.lvl_off, a.nlev, lvlrot, cnt.p);
    return launched("regroup_levels");
}

}  // namespace pmmf
