// rotmath.cuh -- the rotation arithmetic shared by the rotation searches
// (internal).  Every function fixes its operation order: the searches must
// produce the same bits as a sequential FP64 evaluation of the same readings.
#pragma once

#include "common.cuh"

namespace pmmf {

// Smaller-angle Jacobi rotation zeroing the off-diagonal of q [[a,b],[b,d]] q^T:
// h = d - a, g = 2b (scaled by an exact power of two when huge or tiny),
// q = |h| + sqrt(h^2 + g^2), den = sqrt(q^2 + g^2), c = q/den, s = sign(h) g/den.
// Comparisons, |.| and the sign test act on the bits (integer pipe): for finite
// doubles the magnitude bits order like the magnitudes.
__device__ __forceinline__ void jacobi2(double a, double b, double d, double &c, double &s) {
    const unsigned long long ABS = 0x7fffffffffffffffull;
    if ((f64_bits(b) & ABS) == 0) {
        c = 1.0;
        s = 0.0;
        return;
    }
    double h = __dsub_rn(d, a);
    double g = __dmul_rn(2.0, b);
    const unsigned long long hm = f64_bits(h) & ABS, gm = f64_bits(g) & ABS;
    const unsigned long long mm = hm > gm ? hm : gm;
    if (mm > (unsigned long long)__double_as_longlong(0x1p500)) {
        h = __dmul_rn(h, 0x1p-600);
        g = __dmul_rn(g, 0x1p-600);
    } else if (mm < (unsigned long long)__double_as_longlong(0x1p-500)) {
        h = __dmul_rn(h, 0x1p600);
        g = __dmul_rn(g, 0x1p600);
    }
    const unsigned long long hb = f64_bits(h);
    const double habs = f64_from_bits(hb & ABS);
    const bool hnonneg = (hb >> 63) == 0 || (hb & ABS) == 0;   // h >= 0, -0 included
    const double g2 = __dmul_rn(g, g);
    const double r = __dsqrt_rn(__dadd_rn(__dmul_rn(h, h), g2));
    const double q = __dadd_rn(habs, r);
    const double den = __dsqrt_rn(__dadd_rn(__dmul_rn(q, q), g2));
    c = __ddiv_rn(q, den);
    s = __ddiv_rn(hnonneg ? g : f64_from_bits(f64_bits(g) ^ ~ABS), den);
}

// jacobi2's c (want_s false) or s (want_s true): the same operations as
// jacobi2 for that value.  Lanes of one warp that call it with different
// want_s share the prefix's instructions and take both divides as one.
__device__ __forceinline__ double jacobi2_one(double a, double b, double d, bool want_s) {
    const unsigned long long ABS = 0x7fffffffffffffffull;
    if ((f64_bits(b) & ABS) == 0) return want_s ? 0.0 : 1.0;
    double h = __dsub_rn(d, a);
    double g = __dmul_rn(2.0, b);
    const unsigned long long hm = f64_bits(h) & ABS, gm = f64_bits(g) & ABS;
    const unsigned long long mm = hm > gm ? hm : gm;
    if (mm > (unsigned long long)__double_as_longlong(0x1p500)) {
        h = __dmul_rn(h, 0x1p-600);
        g = __dmul_rn(g, 0x1p-600);
    } else if (mm < (unsigned long long)__double_as_longlong(0x1p-500)) {
        h = __dmul_rn(h, 0x1p600);
        g = __dmul_rn(g, 0x1p600);
    }
    const unsigned long long hb = f64_bits(h);
    const double habs = f64_from_bits(hb & ABS);
    const bool hnonneg = (hb >> 63) == 0 || (hb & ABS) == 0;
    const double g2 = __dmul_rn(g, g);
    const double r = __dsqrt_rn(__dadd_rn(__dmul_rn(h, h), g2));
    const double q = __dadd_rn(habs, r);
    const double den = __dsqrt_rn(__dadd_rn(__dmul_rn(q, q), g2));
    const double num = want_s ? (hnonneg ? g : f64_from_bits(f64_bits(g) ^ ~ABS)) : q;
    return __ddiv_rn(num, den);
}

// Row a of x_T' = O x_T for a k x k block O (row-major, stride kk): an fma
// chain over b from kk-1 down to 0.  For kk = 2 and O = [[c, -s], [s, c]]
// this is rot_pair.
__device__ __forceinline__ double rot_row(const double *O, int kk, int a, const double *in) {
    double acc = __dmul_rn(O[a * kk + kk - 1], in[kk - 1]);
    for (int b = kk - 2; b >= 0; --b) acc = __fma_rn(O[a * kk + b], in[b], acc);
    return acc;
}

// Row a of O x for a tuple of kk <= KM entries held in registers: rot_row's
// chain (the last column's product, then fmas down to column 0) unrolled over
// KM, so in[] is never indexed at run time.
template <int KM>
__device__ __forceinline__ double rot_row_u(const double *O, int kk, int a, const double (&in)[KM]) {
    double acc = 0.0;
#pragma unroll
    for (int b = KM - 1; b >= 0; --b) {
        if (b == kk - 1) acc = __dmul_rn(O[a * kk + b], in[b]);
        else if (b < kk - 1) acc = __fma_rn(O[a * kk + b], in[b], acc);
    }
    return acc;
}

// Row a of x_T' = O^T x_T (the same chain on the transposed block).
__device__ __forceinline__ double rot_row_t(const double *O, int kk, int a, const double *in) {
    double acc = __dmul_rn(O[(kk - 1) * kk + a], in[kk - 1]);
    for (int b = kk - 2; b >= 0; --b) acc = __fma_rn(O[b * kk + a], in[b], acc);
    return acc;
}

// k x k rotation (k >= 3) diagonalizing a symmetric block g (R7), by the 32
// lanes of one warp (every lane calls it, with g's k x k block in gs): cyclic
// Jacobi on the block, pairs (0,1), (0,2), ..., (k-2,k-1), a pair whose entry
// is exactly zero skipped; converged before a sweep when the sum of squared
// off-diagonal entries (in pair order) is at most 1e-30 times the sum of
// squared diagonal entries; at most 32 sweeps (false: not converged).  A
// pair's rotation J = [[c, -s], [s, c]] (jacobi2) updates g <- J g J^T
// (rows p, q recomputed at the other columns from the old values and
// mirrored; the 2 x 2 block as R = J g_TT, then R J^T for a <= b, mirrored)
// and O (starting at I) <- J O on rows p, q.  Lanes 0 and 1 take the serial
// parts (the sweep's two sums side by side; each pair's angle, c on lane 0
// and s on lane 1 from one instruction stream); every new entry is fma(P0, Q0, P1 * Q1) of pre-pair
// values (the rows p, q of g at the other columns, R = J X_TT, the rows p, q
// of O), one lane per entry (2(k-2) + 4 + 2k <= 32 for k <= 8), then the
// 2 x 2 block's R J^T by three lanes, each the same operations on the same
// operands as a sequential evaluation, so the same bits.  gs, os (k x k) and
// js, rs (4 each) are the warp's shared memory; O is left in os.
__device__ inline bool jacobi_k_warp(int k, double *gs, double *os, double *js, double *rs) {
    const int lane = threadIdx.x & 31;
    const unsigned full = 0xffffffffu;
    for (int a = lane; a < k * k; a += 32) os[a] = (a / k == a % k) ? 1.0 : 0.0;
    __syncwarp();
    const int ny = 2 * (k - 2), nt = ny + 4 + 2 * k;
    for (int sweep = 0;; ++sweep) {
        // the sweep's two sums side by side: the off-diagonal one on lane 0,
        // the diagonal one on lane 1 (each the same sequence of operations)
        double sum = 0.0;
        if (lane == 0) {
            for (int p = 0; p < k; ++p)
                for (int q = p + 1; q < k; ++q) sum = __dadd_rn(sum, __dmul_rn(gs[p * k + q], gs[p * k + q]));
        } else if (lane == 1) {
            for (int p = 0; p < k; ++p) sum = __dadd_rn(sum, __dmul_rn(gs[p * k + p], gs[p * k + p]));
        }
        const double dg = __shfl_sync(full, sum, 1);
        int state = 0;
        if (lane == 0) state = sum <= __dmul_rn(1e-30, dg) ? 1 : (sweep == 32 ? 2 : 0);
        state = __shfl_sync(full, state, 0);
        if (state) return state == 1;
        for (int p = 0; p < k - 1; ++p) {
            for (int q = p + 1; q < k; ++q) {
                if (gs[p * k + q] == 0.0) continue;   // the same value in every lane
                // the pair's angle: c on lane 0, s on lane 1 (one divide)
                {
                    const double v = jacobi2_one(gs[p * k + p], gs[p * k + q], gs[q * k + q], lane == 1);
                    if (lane == 0) {
                        js[0] = v;
                        js[3] = v;
                    } else if (lane == 1) {
                        js[1] = -v;
                        js[2] = v;
                    }
                }
                __syncwarp();
                // this lane's entry: fma(J[2a], x_p, J[2a+1] x_q) with (x_p, x_q)
                // the pair's rows p, q of g at column y (y-entries, R) or of O
                int a = 0, col = 0;
                const double *src = gs;
                if (lane < ny) {
                    const int yi = lane >> 1;
                    a = lane & 1;
                    col = yi + (yi >= p) + (yi + (yi >= p) >= q);   // the yi-th column not in {p, q}
                } else if (lane < ny + 4) {
                    const int t = lane - ny;                      // R[a * 2 + cc]
                    a = t >> 1;
                    col = (t & 1) ? q : p;
                } else if (lane < nt) {
                    const int t = lane - ny - 4;                  // O[T[a]][x]
                    a = t / k;
                    col = t - a * k;
                    src = os;
                }
                double v = 0.0;
                if (lane < nt) v = __fma_rn(js[2 * a], src[p * k + col], __dmul_rn(js[2 * a + 1], src[q * k + col]));
                __syncwarp();
                if (lane < ny) {
                    const int row = a ? q : p;
                    gs[row * k + col] = v;
                    gs[col * k + row] = v;
                } else if (lane < ny + 4) {
                    rs[lane - ny] = v;
                } else if (lane < nt) {
                    os[(a ? q : p) * k + col] = v;
                }
                __syncwarp();
                // the 2 x 2 block: (R J^T)_ab for a <= b, mirrored
                if (lane < 3) {
                    const int aa = lane == 2 ? 1 : 0, bb = lane == 0 ? 0 : 1;
                    double acc = __dmul_rn(rs[aa * 2 + 1], js[bb * 2 + 1]);
                    acc = __fma_rn(rs[aa * 2 + 0], js[bb * 2 + 0], acc);
                    const int ra = aa ? q : p, rb = bb ? q : p;
                    gs[ra * k + rb] = acc;
                    gs[rb * k + ra] = acc;
                }
                __syncwarp();
            }
        }
    }
}

}  // namespace pmmf
