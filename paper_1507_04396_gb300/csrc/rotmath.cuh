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

// Row a of x_T' = O x_T for a k x k block O (row-major, stride kk): an fma
// chain over b from kk-1 down to 0.  For kk = 2 and O = [[c, -s], [s, c]]
// this is rot_pair.
__device__ __forceinline__ double rot_row(const double *O, int kk, int a, const double *in) {
    double acc = __dmul_rn(O[a * kk + kk - 1], in[kk - 1]);
    for (int b = kk - 2; b >= 0; --b) acc = __fma_rn(O[a * kk + b], in[b], acc);
    return acc;
}

// Row a of x_T' = O^T x_T (the same chain on the transposed block).
__device__ __forceinline__ double rot_row_t(const double *O, int kk, int a, const double *in) {
    double acc = __dmul_rn(O[(kk - 1) * kk + a], in[kk - 1]);
    for (int b = kk - 2; b >= 0; --b) acc = __fma_rn(O[b * kk + a], in[b], acc);
    return acc;
}

// X <- J X J^T on the pair (p, q) of a small symmetric k x k matrix X
// (row-major): rows p, q recomputed for every other column and mirrored; the
// 2 x 2 block as R = J X_TT, then R J^T for a <= b, mirrored.
__device__ __forceinline__ void sym_rotate_pair(double *X, int k, int p, int q, const double *J) {
    for (int y = 0; y < k; ++y) {
        if (y == p || y == q) continue;
        const double in[2] = {X[p * k + y], X[q * k + y]};
        const double o0 = rot_row(J, 2, 0, in), o1 = rot_row(J, 2, 1, in);
        X[p * k + y] = o0;
        X[y * k + p] = o0;
        X[q * k + y] = o1;
        X[y * k + q] = o1;
    }
    const int T[2] = {p, q};
    double R[4];
    for (int cc = 0; cc < 2; ++cc) {
        const double in[2] = {X[T[0] * k + T[cc]], X[T[1] * k + T[cc]]};
        for (int a = 0; a < 2; ++a) R[a * 2 + cc] = rot_row(J, 2, a, in);
    }
    for (int a = 0; a < 2; ++a)
        for (int b = a; b < 2; ++b) {
            double acc = __dmul_rn(R[a * 2 + 1], J[b * 2 + 1]);
            acc = __fma_rn(R[a * 2 + 0], J[b * 2 + 0], acc);
            X[T[a] * k + T[b]] = acc;
            X[T[b] * k + T[a]] = acc;
        }
}

// k x k rotation (k >= 3) diagonalizing a symmetric block g (R7): cyclic
// Jacobi on a copy, pairs (0,1), (0,2), ..., (k-2,k-1), a pair whose entry is
// exactly zero skipped; converged before a sweep when the sum of squared
// off-diagonal entries is at most 1e-30 times the sum of squared diagonal
// entries; at most 32 sweeps.  O accumulates J O.  Returns false when not
// converged after 32 sweeps.
__device__ inline bool jacobi_k(int k, const double *gin, double *O) {
    double g[64];
    for (int a = 0; a < k * k; ++a) g[a] = gin[a];
    for (int a = 0; a < k * k; ++a) O[a] = 0.0;
    for (int a = 0; a < k; ++a) O[a * k + a] = 1.0;
    for (int sweep = 0;; ++sweep) {
        double off = 0.0, dg = 0.0;
        for (int p = 0; p < k; ++p)
            for (int q = p + 1; q < k; ++q) off = __dadd_rn(off, __dmul_rn(g[p * k + q], g[p * k + q]));
        for (int p = 0; p < k; ++p) dg = __dadd_rn(dg, __dmul_rn(g[p * k + p], g[p * k + p]));
        if (off <= __dmul_rn(1e-30, dg)) return true;
        if (sweep == 32) return false;
        for (int p = 0; p < k - 1; ++p) {
            for (int q = p + 1; q < k; ++q) {
                if (g[p * k + q] == 0.0) continue;
                double c, s;
                jacobi2(g[p * k + p], g[p * k + q], g[q * k + q], c, s);
                const double J[4] = {c, -s, s, c};
                sym_rotate_pair(g, k, p, q, J);
                for (int x = 0; x < k; ++x) {
                    const double in2[2] = {O[p * k + x], O[q * k + x]};
                    O[p * k + x] = rot_row(J, 2, 0, in2);
                    O[q * k + x] = rot_row(J, 2, 1, in2);
                }
            }
        }
    }
}

}  // namespace pmmf
