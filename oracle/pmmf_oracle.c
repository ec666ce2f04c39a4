/*
 * pmmf_oracle.c -- plain, slow FP64 CPU reference of parallel MMF (pMMF).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline leg.  It shares no code with the CUDA library.
 *
 * Paper: Kondor, Teneva, Mudrakarta, "Parallel MMF: a Multiresolution Approach
 * to Matrix Computation" (arXiv 1507.04396).  Section numbers below refer to it.
 *
 * Readings used where the paper is silent, garbled or ambiguous (each is also
 * stated where it is used):
 *  R1  Givens convention (Sec. 2, the rotation's four entries; one of them is
 *      garbled): the rotation q on (i, j) maps x_i' = c x_i - s x_j,
 *      x_j' = s x_i + c x_j, and acts as A <- q A q^T, G <- q G q^T (Alg. 2).
 *  R2  Rows of the Gram: the stage-start active set S_{p-1} (all of [n] at
 *      stage 1).  G^u is formed once per stage and only rotated afterwards.
 *  R3  Elimination (Sec. 2.2, Alg. 2): off-norm^2 d(x) = G_xx - M_xx * M_xx of
 *      the locally rotated Gram G and local block M; k = 2: eliminate i when
 *      d(i) < d(j), else j; k >= 3: argmin over the tuple, ties to the later
 *      tuple position.
 *  R4  Residual: contrib_p = sum of A_p[x,y]^2 over x != y in S_{p-1} with x or
 *      y eliminated in stage p; error = sqrt(sum_p contrib_p) / ||A||_F.
 *  R5  Random pick (Alg. 2, "uniformly at random"): counter-based splitmix64.
 *      The generator is pinned by the published known answers; the choice of
 *      stream is this file's definition (the paper gives none): parity
 *      unpinned beyond its properties.
 *  R6  Partner score (Sec. 2.2, absolute value per the text): |G_ij| * w_j
 *      with w_j = 1 / sqrt(G_jj) (0 when G_jj is not positive); top k-1 by score,
 *      ties to the smaller local index.
 *  R7  Angle (Sec. 2.2, "diagonalizing" the Gram sub-block): k = 2 uses the
 *      smaller-angle Jacobi rotation; k >= 3 uses cyclic Jacobi on a k x k copy.
 *  R8  Canonical arithmetic: explicit fma / mul / add in a fixed order, with
 *      this file compiled with -ffp-contract=off.
 *  R9  Gram entries: G_ab = sum over r in S ascending of A[x_a][r] * A[x_b][r]
 *      as a sequential fma chain (rows of the stored matrix).
 *  R10 Clustering (Alg. 1 "cluster", unspecified): k-means on quantized
 *      integer coordinates, Morton-order initialisation, exact integer arithmetic.
 *      This file's definition (the paper gives none): parity unpinned, checked
 *      by properties only (well-separated blobs recovered up to relabelling,
 *      one-dimensional clusters are intervals).
 *  R11 Stage schedule: e_u = floor(eta c_u); trimmed so |S_p| >= core size.
 *  R12 Inverse (Sec. 2.4): 1/H_xx on wavelet coordinates, core by Cholesky.
 *  R13 Blocked update (Alg. 1): A_p = (A_{p-1} Q^T)^T Q^T, i.e. Q applied to
 *      every row, a transpose, then Q applied to every row again; exact zeros
 *      are not stored.
 */
#include "pmmf_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Host threads a factorization uses: 1 for the plain build; the OpenMP
 * build (timing baseline only) spreads clusters and rows over this many. */
int or_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

#define KMAX 8

/* ------------------------------------------------------------------------ */
/* Counter-based random numbers (R5).  splitmix64 as published by Steele, Lea
 * and Flood (OOPSLA 2014): state += golden gamma, then the variant-13 mixer. */

uint64_t or_splitmix64_next(uint64_t *state) {
    uint64_t z = (*state += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static uint64_t mix1(uint64_t x) {
    uint64_t st = x;
    return or_splitmix64_next(&st);
}

/* The draw for (seed, stage p, cluster u, step t): chained hashing. */
uint64_t or_draw(uint64_t seed, int64_t p, int64_t u, int64_t t) {
    uint64_t h = mix1(seed);
    h = mix1(h ^ (uint64_t)p);
    h = mix1(h ^ (uint64_t)u);
    return mix1(h ^ (uint64_t)t);
}

/* Position in [0, count): the high 64 bits of r * count. */
int64_t or_pick(uint64_t r, int64_t count) {
    return (int64_t)(((unsigned __int128)r * (unsigned __int128)(uint64_t)count) >> 64);
}

/* ------------------------------------------------------------------------ */
/* Rotations.                                                               */

/* R7, k = 2: the rotation (c, s) in the convention of R1 that zeroes the
 * off-diagonal of q [[a, b], [b, d]] q^T, with |theta| <= pi/4.  With
 * h = d - a and g = 2b, t = tan(theta) is the smaller root of
 * g t^2 + 2 h t - g = 0, t = sign(h) g / (|h| + sqrt(h^2 + g^2)) (sign(0) = +1).
 * With q = |h| + sqrt(h^2 + g^2) and den = sqrt(q^2 + g^2):
 *     c = q / den,   s = sign(h) g / den.
 * h and g are first scaled by an exact power of two when they are huge or tiny,
 * so that the squares neither overflow nor underflow (the angle is unchanged). */
void or_jacobi2(double a, double b, double d, double *c, double *s) {
    if (b == 0.0) {
        *c = 1.0;
        *s = 0.0;
        return;
    }
    double h = d - a;
    double g = 2.0 * b;
    double m = fabs(h) > fabs(g) ? fabs(h) : fabs(g);
    if (m > 0x1p500) {
        h = h * 0x1p-600;
        g = g * 0x1p-600;
    } else if (m < 0x1p-500) {
        h = h * 0x1p600;
        g = g * 0x1p600;
    }
    double r = sqrt(h * h + g * g);
    double q = fabs(h) + r;
    double den = sqrt(q * q + g * g);
    *c = q / den;
    *s = (h >= 0.0 ? g : -g) / den;
}

/* A k x k rotation block O (row-major, stride k) acting as x_T' = O x_T.
 * Row a of the result is an fma chain over b from k-1 down to 0; for k = 2
 * and O = [[c, -s], [s, c]] this is x_i' = fma(c, x_i, -(s x_j)),
 * x_j' = fma(s, x_i, c x_j). */
static double rot_row(const double *O, int kk, int a, const double *in) {
    double acc = O[a * kk + kk - 1] * in[kk - 1];
    for (int b = kk - 2; b >= 0; --b) acc = fma(O[a * kk + b], in[b], acc);
    return acc;
}

/* Two-sided update X <- O X O^T of an exactly symmetric nn x nn matrix X
 * (row-major, leading dimension ld) on the tuple T.  Rows T are recomputed
 * and mirrored into the columns; the k x k block is formed as R = O X_TT
 * (row step) then R O^T (column step) for a <= b and mirrored.  The result is
 * exactly symmetric. */
void or_sym_rotate(double *X, int64_t ld, int64_t nn, int kk, const int64_t *T, const double *O) {
    double in[KMAX], out[KMAX];
    for (int64_t y = 0; y < nn; ++y) {
        int inT = 0;
        for (int a = 0; a < kk; ++a) inT |= (T[a] == y);
        if (inT) continue;
        for (int a = 0; a < kk; ++a) in[a] = X[T[a] * ld + y];
        for (int a = 0; a < kk; ++a) out[a] = rot_row(O, kk, a, in);
        for (int a = 0; a < kk; ++a) {
            X[T[a] * ld + y] = out[a];
            X[y * ld + T[a]] = out[a];
        }
    }
    double R[KMAX * KMAX];
    for (int cc = 0; cc < kk; ++cc) {
        for (int b = 0; b < kk; ++b) in[b] = X[T[b] * ld + T[cc]];
        for (int a = 0; a < kk; ++a) R[a * kk + cc] = rot_row(O, kk, a, in);
    }
    for (int a = 0; a < kk; ++a) {
        for (int b = a; b < kk; ++b) {
            /* (R O^T)[a][b] = sum_c R[a][c] O[b][c], chain over c from k-1 down */
            double acc = R[a * kk + kk - 1] * O[b * kk + kk - 1];
            for (int cc = kk - 2; cc >= 0; --cc) acc = fma(R[a * kk + cc], O[b * kk + cc], acc);
            X[T[a] * ld + T[b]] = acc;
            X[T[b] * ld + T[a]] = acc;
        }
    }
}

/* R7, k >= 3: cyclic Jacobi on a copy of the k x k Gram sub-block.  Pairs in
 * row-cyclic order (0,1), (0,2), ..., (k-2,k-1); a pair whose entry is exactly
 * zero is skipped.  Converged before a sweep when the sum of squared
 * off-diagonal entries is at most 1e-30 times the sum of squared diagonal
 * entries; at most 32 sweeps.  O accumulates the rotations (O <- J O), so
 * O G O^T is (nearly) diagonal.  Returns OR_ERR_NOT_CONVERGED after 32 sweeps. */
int or_jacobik(int k, const double *g_in, double *O) {
    double g[KMAX * KMAX];
    memcpy(g, g_in, sizeof(double) * (size_t)(k * k));
    for (int a = 0; a < k * k; ++a) O[a] = 0.0;
    for (int a = 0; a < k; ++a) O[a * k + a] = 1.0;
    for (int sweep = 0;; ++sweep) {
        double off = 0.0, dg = 0.0;
        for (int p = 0; p < k; ++p)
            for (int q = p + 1; q < k; ++q) off = off + g[p * k + q] * g[p * k + q];
        for (int p = 0; p < k; ++p) dg = dg + g[p * k + p] * g[p * k + p];
        if (off <= 1e-30 * dg) return OR_OK;
        if (sweep == 32) return OR_ERR_NOT_CONVERGED;
        for (int p = 0; p < k - 1; ++p) {
            for (int q = p + 1; q < k; ++q) {
                if (g[p * k + q] == 0.0) continue;
                double c, s;
                or_jacobi2(g[p * k + p], g[p * k + q], g[q * k + q], &c, &s);
                double J[4] = {c, -s, s, c};
                int64_t T[2] = {p, q};
                or_sym_rotate(g, k, k, 2, T, J);
                for (int x = 0; x < k; ++x) {
                    double op = O[p * k + x], oq = O[q * k + x];
                    double in2[2] = {op, oq};
                    O[p * k + x] = rot_row(J, 2, 0, in2);
                    O[q * k + x] = rot_row(J, 2, 1, in2);
                }
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Gram of a cluster (Alg. 2 "compute the Gram matrix", R2, R9) and its local
 * symmetric diagonal block M (entries of row min(x_a, x_b), mirrored).      */

void or_gram(int64_t n, const int64_t *rowptr, const int32_t *col, const double *val,
             int64_t cu, const int32_t *members, double *G, double *M) {
    (void)n;
    for (int64_t a = 0; a < cu; ++a) {
        for (int64_t b = a; b < cu; ++b) {
            int64_t xa = members[a], xb = members[b];
            int64_t pa = rowptr[xa], ea = rowptr[xa + 1];
            int64_t pb = rowptr[xb], eb = rowptr[xb + 1];
            double acc = 0.0, mv = 0.0;
            for (int64_t q = pa; q < ea; ++q)
                if (col[q] == xb) mv = val[q];
            while (pa < ea && pb < eb) {
                if (col[pa] < col[pb]) {
                    ++pa;
                } else if (col[pa] > col[pb]) {
                    ++pb;
                } else {
                    acc = fma(val[pa], val[pb], acc);
                    ++pa;
                    ++pb;
                }
            }
            G[a * cu + b] = acc;
            G[b * cu + a] = acc;
            M[a * cu + b] = mv;
            M[b * cu + a] = mv;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Clustering (Alg. 1 "cluster the active columns", R10).
 * Coordinates are quantized once to 15-bit integers per dimension over the
 * bounding box of all n points; initial centroids are the means of m equal
 * chunks of the active points in Morton order (ties by index); then Lloyd
 * iterations with squared integer distances (ties to the lower centroid) and
 * centroids rounded to the integer grid, round(sum / count) with halves up.
 * An empty cluster keeps its centroid.  All arithmetic is exact.            */

#define QMAX 32767u

void or_quantize(int64_t n, const double *coords, int dim, uint32_t *q) {
    for (int d = 0; d < dim; ++d) {
        double lo = coords[d], hi = coords[d];
        for (int64_t i = 1; i < n; ++i) {
            double v = coords[i * dim + d];
            if (v < lo) lo = v;
            if (v > hi) hi = v;
        }
        double span = hi - lo;
        double scale = span > 0.0 ? (double)QMAX / span : 0.0;
        for (int64_t i = 0; i < n; ++i) {
            double f = floor((coords[i * dim + d] - lo) * scale);
            uint32_t v = f <= 0.0 ? 0u : (f >= (double)QMAX ? QMAX : (uint32_t)f);
            q[i * dim + d] = v;
        }
    }
}

static uint64_t morton_code(const uint32_t *q, int dim) {
    uint64_t code = 0;
    for (int b = 0; b < 15; ++b)
        for (int d = 0; d < dim; ++d) code |= (uint64_t)((q[d] >> b) & 1u) << (b * dim + d);
    return code;
}

typedef struct { uint64_t key; int32_t id; } keyed;

static int cmp_keyed(const void *x, const void *y) {
    const keyed *a = (const keyed *)x, *b = (const keyed *)y;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    return (a->id > b->id) - (a->id < b->id);
}

static uint64_t dist2(const uint32_t *q, const int64_t *c, int dim) {
    uint64_t s = 0;
    for (int d = 0; d < dim; ++d) {
        int64_t t = (int64_t)q[d] - c[d];
        s += (uint64_t)(t * t);
    }
    return s;
}

static int partition_q(const uint32_t *q, int dim, int64_t s, const int32_t *active, int64_t m,
                       int iters, int32_t *label) {
    keyed *ord = (keyed *)malloc(sizeof(keyed) * (size_t)s);
    int64_t *cen = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m * dim));
    int64_t *sum = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m * dim));
    int64_t *cnt = (int64_t *)malloc(sizeof(int64_t) * (size_t)m);
    if (!ord || !cen || !sum || !cnt) {
        free(ord); free(cen); free(sum); free(cnt);
        return OR_ERR_OOM;
    }
    for (int64_t r = 0; r < s; ++r) {
        ord[r].key = morton_code(q + (int64_t)active[r] * dim, dim);
        ord[r].id = active[r];
    }
    qsort(ord, (size_t)s, sizeof(keyed), cmp_keyed);
    for (int64_t t = 0; t < m; ++t) {
        int64_t lo = t * s / m, hi = (t + 1) * s / m;
        for (int d = 0; d < dim; ++d) {
            int64_t acc = 0;
            for (int64_t r = lo; r < hi; ++r) acc += q[(int64_t)ord[r].id * dim + d];
            int64_t c = hi - lo;
            cen[t * dim + d] = (acc + c / 2) / c;
        }
    }
    for (int it = 0; it < iters; ++it) {
        for (int64_t r = 0; r < s; ++r) {
            const uint32_t *qp = q + (int64_t)active[r] * dim;
            int64_t best = 0;
            uint64_t bd = dist2(qp, cen, dim);
            for (int64_t t = 1; t < m; ++t) {
                uint64_t dd = dist2(qp, cen + t * dim, dim);
                if (dd < bd) {
                    bd = dd;
                    best = t;
                }
            }
            label[r] = (int32_t)best;
        }
        memset(sum, 0, sizeof(int64_t) * (size_t)(m * dim));
        memset(cnt, 0, sizeof(int64_t) * (size_t)m);
        for (int64_t r = 0; r < s; ++r) {
            cnt[label[r]] += 1;
            for (int d = 0; d < dim; ++d) sum[label[r] * dim + d] += q[(int64_t)active[r] * dim + d];
        }
        for (int64_t t = 0; t < m; ++t)
            if (cnt[t] > 0)
                for (int d = 0; d < dim; ++d) cen[t * dim + d] = (sum[t * dim + d] + cnt[t] / 2) / cnt[t];
    }
    free(ord); free(cen); free(sum); free(cnt);
    return OR_OK;
}

int or_partition(int64_t n, const double *coords, int dim, int64_t s, const int32_t *active,
                 int64_t m, int iters, int32_t *label) {
    uint32_t *q = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n * dim));
    if (!q) return OR_ERR_OOM;
    or_quantize(n, coords, dim, q);
    int st = partition_q(q, dim, s, active, m, iters, label);
    free(q);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Sparse rows indexed by global id.                                        */

typedef struct { int64_t len; int32_t *col; double *val; } orow;

static void rows_free(orow *r, int64_t n) {
    if (!r) return;
    for (int64_t i = 0; i < n; ++i) { free(r[i].col); free(r[i].val); }
    free(r);
}

typedef struct {
    int64_t s;            /* |S_{p-1}| */
    int64_t m;
    int64_t *coff;        /* m + 1 */
    int32_t *members;     /* s: clusters in order, members ascending */
    int64_t nrot;
    int64_t *roff;        /* m + 1 */
    int32_t *rcl, *rk, *ridx, *relim;   /* ridx: K slots per rotation */
    double *rO;           /* K*K slots per rotation (stride kk inside) */
    double contrib;
    int64_t nnz;
    int64_t *rec_rowptr;  /* n + 1 over global ids (rows outside S_p empty) */
    int32_t *rec_col;
    double *rec_val;
} ostage;

struct or_fact {
    int status;
    int64_t n;
    int K;
    int nst, cap;
    ostage *st;
    double *hdiag;
    int64_t ncore;
    int32_t *core_idx;
    double *core;
    double *chol;         /* lower Cholesky factor of the core, lazily */
    int chol_status;
    double *isqrt;        /* core^{-1/2}, lazily (xi = 1/2 preconditioner) */
    int isqrt_status;
    double err, norm_a;
};

static void stage_free(ostage *s) {
    free(s->coff); free(s->members); free(s->roff); free(s->rcl); free(s->rk);
    free(s->ridx); free(s->relim); free(s->rO);
    free(s->rec_rowptr); free(s->rec_col); free(s->rec_val);
}

void or_free(or_fact *f) {
    if (!f) return;
    for (int p = 0; p < f->nst; ++p) stage_free(&f->st[p]);
    free(f->st); free(f->hdiag); free(f->core_idx); free(f->core); free(f->chol);
    free(f->isqrt);
    free(f);
}

int or_status(const or_fact *f) { return f ? f->status : OR_ERR_OOM; }

/* ------------------------------------------------------------------------ */
/* Row transform: apply the stage's rotations Q to one sparse row vector
 * (the row of A Q^T).  Each touched cluster's part is expanded into a dense
 * local vector, every rotation of that cluster is applied in step order, and
 * the nonzero results are emitted.  Output sorted by column.               */

typedef struct {
    const ostage *st;
    const int32_t *cl;    /* global id -> cluster ordinal (this stage) */
    const int32_t *loc;   /* global id -> local index */
    int K;
    double *dense;        /* max cluster size */
    int32_t *touched;     /* scratch, max row length */
    int32_t *ocol;        /* output scratch */
    double *oval;
    int64_t ocap;
} xform_ctx;

static int cmp_i32(const void *x, const void *y) {
    int32_t a = *(const int32_t *)x, b = *(const int32_t *)y;
    return (a > b) - (a < b);
}

typedef struct { int32_t col; double val; } cv;
static int cmp_cv(const void *x, const void *y) {
    const cv *a = (const cv *)x, *b = (const cv *)y;
    return (a->col > b->col) - (a->col < b->col);
}

static int transform_row(xform_ctx *cx, const orow *in, orow *out) {
    const ostage *st = cx->st;
    int64_t nt = 0;
    for (int64_t e = 0; e < in->len; ++e) cx->touched[nt++] = cx->cl[in->col[e]];
    qsort(cx->touched, (size_t)nt, sizeof(int32_t), cmp_i32);
    int64_t nu = 0;
    for (int64_t e = 0; e < nt; ++e)
        if (nu == 0 || cx->touched[nu - 1] != cx->touched[e]) cx->touched[nu++] = cx->touched[e];
    int64_t no = 0;
    for (int64_t ui = 0; ui < nu; ++ui) {
        int32_t u = cx->touched[ui];
        int64_t base = st->coff[u], cu = st->coff[u + 1] - base;
        for (int64_t l = 0; l < cu; ++l) cx->dense[l] = 0.0;
        for (int64_t e = 0; e < in->len; ++e)
            if (cx->cl[in->col[e]] == u) cx->dense[cx->loc[in->col[e]]] = in->val[e];
        for (int64_t t = st->roff[u]; t < st->roff[u + 1]; ++t) {
            int kk = st->rk[t];
            double vin[KMAX], vout[KMAX];
            int64_t T[KMAX];
            for (int a = 0; a < kk; ++a) {
                T[a] = cx->loc[st->ridx[t * cx->K + a]];
                vin[a] = cx->dense[T[a]];
            }
            for (int a = 0; a < kk; ++a) vout[a] = rot_row(st->rO + t * cx->K * cx->K, kk, a, vin);
            for (int a = 0; a < kk; ++a) cx->dense[T[a]] = vout[a];
        }
        for (int64_t l = 0; l < cu; ++l) {
            if (cx->dense[l] != 0.0) {
                if (no >= cx->ocap) return OR_ERR_OOM;
                cx->ocol[no] = st->members[base + l];
                cx->oval[no] = cx->dense[l];
                ++no;
            }
        }
    }
    cv *tmp = (cv *)malloc(sizeof(cv) * (size_t)(no ? no : 1));
    out->col = (int32_t *)malloc(sizeof(int32_t) * (size_t)(no ? no : 1));
    out->val = (double *)malloc(sizeof(double) * (size_t)(no ? no : 1));
    if (!tmp || !out->col || !out->val) { free(tmp); return OR_ERR_OOM; }
    for (int64_t e = 0; e < no; ++e) { tmp[e].col = cx->ocol[e]; tmp[e].val = cx->oval[e]; }
    qsort(tmp, (size_t)no, sizeof(cv), cmp_cv);
    for (int64_t e = 0; e < no; ++e) { out->col[e] = tmp[e].col; out->val[e] = tmp[e].val; }
    out->len = no;
    free(tmp);
    return OR_OK;
}

/* out[x] = in[x] Q^T for every active row x (rows are independent; with
 * OpenMP they are spread over the host's cores, each thread with its own
 * scratch, and the results do not depend on the thread count). */
static int transform_rows(const ostage *st, const int32_t *cl, const int32_t *loc, int K,
                          int64_t s, int64_t cmax, int64_t rowcap, const orow *in,
                          const int32_t *act, orow *out) {
    int status = OR_OK;
#ifdef _OPENMP
#pragma omp parallel
#endif
    {
        xform_ctx cx;
        cx.st = st; cx.cl = cl; cx.loc = loc; cx.K = K;
        cx.ocap = rowcap;
        cx.dense = (double *)malloc(sizeof(double) * (size_t)(cmax ? cmax : 1));
        cx.touched = (int32_t *)malloc(sizeof(int32_t) * (size_t)(rowcap ? rowcap : 1));
        cx.ocol = (int32_t *)malloc(sizeof(int32_t) * (size_t)(rowcap ? rowcap : 1));
        cx.oval = (double *)malloc(sizeof(double) * (size_t)(rowcap ? rowcap : 1));
        const int ok = cx.dense && cx.touched && cx.ocol && cx.oval;
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 64)
#endif
        for (int64_t r = 0; r < s; ++r) {
            const int64_t x = act ? act[r] : r;   /* act NULL: rows in order */
            int sr = ok ? transform_row(&cx, &in[x], &out[x]) : OR_ERR_OOM;
            if (sr != OR_OK) {
#ifdef _OPENMP
#pragma omp critical
#endif
                if (status == OR_OK) status = sr;
            }
        }
        free(cx.dense); free(cx.touched); free(cx.ocol); free(cx.oval);
    }
    return status;
}

/* Transpose rows (indexed by global id, only rows in act[0..s)); entries of
 * each output row come out sorted by the source row id. */
static orow *transpose_rows(const orow *in, int64_t n, const int32_t *act, int64_t s) {
    int64_t *cnt = (int64_t *)calloc((size_t)n, sizeof(int64_t));
    orow *out = (orow *)calloc((size_t)n, sizeof(orow));
    if (!cnt || !out) { free(cnt); free(out); return NULL; }
    for (int64_t r = 0; r < s; ++r) {
        const orow *w = &in[act[r]];
        for (int64_t e = 0; e < w->len; ++e) cnt[w->col[e]]++;
    }
    for (int64_t y = 0; y < n; ++y) {
        if (cnt[y]) {
            out[y].col = (int32_t *)malloc(sizeof(int32_t) * (size_t)cnt[y]);
            out[y].val = (double *)malloc(sizeof(double) * (size_t)cnt[y]);
            if (!out[y].col || !out[y].val) { free(cnt); rows_free(out, n); return NULL; }
        }
    }
    for (int64_t r = 0; r < s; ++r) {
        int32_t x = act[r];
        const orow *w = &in[x];
        for (int64_t e = 0; e < w->len; ++e) {
            orow *o = &out[w->col[e]];
            o->col[o->len] = x;
            o->val[o->len] = w->val[e];
            o->len++;
        }
    }
    free(cnt);
    return out;
}

/* ------------------------------------------------------------------------ */
/* One cluster's rotation search: Algorithm 2 generalised to k-point
 * rotations (Sec. 2.2).  G and M are the cluster's c_u x c_u local Gram and
 * symmetric diagonal block (row-major), modified in place.                 */

static int find_rotations(ostage *st, int64_t u, int64_t e_u, double *G, double *M,
                          const or_params *prm, int p, int K, int64_t *rpos) {
    int64_t base = st->coff[u], cu = st->coff[u + 1] - base;
    int64_t *act = (int64_t *)malloc(sizeof(int64_t) * (size_t)cu);
    if (!act) return OR_ERR_OOM;
    int64_t na = cu;
    for (int64_t l = 0; l < cu; ++l) act[l] = l;
    for (int64_t t = 0; t < e_u; ++t) {
        /* select i uniformly at random among the active local indices (R5) */
        uint64_t r = or_draw(prm->seed, p, u, t);
        int64_t i = act[or_pick(r, na)];
        int kk = prm->k < na ? prm->k : (int)na;
        int64_t T[KMAX];
        T[0] = i;
        /* top kk-1 partners by |G_ij| / ||col j|| (R6) */
        for (int a = 1; a < kk; ++a) {
            int64_t best = -1;
            double bs = 0.0;
            for (int64_t q = 0; q < na; ++q) {
                int64_t j = act[q];
                int used = 0;
                for (int b = 0; b < a; ++b) used |= (T[b] == j);
                if (used) continue;
                double gjj = G[j * cu + j];
                double w = gjj > 0.0 ? 1.0 / sqrt(gjj) : 0.0;
                double sc = fabs(G[i * cu + j]) * w;
                if (best < 0 || sc > bs) { best = j; bs = sc; }
            }
            T[a] = best;
        }
        /* the rotation diagonalizing the Gram sub-block (R7) */
        double O[KMAX * KMAX];
        if (kk == 2) {
            double c, s;
            or_jacobi2(G[i * cu + i], G[i * cu + T[1]], G[T[1] * cu + T[1]], &c, &s);
            O[0] = c; O[1] = -s; O[2] = s; O[3] = c;
        } else {
            double sub[KMAX * KMAX];
            for (int a = 0; a < kk; ++a)
                for (int b = 0; b < kk; ++b) sub[a * kk + b] = G[T[a] * cu + T[b]];
            int js = or_jacobik(kk, sub, O);
            if (js != OR_OK) { free(act); return js; }
        }
        /* G <- q G q^T and A <- q A q^T restricted to the cluster (Alg. 2) */
        or_sym_rotate(G, cu, cu, kk, T, O);
        or_sym_rotate(M, cu, cu, kk, T, O);
        /* eliminate the tuple member of smallest off-diagonal norm (R3) */
        int bi = 0;
        double dbest = G[T[0] * cu + T[0]] - M[T[0] * cu + T[0]] * M[T[0] * cu + T[0]];
        for (int a = 1; a < kk; ++a) {
            double d = G[T[a] * cu + T[a]] - M[T[a] * cu + T[a]] * M[T[a] * cu + T[a]];
            if (d <= dbest) { dbest = d; bi = a; }
        }
        int64_t x = T[bi];
        int64_t q = 0;
        while (act[q] != x) ++q;
        for (; q + 1 < na; ++q) act[q] = act[q + 1];
        --na;
        /* record, global ids */
        int64_t rp = (*rpos)++;
        st->rcl[rp] = (int32_t)u;
        st->rk[rp] = kk;
        for (int a = 0; a < K; ++a) st->ridx[rp * K + a] = a < kk ? st->members[base + T[a]] : -1;
        for (int a = 0; a < K * K; ++a) st->rO[rp * K * K + a] = a < kk * kk ? O[a] : 0.0;
        st->relim[rp] = st->members[base + x];
    }
    free(act);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1.                                                             */

static int validate(int64_t n, const int64_t *rowptr, const int32_t *col, const double *val) {
    for (int64_t i = 0; i < n; ++i) {
        if (rowptr[i + 1] < rowptr[i]) return OR_ERR_INVALID_ARG;
        for (int64_t q = rowptr[i]; q < rowptr[i + 1]; ++q) {
            if (col[q] < 0 || col[q] >= n) return OR_ERR_INVALID_ARG;
            if (q > rowptr[i] && col[q] <= col[q - 1]) return OR_ERR_INVALID_ARG;
            if (!isfinite(val[q])) return OR_ERR_NONFINITE;
        }
    }
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t q = rowptr[i]; q < rowptr[i + 1]; ++q) {
            int64_t j = col[q];
            int64_t lo = rowptr[j], hi = rowptr[j + 1];
            int found = 0;
            while (lo < hi) {
                int64_t mid = (lo + hi) / 2;
                if (col[mid] < i) lo = mid + 1;
                else if (col[mid] > i) hi = mid;
                else { found = (memcmp(&val[mid], &val[q], sizeof(double)) == 0); break; }
            }
            if (!found) return OR_ERR_NOT_SYMMETRIC;
        }
    }
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* The clusters of stage p (Alg. 1 "cluster"; R10) and their rotation counts
 * (R11) for the active set act[0..s) (ascending): *mm clusters, offsets
 * coff[mm + 1] into members[s] (ascending inside each cluster), e[mm]
 * rotations each, all allocated here; cl / loc receive every active
 * coordinate's cluster and index inside it.  q: the quantized points of all
 * coordinates (have_coords = 0: one cluster per stage).                     */

static int stage_clusters(const uint32_t *q, int dim, int have_coords, int64_t s,
                          const int32_t *act, int p, const or_params *prm, int64_t *mm_out,
                          int64_t **coff_out, int32_t **members_out, int64_t **e_out,
                          int32_t *cl, int32_t *loc) {
    *coff_out = NULL;
    *members_out = NULL;
    *e_out = NULL;
    int64_t m = (s + prm->cluster_size / 2) / prm->cluster_size;
    if (m < 1) m = 1;
    if (!have_coords) m = 1;
    if (p == 1 && prm->labels) m = prm->num_labels;
    int32_t *label = (int32_t *)calloc((size_t)s, sizeof(int32_t));
    if (!label) return OR_ERR_OOM;
    if (p == 1 && prm->labels) {
        /* given stage-1 clusters (R10: grid bricks for structured grids) */
        for (int64_t r = 0; r < s; ++r) {
            int32_t l = prm->labels[act[r]];
            if (l < 0 || l >= m) { free(label); return OR_ERR_INVALID_ARG; }
            label[r] = l;
        }
    } else if (m > 1) {
        int ps = partition_q(q, dim, s, act, m, prm->lloyd_iters, label);
        if (ps) { free(label); return ps; }
    }
    /* nonempty labels in ascending order become cluster ordinals */
    int64_t *lcount = (int64_t *)calloc((size_t)m, sizeof(int64_t));
    int64_t *lmap = (int64_t *)malloc(sizeof(int64_t) * (size_t)m);
    if (!lcount || !lmap) { free(label); free(lcount); free(lmap); return OR_ERR_OOM; }
    for (int64_t r = 0; r < s; ++r) lcount[label[r]]++;
    int64_t mm = 0;
    for (int64_t t = 0; t < m; ++t) lmap[t] = lcount[t] ? mm++ : -1;
    /* elimination counts (R11) */
    int64_t *coff = (int64_t *)calloc((size_t)(mm + 1), sizeof(int64_t));
    int64_t *e = (int64_t *)calloc((size_t)(mm ? mm : 1), sizeof(int64_t));
    int32_t *members = (int32_t *)malloc(sizeof(int32_t) * (size_t)(s ? s : 1));
    int64_t *fill = (int64_t *)calloc((size_t)(mm ? mm : 1), sizeof(int64_t));
    if (!coff || !e || !members || !fill) {
        free(label); free(lcount); free(lmap); free(coff); free(e); free(members); free(fill);
        return OR_ERR_OOM;
    }
    for (int64_t t = 0; t < m; ++t)
        if (lcount[t]) coff[lmap[t] + 1] = lcount[t];
    for (int64_t u = 0; u < mm; ++u) coff[u + 1] += coff[u];
    int64_t esum = 0;
    for (int64_t u = 0; u < mm; ++u) {
        e[u] = (int64_t)floor(prm->eta * (double)(coff[u + 1] - coff[u]));
        esum += e[u];
    }
    int64_t target = s - prm->core_size;
    while (esum > target) {
        int64_t bu = 0;
        for (int64_t u = 1; u < mm; ++u)
            if (e[u] > e[bu]) bu = u;
        e[bu]--;
        esum--;
    }
    if (esum == 0) {
        /* every cluster too small to rotate: one cluster for this stage */
        for (int64_t r = 0; r < s; ++r) label[r] = 0;
        mm = 1;
        lmap[0] = 0;
        for (int64_t t = 1; t < m; ++t) lmap[t] = 0;
        coff[0] = 0;
        coff[1] = s;
        int64_t ee = (int64_t)floor(prm->eta * (double)s);
        if (ee > target) ee = target;
        if (ee < 1) ee = 1;
        e[0] = ee;
    }
    for (int64_t r = 0; r < s; ++r) {
        int64_t u = lmap[label[r]];
        int64_t pos = coff[u] + fill[u]++;
        members[pos] = act[r];
        cl[act[r]] = (int32_t)u;
        loc[act[r]] = (int32_t)(pos - coff[u]);
    }
    free(fill); free(label); free(lcount); free(lmap);
    *mm_out = mm;
    *coff_out = coff;
    *members_out = members;
    *e_out = e;
    return OR_OK;
}

or_fact *or_factor(int64_t n, const int64_t *rowptr, const int32_t *col, const double *val,
                   const double *coords, int dim, const or_params *prm, int record) {
    or_fact *f = (or_fact *)calloc(1, sizeof(or_fact));
    if (!f) return NULL;
    f->n = n;
    f->K = prm->k;
    if (n < 1 || prm->k < 2 || prm->k > KMAX || !(prm->eta > 0.0 && prm->eta < 1.0) ||
        prm->cluster_size < prm->k || prm->core_size < 1 || prm->core_size > n ||
        (coords && (dim < 1 || dim > 3)) || (prm->labels && prm->num_labels < 1)) {
        f->status = OR_ERR_INVALID_ARG;
        return f;
    }
    f->status = validate(n, rowptr, col, val);
    if (f->status) return f;
    const int K = prm->k;

    /* working copy of A as rows by global id; ||A||_F */
    orow *A = (orow *)calloc((size_t)n, sizeof(orow));
    int32_t *act = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *cl = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *loc = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int8_t *elim = (int8_t *)calloc((size_t)n, 1);
    f->hdiag = (double *)calloc((size_t)n, sizeof(double));
    uint32_t *q = coords ? (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n * dim)) : NULL;
    if (!A || !act || !cl || !loc || !elim || !f->hdiag || (coords && !q)) goto oom;
    double nrm = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t len = rowptr[i + 1] - rowptr[i];
        A[i].len = len;
        A[i].col = (int32_t *)malloc(sizeof(int32_t) * (size_t)(len ? len : 1));
        A[i].val = (double *)malloc(sizeof(double) * (size_t)(len ? len : 1));
        if (!A[i].col || !A[i].val) goto oom;
        memcpy(A[i].col, col + rowptr[i], sizeof(int32_t) * (size_t)len);
        memcpy(A[i].val, val + rowptr[i], sizeof(double) * (size_t)len);
        for (int64_t e = 0; e < len; ++e) nrm = nrm + A[i].val[e] * A[i].val[e];
        act[i] = (int32_t)i;
    }
    f->norm_a = sqrt(nrm);
    if (coords) or_quantize(n, coords, dim, q);

    int64_t s = n;
    double total = 0.0;
    int p = 0;
    while (s > prm->core_size && (prm->max_stages <= 0 || p < prm->max_stages)) {
        ++p;
        if (f->nst == f->cap) {
            int nc = f->cap ? 2 * f->cap : 16;
            ostage *ns = (ostage *)realloc(f->st, sizeof(ostage) * (size_t)nc);
            if (!ns) goto oom;
            f->st = ns;
            f->cap = nc;
        }
        ostage *st = &f->st[f->nst++];
        memset(st, 0, sizeof(*st));
        st->s = s;

        /* ---- cluster the active coordinates (Alg. 1; R10) and count the
         *      stage's rotations per cluster (R11) ---- */
        int64_t mm = 0, esum = 0;
        int64_t *e = NULL;
        {
            int cs = stage_clusters(q, dim, coords != NULL, s, act, p, prm, &mm, &st->coff,
                                    &st->members, &e, cl, loc);
            if (cs == OR_ERR_INVALID_ARG) { f->status = cs; goto done; }
            if (cs != OR_OK) goto oom;
        }
        st->m = mm;
        for (int64_t u = 0; u < mm; ++u) esum += e[u];

        /* ---- per-cluster rotation search (Alg. 2) ---- */
        st->nrot = esum;
        st->roff = (int64_t *)calloc((size_t)(mm + 1), sizeof(int64_t));
        st->rcl = (int32_t *)malloc(sizeof(int32_t) * (size_t)(esum + 1));
        st->rk = (int32_t *)malloc(sizeof(int32_t) * (size_t)(esum + 1));
        st->ridx = (int32_t *)malloc(sizeof(int32_t) * (size_t)((esum + 1) * K));
        st->relim = (int32_t *)malloc(sizeof(int32_t) * (size_t)(esum + 1));
        st->rO = (double *)malloc(sizeof(double) * (size_t)((esum + 1) * K * K));
        if (!st->roff || !st->rcl || !st->rk || !st->ridx || !st->relim || !st->rO) { free(e); goto oom; }
        int64_t cmax = 0;
        for (int64_t u = 0; u < mm; ++u) {
            st->roff[u + 1] = st->roff[u] + e[u];
            if (st->coff[u + 1] - st->coff[u] > cmax) cmax = st->coff[u + 1] - st->coff[u];
        }
        {
            double *G = (double *)malloc(sizeof(double) * (size_t)(cmax * cmax));
            double *M = (double *)malloc(sizeof(double) * (size_t)(cmax * cmax));
            int64_t *rp = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
            int32_t *cc = NULL;
            double *vv = NULL;
            int64_t nnz = 0;
            if (!G || !M || !rp) { free(G); free(M); free(rp); free(e); goto oom; }
            /* present the stored rows as one CSR over global ids for or_gram */
            for (int64_t i = 0; i < n; ++i) nnz += A[i].len;
            cc = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnz ? nnz : 1));
            vv = (double *)malloc(sizeof(double) * (size_t)(nnz ? nnz : 1));
            if (!cc || !vv) { free(G); free(M); free(rp); free(cc); free(vv); free(e); goto oom; }
            rp[0] = 0;
            for (int64_t i = 0; i < n; ++i) {
                memcpy(cc + rp[i], A[i].col, sizeof(int32_t) * (size_t)A[i].len);
                memcpy(vv + rp[i], A[i].val, sizeof(double) * (size_t)A[i].len);
                rp[i + 1] = rp[i] + A[i].len;
            }
            int status = OR_OK;
            /* Clusters are independent (Sec. 2.1): each writes its rotations
             * from its own offset roff[u].  Built with OpenMP, the clusters
             * are spread over the host's cores (the paper's m-fold
             * parallelism), each thread with its own G and M; the results do
             * not depend on the thread count. */
#ifdef _OPENMP
#pragma omp parallel
#endif
            {
                double *Gt = G, *Mt = M;
#ifdef _OPENMP
                if (omp_get_thread_num() != 0) {
                    Gt = (double *)malloc(sizeof(double) * (size_t)(cmax * cmax));
                    Mt = (double *)malloc(sizeof(double) * (size_t)(cmax * cmax));
                }
#pragma omp for schedule(dynamic, 1)
#endif
                for (int64_t u = 0; u < mm; ++u) {
                    int su = OR_OK;
                    if (!Gt || !Mt) {
                        su = OR_ERR_OOM;
                    } else {
                        int64_t cu = st->coff[u + 1] - st->coff[u];
                        int64_t rpos = st->roff[u];
                        or_gram(n, rp, cc, vv, cu, st->members + st->coff[u], Gt, Mt);
                        su = find_rotations(st, u, e[u], Gt, Mt, prm, p, K, &rpos);
                    }
                    if (su != OR_OK) {
#ifdef _OPENMP
#pragma omp critical
#endif
                        if (status == OR_OK) status = su;
                    }
                }
                if (Gt != G) free(Gt);
                if (Mt != M) free(Mt);
            }
            free(G); free(M); free(rp); free(cc); free(vv);
            if (status != OR_OK) { free(e); f->status = status; goto done; }
        }
        free(e);
        for (int64_t t = 0; t < st->nrot; ++t) elim[st->relim[t]] = 1;

        /* ---- blocked update A_p = (A Q^T)^T Q^T (Alg. 1; R13) ---- */
        {
            int64_t maxlen = 1;
            for (int64_t r = 0; r < s; ++r)
                if (A[act[r]].len > maxlen) maxlen = A[act[r]].len;
            orow *V = (orow *)calloc((size_t)n, sizeof(orow));
            if (!V) goto oom;
            int status = transform_rows(st, cl, loc, K, s, cmax, s, A, act, V);
            orow *W = status == OR_OK ? transpose_rows(V, n, act, s) : NULL;
            rows_free(V, n);
            if (!W) status = status ? status : OR_ERR_OOM;
            orow *Ap = (orow *)calloc((size_t)n, sizeof(orow));
            if (!Ap) status = OR_ERR_OOM;
            if (status == OR_OK) status = transform_rows(st, cl, loc, K, s, cmax, s, W, act, Ap);
            rows_free(W, n);
            if (status != OR_OK) { rows_free(Ap, n); f->status = status; goto done; }

            /* ---- residual, H diagonal, compaction to S_p (Alg. 1; R4) ---- */
            double contrib = 0.0;
            int64_t ns = 0, nnz = 0;
            for (int64_t r = 0; r < s; ++r) {
                int32_t x = act[r];
                orow *w = &Ap[x];
                if (elim[x]) {
                    f->hdiag[x] = 0.0;
                    for (int64_t e2 = 0; e2 < w->len; ++e2) {
                        if (w->col[e2] == x) f->hdiag[x] = w->val[e2];
                        else contrib = contrib + w->val[e2] * w->val[e2];
                    }
                    free(w->col); free(w->val);
                    w->col = NULL; w->val = NULL; w->len = 0;
                } else {
                    int64_t o = 0;
                    for (int64_t e2 = 0; e2 < w->len; ++e2) {
                        if (elim[w->col[e2]]) {
                            contrib = contrib + w->val[e2] * w->val[e2];
                        } else {
                            w->col[o] = w->col[e2];
                            w->val[o] = w->val[e2];
                            ++o;
                        }
                    }
                    w->len = o;
                    nnz += o;
                    act[ns++] = x;
                }
            }
            st->contrib = contrib;
            st->nnz = nnz;
            total = total + contrib;
            rows_free(A, n);
            A = Ap;
            s = ns;
            for (int64_t i = 0; i < n; ++i)
                if (elim[i] == 1) elim[i] = 2;   /* eliminated in an earlier stage */
            if (record) {
                st->rec_rowptr = (int64_t *)calloc((size_t)(n + 1), sizeof(int64_t));
                st->rec_col = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnz ? nnz : 1));
                st->rec_val = (double *)malloc(sizeof(double) * (size_t)(nnz ? nnz : 1));
                if (!st->rec_rowptr || !st->rec_col || !st->rec_val) goto oom;
                for (int64_t i = 0; i < n; ++i) {
                    st->rec_rowptr[i + 1] = st->rec_rowptr[i] + A[i].len;
                    memcpy(st->rec_col + st->rec_rowptr[i], A[i].col, sizeof(int32_t) * (size_t)A[i].len);
                    memcpy(st->rec_val + st->rec_rowptr[i], A[i].val, sizeof(double) * (size_t)A[i].len);
                }
            }
        }
    }
    /* ---- H: the core A_L[S_L, S_L] plus the diagonal (Alg. 1) ---- */
    f->ncore = s;
    f->core_idx = (int32_t *)malloc(sizeof(int32_t) * (size_t)(s ? s : 1));
    f->core = (double *)calloc((size_t)(s > 0 ? s * s : 1), sizeof(double));
    if (!f->core_idx || !f->core) goto oom;
    for (int64_t a = 0; a < s; ++a) {
        f->core_idx[a] = act[a];
        cl[act[a]] = (int32_t)a;   /* reuse as core position */
    }
    for (int64_t a = 0; a < s; ++a) {
        orow *w = &A[act[a]];
        for (int64_t e2 = 0; e2 < w->len; ++e2) f->core[a * s + cl[w->col[e2]]] = w->val[e2];
        f->hdiag[act[a]] = f->core[a * s + a];
    }
    f->err = f->norm_a > 0.0 ? sqrt(total) / f->norm_a : 0.0;
    goto done;
oom:
    f->status = OR_ERR_OOM;
done:
    rows_free(A, n);
    free(act); free(cl); free(loc); free(elim); free(q);
    return f;
}

/* ------------------------------------------------------------------------ */
/* Accessors.                                                               */

int or_num_stages(const or_fact *f) { return f->nst; }
int64_t or_stage_active(const or_fact *f, int p) { return f->st[p].s; }
int64_t or_stage_clusters(const or_fact *f, int p) { return f->st[p].m; }
void or_stage_cluster_offsets(const or_fact *f, int p, int64_t *out) {
    memcpy(out, f->st[p].coff, sizeof(int64_t) * (size_t)(f->st[p].m + 1));
}
void or_stage_members(const or_fact *f, int p, int32_t *out) {
    memcpy(out, f->st[p].members, sizeof(int32_t) * (size_t)f->st[p].s);
}
int64_t or_stage_rotations(const or_fact *f, int p) { return f->st[p].nrot; }
void or_stage_rotation_data(const or_fact *f, int p, int32_t *cluster, int32_t *kk,
                            int32_t *idx, double *O, int32_t *elimid) {
    const ostage *st = &f->st[p];
    int K = f->K;
    memcpy(cluster, st->rcl, sizeof(int32_t) * (size_t)st->nrot);
    memcpy(kk, st->rk, sizeof(int32_t) * (size_t)st->nrot);
    memcpy(idx, st->ridx, sizeof(int32_t) * (size_t)(st->nrot * K));
    memcpy(O, st->rO, sizeof(double) * (size_t)(st->nrot * K * K));
    memcpy(elimid, st->relim, sizeof(int32_t) * (size_t)st->nrot);
}
double or_stage_contrib(const or_fact *f, int p) { return f->st[p].contrib; }
int64_t or_stage_nnz(const or_fact *f, int p) { return f->st[p].nnz; }
int64_t or_stage_matrix(const or_fact *f, int p, int64_t *rowptr_n1, int32_t *col, double *val) {
    const ostage *st = &f->st[p];
    if (!st->rec_rowptr) return -1;
    if (rowptr_n1) memcpy(rowptr_n1, st->rec_rowptr, sizeof(int64_t) * (size_t)(f->n + 1));
    if (col) memcpy(col, st->rec_col, sizeof(int32_t) * (size_t)st->nnz);
    if (val) memcpy(val, st->rec_val, sizeof(double) * (size_t)st->nnz);
    return st->nnz;
}
double or_error(const or_fact *f) { return f->err; }
double or_norm_a(const or_fact *f) { return f->norm_a; }
int64_t or_core_size(const or_fact *f) { return f->ncore; }
void or_core(const or_fact *f, int32_t *idx, double *core) {
    memcpy(idx, f->core_idx, sizeof(int32_t) * (size_t)f->ncore);
    memcpy(core, f->core, sizeof(double) * (size_t)(f->ncore * f->ncore));
}
void or_hdiag(const or_fact *f, double *hdiag) { memcpy(hdiag, f->hdiag, sizeof(double) * (size_t)f->n); }

/* ------------------------------------------------------------------------ */
/* Matrix-free arithmetic (Sec. 2.4): U x applies the stages in order and each
 * stage's rotations in step order; U^T x runs backwards with transposed
 * blocks; H acts as diagonal on wavelet coordinates and as the dense core on
 * S_L; H^{-1} inverts the diagonal entries and solves with the core's
 * Cholesky factor (R12).                                                   */

static void apply_u(const or_fact *f, double *z, int64_t nrhs, int transpose) {
    int K = f->K;
    for (int pi = 0; pi < f->nst; ++pi) {
        int p = transpose ? f->nst - 1 - pi : pi;
        const ostage *st = &f->st[p];
        for (int64_t ti = 0; ti < st->nrot; ++ti) {
            int64_t t = transpose ? st->nrot - 1 - ti : ti;
            int kk = st->rk[t];
            const double *O = st->rO + t * K * K;
            double Ot[KMAX * KMAX];
            if (transpose) {
                for (int a = 0; a < kk; ++a)
                    for (int b = 0; b < kk; ++b) Ot[a * kk + b] = O[b * kk + a];
                O = Ot;
            }
            for (int64_t r = 0; r < nrhs; ++r) {
                double in[KMAX];
                for (int a = 0; a < kk; ++a) in[a] = z[(int64_t)st->ridx[t * K + a] * nrhs + r];
                for (int a = 0; a < kk; ++a) z[(int64_t)st->ridx[t * K + a] * nrhs + r] = rot_row(O, kk, a, in);
            }
        }
    }
}

static int core_cholesky(or_fact *f) {
    if (f->chol) return f->chol_status;
    int64_t m = f->ncore;
    f->chol = (double *)calloc((size_t)(m > 0 ? m * m : 1), sizeof(double));
    if (!f->chol) return OR_ERR_OOM;
    double *L = f->chol;
    f->chol_status = OR_OK;
    for (int64_t j = 0; j < m; ++j) {
        double d = f->core[j * m + j];
        for (int64_t c = 0; c < j; ++c) d = d - L[j * m + c] * L[j * m + c];
        if (!(d > 0.0)) { f->chol_status = OR_ERR_NOT_SPD; return f->chol_status; }
        L[j * m + j] = sqrt(d);
        for (int64_t i = j + 1; i < m; ++i) {
            double v = f->core[i * m + j];
            for (int64_t c = 0; c < j; ++c) v = v - L[i * m + c] * L[j * m + c];
            L[i * m + j] = v / L[j * m + j];
        }
    }
    return OR_OK;
}

/* Symmetric eigendecomposition S = V diag(w) V^T of an m x m matrix by
 * classical cyclic Jacobi (rows of V are eigenvectors): sweeps over all pairs
 * (p, q), each rotation zeroing S_pq with the smaller-angle rotation of R7,
 * until the off-diagonal sum of squares is at most 1e-30 times the total. */
static int sym_eig(int64_t m, double *S, double *w, double *V) {
    for (int64_t a = 0; a < m * m; ++a) V[a] = 0.0;
    for (int64_t a = 0; a < m; ++a) V[a * m + a] = 1.0;
    for (int sweep = 0; sweep < 64; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int64_t p = 0; p < m; ++p)
            for (int64_t q = 0; q < m; ++q) {
                tot = tot + S[p * m + q] * S[p * m + q];
                if (p != q) off = off + S[p * m + q] * S[p * m + q];
            }
        if (off <= 1e-30 * tot) {
            for (int64_t a = 0; a < m; ++a) w[a] = S[a * m + a];
            return OR_OK;
        }
        for (int64_t p = 0; p < m - 1; ++p)
            for (int64_t q = p + 1; q < m; ++q) {
                if (S[p * m + q] == 0.0) continue;
                double c, sn;
                or_jacobi2(S[p * m + p], S[p * m + q], S[q * m + q], &c, &sn);
                /* rows p, q then columns p, q of S; rows p, q of V */
                for (int64_t y = 0; y < m; ++y) {
                    double sp = S[p * m + y], sq = S[q * m + y];
                    S[p * m + y] = c * sp - sn * sq;
                    S[q * m + y] = sn * sp + c * sq;
                }
                for (int64_t y = 0; y < m; ++y) {
                    double sp = S[y * m + p], sq = S[y * m + q];
                    S[y * m + p] = c * sp - sn * sq;
                    S[y * m + q] = sn * sp + c * sq;
                }
                for (int64_t y = 0; y < m; ++y) {
                    double vp = V[p * m + y], vq = V[q * m + y];
                    V[p * m + y] = c * vp - sn * vq;
                    V[q * m + y] = sn * vp + c * vq;
                }
            }
    }
    return OR_ERR_NOT_CONVERGED;
}

/* core^{-1/2} = V^T diag(w^{-1/2}) V of the core's lower triangle mirrored
 * (the symmetric matrix the inverse also uses, R12); NOT_SPD if an
 * eigenvalue is not positive. */
static int core_isqrt(or_fact *f) {
    if (f->isqrt) return f->isqrt_status;
    const int64_t m = f->ncore;
    const size_t mm = (size_t)(m > 0 ? m * m : 1);
    f->isqrt = (double *)calloc(mm, sizeof(double));
    double *S = (double *)malloc(sizeof(double) * mm);
    double *V = (double *)malloc(sizeof(double) * mm);
    double *w = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    if (!f->isqrt || !S || !V || !w) {
        free(S); free(V); free(w);
        return OR_ERR_OOM;
    }
    for (int64_t i = 0; i < m; ++i)
        for (int64_t j = 0; j < m; ++j) S[i * m + j] = i >= j ? f->core[i * m + j] : f->core[j * m + i];
    f->isqrt_status = sym_eig(m, S, w, V);
    if (f->isqrt_status == OR_OK) {
        for (int64_t a = 0; a < m; ++a)
            if (!(w[a] > 0.0)) f->isqrt_status = OR_ERR_NOT_SPD;
    }
    if (f->isqrt_status == OR_OK)
        for (int64_t i = 0; i < m; ++i)
            for (int64_t j = 0; j < m; ++j) {
                double acc = 0.0;
                for (int64_t a = 0; a < m; ++a) acc = acc + V[a * m + i] * V[a * m + j] / sqrt(w[a]);
                f->isqrt[i * m + j] = acc;
            }
    free(S); free(V); free(w);
    return f->isqrt_status;
}

/* mode 0: H; 1: H^{-1}; 2: H^{-1/2} (wavelets 1/sqrt(H_xx), the core's
 * inverse square root). */
static int apply_h(or_fact *f, double *z, int64_t nrhs, int inverse) {
    int64_t n = f->n, m = f->ncore;
    int8_t *isc = (int8_t *)calloc((size_t)n, 1);
    double *zc = (double *)malloc(sizeof(double) * (size_t)(m > 0 && nrhs > 0 ? m * nrhs : 1));
    double *wc = (double *)malloc(sizeof(double) * (size_t)(m > 0 && nrhs > 0 ? m * nrhs : 1));
    if (!isc || !zc || !wc) { free(isc); free(zc); free(wc); return OR_ERR_OOM; }
    for (int64_t a = 0; a < m; ++a) isc[f->core_idx[a]] = 1;
    if (inverse) {
        for (int64_t x = 0; x < n; ++x)
            if (!isc[x] && !(f->hdiag[x] > 0.0)) { free(isc); free(zc); free(wc); return OR_ERR_NOT_SPD; }
        int cs = inverse == 2 ? core_isqrt(f) : core_cholesky(f);
        if (cs) { free(isc); free(zc); free(wc); return cs; }
    }
    for (int64_t a = 0; a < m; ++a)
        for (int64_t r = 0; r < nrhs; ++r) zc[a * nrhs + r] = z[(int64_t)f->core_idx[a] * nrhs + r];
    for (int64_t x = 0; x < n; ++x) {
        if (isc[x]) continue;
        for (int64_t r = 0; r < nrhs; ++r)
            z[x * nrhs + r] = inverse == 2 ? z[x * nrhs + r] / sqrt(f->hdiag[x])
                            : inverse ? z[x * nrhs + r] / f->hdiag[x] : f->hdiag[x] * z[x * nrhs + r];
    }
    for (int64_t r = 0; r < nrhs; ++r) {
        if (inverse != 1) {
            const double *C = inverse == 2 ? f->isqrt : f->core;
            for (int64_t a = 0; a < m; ++a) {
                double acc = 0.0;
                for (int64_t b = 0; b < m; ++b) acc = acc + C[a * m + b] * zc[b * nrhs + r];
                wc[a * nrhs + r] = acc;
            }
        } else {
            const double *L = f->chol;
            for (int64_t a = 0; a < m; ++a) {          /* L y = z */
                double v = zc[a * nrhs + r];
                for (int64_t b = 0; b < a; ++b) v = v - L[a * m + b] * wc[b * nrhs + r];
                wc[a * nrhs + r] = v / L[a * m + a];
            }
            for (int64_t a = m - 1; a >= 0; --a) {     /* L^T w = y */
                double v = wc[a * nrhs + r];
                for (int64_t b = a + 1; b < m; ++b) v = v - L[b * m + a] * wc[b * nrhs + r];
                wc[a * nrhs + r] = v / L[a * m + a];
            }
        }
    }
    for (int64_t a = 0; a < m; ++a)
        for (int64_t r = 0; r < nrhs; ++r) z[(int64_t)f->core_idx[a] * nrhs + r] = wc[a * nrhs + r];
    free(isc); free(zc); free(wc);
    return OR_OK;
}

int or_apply(const or_fact *fc, int op, const double *x, double *y, int64_t nrhs) {
    or_fact *f = (or_fact *)fc;
    if (!f || f->status) return OR_ERR_INVALID_ARG;
    if (y != x) memcpy(y, x, sizeof(double) * (size_t)(f->n * nrhs));
    int st = OR_OK;
    switch (op) {
    case OR_OP_U: apply_u(f, y, nrhs, 0); break;
    case OR_OP_UT: apply_u(f, y, nrhs, 1); break;
    case OR_OP_H: st = apply_h(f, y, nrhs, 0); break;
    case OR_OP_H_INV: st = apply_h(f, y, nrhs, 1); break;
    case OR_OP_H_INV_SQRT: st = apply_h(f, y, nrhs, 2); break;
    case OR_OP_A:
    case OR_OP_A_INV:
    case OR_OP_A_INV_SQRT:
        apply_u(f, y, nrhs, 0);
        st = apply_h(f, y, nrhs, op == OR_OP_A ? 0 : op == OR_OP_A_INV ? 1 : 2);
        if (st == OR_OK) apply_u(f, y, nrhs, 1);
        break;
    default: return OR_ERR_INVALID_ARG;
    }
    return st;
}

/* Preconditioned conjugate gradients with M^{-1} = (U^T H U)^{-1} (Sec. 4,
 * xi = 1), each right-hand side independently, x_0 = 0, stopping when the
 * recurrence residual satisfies ||r|| / ||b|| <= rtol.  relres reports the
 * true residual ||b - A x|| / ||b|| at exit. */
static void spmv(int64_t n, const int64_t *rp, const int32_t *ci, const double *v,
                 const double *x, double *y, int64_t nrhs) {
    for (int64_t i = 0; i < n; ++i)
        for (int64_t r = 0; r < nrhs; ++r) {
            double acc = 0.0;
            for (int64_t q = rp[i]; q < rp[i + 1]; ++q) acc = acc + v[q] * x[(int64_t)ci[q] * nrhs + r];
            y[i * nrhs + r] = acc;
        }
}

int or_pcg(const or_fact *fc, int64_t n, const int64_t *rowptr, const int32_t *col,
           const double *val, const double *b, double *x, int64_t nrhs, double rtol,
           int maxit, int32_t *iters, double *relres) {
    or_fact *f = (or_fact *)fc;
    if (!f || f->status || n != f->n) return OR_ERR_INVALID_ARG;
    size_t sz = sizeof(double) * (size_t)(n * nrhs);
    double *r = (double *)malloc(sz), *z = (double *)malloc(sz), *pv = (double *)malloc(sz),
           *qv = (double *)malloc(sz);
    double *rz = (double *)malloc(sizeof(double) * (size_t)nrhs);
    double *bn = (double *)malloc(sizeof(double) * (size_t)nrhs);
    int8_t *done = (int8_t *)calloc((size_t)nrhs, 1);
    if (!r || !z || !pv || !qv || !rz || !bn || !done) {
        free(r); free(z); free(pv); free(qv); free(rz); free(bn); free(done);
        return OR_ERR_OOM;
    }
    memset(x, 0, sz);
    memcpy(r, b, sz);
    int st = or_apply(f, OR_OP_A_INV, r, z, nrhs);
    if (st) goto out;
    memcpy(pv, z, sz);
    for (int64_t c = 0; c < nrhs; ++c) {
        double a = 0.0, bb = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            a = a + r[i * nrhs + c] * z[i * nrhs + c];
            bb = bb + b[i * nrhs + c] * b[i * nrhs + c];
        }
        rz[c] = a;
        bn[c] = sqrt(bb);
        iters[c] = 0;
        if (bn[c] == 0.0) done[c] = 1;
    }
    for (int it = 1; it <= maxit; ++it) {
        int all = 1;
        for (int64_t c = 0; c < nrhs; ++c) all &= done[c];
        if (all) break;
        spmv(n, rowptr, col, val, pv, qv, nrhs);
        for (int64_t c = 0; c < nrhs; ++c) {
            if (done[c]) continue;
            double pq = 0.0;
            for (int64_t i = 0; i < n; ++i) pq = pq + pv[i * nrhs + c] * qv[i * nrhs + c];
            double alpha = rz[c] / pq;
            double rr = 0.0;
            for (int64_t i = 0; i < n; ++i) {
                x[i * nrhs + c] = x[i * nrhs + c] + alpha * pv[i * nrhs + c];
                r[i * nrhs + c] = r[i * nrhs + c] - alpha * qv[i * nrhs + c];
                rr = rr + r[i * nrhs + c] * r[i * nrhs + c];
            }
            iters[c] = it;
            if (sqrt(rr) / bn[c] <= rtol) done[c] = 1;
        }
        st = or_apply(f, OR_OP_A_INV, r, z, nrhs);
        if (st) goto out;
        for (int64_t c = 0; c < nrhs; ++c) {
            if (done[c]) continue;
            double a = 0.0;
            for (int64_t i = 0; i < n; ++i) a = a + r[i * nrhs + c] * z[i * nrhs + c];
            double beta = a / rz[c];
            rz[c] = a;
            for (int64_t i = 0; i < n; ++i) pv[i * nrhs + c] = z[i * nrhs + c] + beta * pv[i * nrhs + c];
        }
    }
    spmv(n, rowptr, col, val, x, qv, nrhs);
    for (int64_t c = 0; c < nrhs; ++c) {
        double rr = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            double d = b[i * nrhs + c] - qv[i * nrhs + c];
            rr = rr + d * d;
        }
        relres[c] = bn[c] > 0.0 ? sqrt(rr) / bn[c] : 0.0;
        if (!done[c]) st = OR_ERR_NOT_CONVERGED;
    }
out:
    free(r); free(z); free(pv); free(qv); free(rz); free(bn); free(done);
    return st;
}

/* Symmetrically preconditioned conjugate gradients (Sec. 4, xi = 1/2): plain
 * CG on the split system W A W y = W b with W = (U^T H U)^{-1/2}
 * = U^T H^{-1/2} U, each right-hand side independently, y_0 = 0, stopping when
 * the split system's recurrence residual satisfies ||r|| / ||W b|| <= rtol;
 * the solution is x = W y.  relres reports the true residual
 * ||b - A x|| / ||b|| at exit. */
int or_pcg_sym(const or_fact *fc, int64_t n, const int64_t *rowptr, const int32_t *col,
               const double *val, const double *b, double *x, int64_t nrhs, double rtol,
               int maxit, int32_t *iters, double *relres) {
    or_fact *f = (or_fact *)fc;
    if (!f || f->status || n != f->n) return OR_ERR_INVALID_ARG;
    size_t sz = sizeof(double) * (size_t)(n * nrhs);
    double *y = (double *)malloc(sz), *r = (double *)malloc(sz), *pv = (double *)malloc(sz),
           *w = (double *)malloc(sz), *qv = (double *)malloc(sz);
    double *rr = (double *)malloc(sizeof(double) * (size_t)nrhs);
    double *bn = (double *)malloc(sizeof(double) * (size_t)nrhs);
    int8_t *done = (int8_t *)calloc((size_t)nrhs, 1);
    if (!y || !r || !pv || !w || !qv || !rr || !bn || !done) {
        free(y); free(r); free(pv); free(w); free(qv); free(rr); free(bn); free(done);
        return OR_ERR_OOM;
    }
    memset(y, 0, sz);
    int st = or_apply(f, OR_OP_A_INV_SQRT, b, r, nrhs);     /* r = W b */
    if (st) goto out;
    memcpy(pv, r, sz);
    for (int64_t c = 0; c < nrhs; ++c) {
        double a = 0.0;
        for (int64_t i = 0; i < n; ++i) a = a + r[i * nrhs + c] * r[i * nrhs + c];
        rr[c] = a;
        bn[c] = sqrt(a);
        iters[c] = 0;
        if (bn[c] == 0.0) done[c] = 1;
    }
    for (int it = 1; it <= maxit; ++it) {
        int all = 1;
        for (int64_t c = 0; c < nrhs; ++c) all &= done[c];
        if (all) break;
        st = or_apply(f, OR_OP_A_INV_SQRT, pv, w, nrhs);    /* q = W A W p */
        if (st) goto out;
        spmv(n, rowptr, col, val, w, qv, nrhs);
        st = or_apply(f, OR_OP_A_INV_SQRT, qv, qv, nrhs);
        if (st) goto out;
        for (int64_t c = 0; c < nrhs; ++c) {
            if (done[c]) continue;
            double pq = 0.0;
            for (int64_t i = 0; i < n; ++i) pq = pq + pv[i * nrhs + c] * qv[i * nrhs + c];
            double alpha = rr[c] / pq;
            double a = 0.0;
            for (int64_t i = 0; i < n; ++i) {
                y[i * nrhs + c] = y[i * nrhs + c] + alpha * pv[i * nrhs + c];
                r[i * nrhs + c] = r[i * nrhs + c] - alpha * qv[i * nrhs + c];
                a = a + r[i * nrhs + c] * r[i * nrhs + c];
            }
            iters[c] = it;
            if (sqrt(a) / bn[c] <= rtol) done[c] = 1;
            else {
                double beta = a / rr[c];
                rr[c] = a;
                for (int64_t i = 0; i < n; ++i) pv[i * nrhs + c] = r[i * nrhs + c] + beta * pv[i * nrhs + c];
            }
        }
    }
    st = or_apply(f, OR_OP_A_INV_SQRT, y, x, nrhs);         /* x = W y */
    if (st) goto out;
    spmv(n, rowptr, col, val, x, qv, nrhs);
    for (int64_t c = 0; c < nrhs; ++c) {
        double a = 0.0, bb = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            double d = b[i * nrhs + c] - qv[i * nrhs + c];
            a = a + d * d;
            bb = bb + b[i * nrhs + c] * b[i * nrhs + c];
        }
        relres[c] = bb > 0.0 ? sqrt(a / bb) : 0.0;
        if (!done[c]) st = OR_ERR_NOT_CONVERGED;
    }
out:
    free(y); free(r); free(pv); free(w); free(qv); free(rr); free(bn); free(done);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Gradient of the factorized operator (Sec. 2.4's matrix-free product with
 * the greedy selections held fixed; not in the paper).  For
 * L = sum_r <g_r, y_r> with y = U^T M U x, M = H (OR_OP_A) or H^{-1}
 * (OR_OP_A_INV), and U the product of every rotation x_T' = O x_T in stage and
 * step order:
 *   - each block O appears once in U (as x_T' = O x_T) and once in U^T (as
 *     x_T' = O^T x_T); for an occurrence with input v and output gradient g',
 *     dL/dO_ab gains sum_r g'_a v_b (in U) or sum_r g'_b v_a (in U^T);
 *   - with z = U x and w = U g: dL/dx = U^T M^T w, dL/dM = w z^T on the
 *     structure of H (diagonal on wavelet coordinates, dense core);
 *   - for M = H^{-1}: dL/dH = -M^T (dL/dM) M^T (M is symmetric up to rounding
 *     and is used as such); the core enters through its lower triangle only
 *     (the inverse is formed from it), so its gradient is folded onto it.
 * For k = 2 blocks O = [[c, -s], [s, c]] with (c, s) = (cos t, sin t):
 *   dL/dt = -s (dO_00 + dO_11) + c (dO_10 - dO_01).
 * Memory: two n x nrhs vectors plus the tuple entries of every occurrence. */

static int64_t total_rotations(const or_fact *f) {
    int64_t T = 0;
    for (int p = 0; p < f->nst; ++p) T += f->st[p].nrot;
    return T;
}

int64_t or_total_rotations(const or_fact *f) { return f ? total_rotations(f) : 0; }

int or_apply_grad(const or_fact *fc, int op, const double *x, const double *g, int64_t nrhs,
                  double *dx, double *dO, double *dtheta, double *dhdiag, double *dcore) {
    or_fact *f = (or_fact *)fc;
    if (!f || f->status || nrhs < 1 || (op != OR_OP_A && op != OR_OP_A_INV)) return OR_ERR_INVALID_ARG;
    const int K = f->K;
    const int64_t n = f->n, m = f->ncore, T = total_rotations(f);
    const int inverse = op == OR_OP_A_INV;
    const size_t nv = (size_t)(n * nrhs);
    /* rotation occurrences in U order: (stage, step) */
    int32_t *tp = (int32_t *)malloc(sizeof(int32_t) * (size_t)(T > 0 ? T : 1));
    int64_t *tt = (int64_t *)malloc(sizeof(int64_t) * (size_t)(T > 0 ? T : 1));
    double *vin = (double *)malloc(sizeof(double) * (size_t)(T > 0 ? T * K * nrhs : 1));
    double *pin = (double *)malloc(sizeof(double) * (size_t)(T > 0 ? T * K * nrhs : 1));
    double *z = (double *)malloc(sizeof(double) * nv);
    double *u = (double *)malloc(sizeof(double) * nv);
    double *a = (double *)malloc(sizeof(double) * nv);
    double *b = (double *)malloc(sizeof(double) * nv);
    double *G = (double *)calloc((size_t)(T > 0 ? T * K * K : 1), sizeof(double));
    int8_t *isc = (int8_t *)calloc((size_t)(n > 0 ? n : 1), 1);
    int rc = OR_OK;
    if (!tp || !tt || !vin || !pin || !z || !u || !a || !b || !G || !isc) { rc = OR_ERR_OOM; goto done; }
    {
        int64_t q = 0;
        for (int p = 0; p < f->nst; ++p)
            for (int64_t t = 0; t < f->st[p].nrot; ++t) { tp[q] = p; tt[q] = t; ++q; }
    }
#define ROT_O(q) (f->st[tp[q]].rO + tt[q] * K * K)
#define ROT_KK(q) (f->st[tp[q]].rk[tt[q]])
#define ROT_IDX(q, c) ((int64_t)f->st[tp[q]].ridx[tt[q] * K + (c)])
    /* forward through U, keeping each occurrence's input entries */
    memcpy(z, x, sizeof(double) * nv);
    for (int64_t q = 0; q < T; ++q) {
        const int kk = ROT_KK(q);
        const double *O = ROT_O(q);
        for (int64_t r = 0; r < nrhs; ++r) {
            double in[KMAX];
            for (int c = 0; c < kk; ++c) {
                in[c] = z[ROT_IDX(q, c) * nrhs + r];
                vin[(q * K + c) * nrhs + r] = in[c];
            }
            for (int c = 0; c < kk; ++c) z[ROT_IDX(q, c) * nrhs + r] = rot_row(O, kk, c, in);
        }
    }
    /* u = M z; then through U^T (occurrences in reverse), keeping inputs */
    memcpy(u, z, sizeof(double) * nv);
    rc = apply_h(f, u, nrhs, inverse);
    if (rc) goto done;
    memcpy(b, u, sizeof(double) * nv);
    for (int64_t q = T - 1; q >= 0; --q) {
        const int kk = ROT_KK(q);
        const double *O = ROT_O(q);
        for (int64_t r = 0; r < nrhs; ++r) {
            double in[KMAX];
            for (int c = 0; c < kk; ++c) {
                in[c] = b[ROT_IDX(q, c) * nrhs + r];
                pin[(q * K + c) * nrhs + r] = in[c];
            }
            for (int c = 0; c < kk; ++c) {
                double acc = 0.0;
                for (int e = 0; e < kk; ++e) acc = acc + O[e * kk + c] * in[e];
                b[ROT_IDX(q, c) * nrhs + r] = acc;
            }
        }
    }
    /* backward through U^T: y = O_1^T ... O_T^T u; the gradient reaching the
     * output of occurrence q's transposed block is a (U order), and then
     * a <- O a carries it to the block's input */
    memcpy(a, g, sizeof(double) * nv);
    for (int64_t q = 0; q < T; ++q) {
        const int kk = ROT_KK(q);
        const double *O = ROT_O(q);
        double *dq = G + q * K * K;
        for (int64_t r = 0; r < nrhs; ++r) {
            double ga[KMAX];
            for (int c = 0; c < kk; ++c) ga[c] = a[ROT_IDX(q, c) * nrhs + r];
            /* output x'_c = sum_e O_ec in_e: dL/dO_ec += ga_c in_e */
            for (int c = 0; c < kk; ++c)
                for (int e = 0; e < kk; ++e) dq[e * kk + c] = dq[e * kk + c] + ga[c] * pin[(q * K + e) * nrhs + r];
            for (int c = 0; c < kk; ++c) a[ROT_IDX(q, c) * nrhs + r] = rot_row(O, kk, c, ga);
        }
    }
    /* a = w = U g.  b = M w is the gradient at z; keep w for dH first */
    for (int64_t e = 0; e < m; ++e) isc[f->core_idx[e]] = 1;
    if (!inverse) {
        if (dhdiag)
            for (int64_t i = 0; i < n; ++i) {
                double acc = 0.0;
                if (!isc[i])
                    for (int64_t r = 0; r < nrhs; ++r) acc = acc + a[i * nrhs + r] * z[i * nrhs + r];
                dhdiag[i] = acc;
            }
        if (dcore)
            for (int64_t e = 0; e < m; ++e)
                for (int64_t c = 0; c < m; ++c) {
                    double acc = 0.0;
                    for (int64_t r = 0; r < nrhs; ++r)
                        acc = acc + a[(int64_t)f->core_idx[e] * nrhs + r] * z[(int64_t)f->core_idx[c] * nrhs + r];
                    dcore[e * m + c] = acc;
                }
    }
    memcpy(b, a, sizeof(double) * nv);
    rc = apply_h(f, b, nrhs, inverse);
    if (rc) goto done;
    if (inverse) {
        /* dL/dH = -(M w)(M z)^T on H's structure; M z = u */
        if (dhdiag)
            for (int64_t i = 0; i < n; ++i) {
                double acc = 0.0;
                if (!isc[i])
                    for (int64_t r = 0; r < nrhs; ++r) acc = acc + b[i * nrhs + r] * u[i * nrhs + r];
                dhdiag[i] = -acc;
            }
        if (dcore) {
            for (int64_t e = 0; e < m; ++e)
                for (int64_t c = 0; c < m; ++c) {
                    double acc = 0.0;
                    for (int64_t r = 0; r < nrhs; ++r)
                        acc = acc + b[(int64_t)f->core_idx[e] * nrhs + r] * u[(int64_t)f->core_idx[c] * nrhs + r];
                    dcore[e * m + c] = -acc;
                }
            /* the inverse is formed from the core's lower triangle (R12): an
             * entry below the diagonal stands for both (e, c) and (c, e), one
             * above it is not read */
            for (int64_t e = 0; e < m; ++e)
                for (int64_t c = 0; c < e; ++c) {
                    dcore[e * m + c] = dcore[e * m + c] + dcore[c * m + e];
                    dcore[c * m + e] = 0.0;
                }
        }
    }
    /* backward through U (occurrences in reverse): b is the gradient at the
     * block's output; dL/dO_ce += b_c in_e; then b <- O^T b */
    for (int64_t q = T - 1; q >= 0; --q) {
        const int kk = ROT_KK(q);
        const double *O = ROT_O(q);
        double *dq = G + q * K * K;
        for (int64_t r = 0; r < nrhs; ++r) {
            double gb[KMAX];
            for (int c = 0; c < kk; ++c) gb[c] = b[ROT_IDX(q, c) * nrhs + r];
            for (int c = 0; c < kk; ++c)
                for (int e = 0; e < kk; ++e) dq[c * kk + e] = dq[c * kk + e] + gb[c] * vin[(q * K + e) * nrhs + r];
            for (int c = 0; c < kk; ++c) {
                double acc = 0.0;
                for (int e = 0; e < kk; ++e) acc = acc + O[e * kk + c] * gb[e];
                b[ROT_IDX(q, c) * nrhs + r] = acc;
            }
        }
    }
    if (dx) memcpy(dx, b, sizeof(double) * nv);
    if (dO) memcpy(dO, G, sizeof(double) * (size_t)(T * K * K));
    if (dtheta)
        for (int64_t q = 0; q < T; ++q) {
            const double *O = ROT_O(q);
            const double *dq = G + q * K * K;
            if (ROT_KK(q) != 2) { dtheta[q] = 0.0; continue; }
            const double c = O[0], s = O[2];
            dtheta[q] = -s * (dq[0] + dq[3]) + c * (dq[2] - dq[1]);
        }
#undef ROT_O
#undef ROT_KK
#undef ROT_IDX
done:
    free(tp); free(tt); free(vin); free(pin); free(z); free(u); free(a); free(b); free(G); free(isc);
    return rc;
}

/* Replace rotation t of stage p (k x k block, stride kk) -- used by the
 * finite-difference pins of the gradient. */
int or_set_rotation(or_fact *f, int p, int64_t t, const double *O) {
    if (!f || p < 0 || p >= f->nst || t < 0 || t >= f->st[p].nrot) return OR_ERR_INVALID_ARG;
    const int kk = f->st[p].rk[t];
    memcpy(f->st[p].rO + t * f->K * f->K, O, sizeof(double) * (size_t)(kk * kk));
    return OR_OK;
}

/* Replace H (diagonal over all n coordinates, core block m x m); the cached
 * Cholesky factor is dropped. */
int or_set_h(or_fact *f, const double *hdiag, const double *core) {
    if (!f || f->status) return OR_ERR_INVALID_ARG;
    if (hdiag) memcpy(f->hdiag, hdiag, sizeof(double) * (size_t)f->n);
    if (core) memcpy(f->core, core, sizeof(double) * (size_t)(f->ncore * f->ncore));
    free(f->chol);
    f->chol = NULL;
    f->chol_status = OR_OK;
    free(f->isqrt);
    f->isqrt = NULL;
    f->isqrt_status = OR_OK;
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Angle parameterisation of a k-point block (the derivative's angles for
 * k >= 3; not in the paper).  Givens elimination of O column by column: for
 * j = 0 .. kk-2 and l = j+1 .. kk-1 in that order, G_i acts on rows (j, l)
 * with theta_i = atan2(A_lj, A_jj), c = cos, s = sin:
 *   row j <- c row j + s row l,   row l <- -s row j + c row l,
 * which zeroes A_lj.  What remains, G_P .. G_1 O, is orthogonal and upper
 * triangular: D = diag(+-1) (its diagonal, rounded to the sign).  Hence
 *   O = G_1^T G_2^T ... G_P^T D,   P = kk (kk - 1) / 2.                      */

static void givens_rows(double *A, int kk, int j, int l, double c, double s) {
    for (int b = 0; b < kk; ++b) {
        const double aj = A[j * kk + b], al = A[l * kk + b];
        A[j * kk + b] = c * aj + s * al;
        A[l * kk + b] = -s * aj + c * al;
    }
}

/* rows (j, l) <- G^T rows (j, l):  row j <- c row j - s row l,
 * row l <- s row j + c row l (dc, ds: the derivative's (dc/dt, ds/dt)). */
static void givens_rows_t(double *A, int kk, int j, int l, double c, double s) {
    for (int b = 0; b < kk; ++b) {
        const double aj = A[j * kk + b], al = A[l * kk + b];
        A[j * kk + b] = c * aj - s * al;
        A[l * kk + b] = s * aj + c * al;
    }
}

int or_block_angles(int kk, const double *O, double *theta, double *D) {
    if (kk < 2 || kk > KMAX) return OR_ERR_INVALID_ARG;
    double A[KMAX * KMAX];
    memcpy(A, O, sizeof(double) * (size_t)(kk * kk));
    int i = 0;
    for (int j = 0; j + 1 < kk; ++j)
        for (int l = j + 1; l < kk; ++l) {
            const double t = atan2(A[l * kk + j], A[j * kk + j]);
            theta[i++] = t;
            givens_rows(A, kk, j, l, cos(t), sin(t));
        }
    for (int a = 0; a < kk; ++a) D[a] = A[a * kk + a] < 0.0 ? -1.0 : 1.0;
    return OR_OK;
}

void or_block_from_angles(int kk, const double *theta, const double *D, double *O) {
    const int P = kk * (kk - 1) / 2;
    for (int a = 0; a < kk; ++a)
        for (int b = 0; b < kk; ++b) O[a * kk + b] = a == b ? D[a] : 0.0;
    /* O = G_1^T (G_2^T ( ... (G_P^T D))) */
    int i = P;
    for (int j = kk - 2; j >= 0; --j)
        for (int l = kk - 1; l > j; --l) {
            --i;
            givens_rows_t(O, kk, j, l, cos(theta[i]), sin(theta[i]));
        }
}

/* dL/dtheta_i = < dO, G_1^T .. G_{i-1}^T (dG_i^T/dtheta) G_{i+1}^T .. G_P^T D >
 * = < Lam_i, (dG_i^T/dtheta) B_i > with Lam_i = G_{i-1} .. G_1 dO and
 * B_i = G_{i+1}^T .. G_P^T D; dG^T/dtheta on rows (j, l) is
 * [[-s, -c], [c, -s]]. */
void or_block_angle_grad(int kk, const double *theta, const double *D, const double *dO,
                         double *dtheta) {
    const int P = kk * (kk - 1) / 2;
    int pj[KMAX * KMAX], pl[KMAX * KMAX];
    {
        int i = 0;
        for (int j = 0; j + 1 < kk; ++j)
            for (int l = j + 1; l < kk; ++l) { pj[i] = j; pl[i] = l; ++i; }
    }
    double B[KMAX * KMAX * KMAX * KMAX / 2 + KMAX * KMAX];   /* P + 1 blocks of kk x kk */
    double *Bi = B + (size_t)P * kk * kk;                      /* B_P = D */
    for (int a = 0; a < kk; ++a)
        for (int b = 0; b < kk; ++b) Bi[a * kk + b] = a == b ? D[a] : 0.0;
    for (int i = P - 1; i >= 1; --i) {     /* B_i = G_{i+1}^T B_{i+1}, stored at slot i */
        double *dst = B + (size_t)i * kk * kk;
        memcpy(dst, B + (size_t)(i + 1) * kk * kk, sizeof(double) * (size_t)(kk * kk));
        givens_rows_t(dst, kk, pj[i], pl[i], cos(theta[i]), sin(theta[i]));
    }
    /* slot i (1-based in the comment) holds B_i for i = 1..P at index i - 1 */
    double Lam[KMAX * KMAX];
    memcpy(Lam, dO, sizeof(double) * (size_t)(kk * kk));
    for (int i = 0; i < P; ++i) {
        const double *Bcur = B + (size_t)(i + 1) * kk * kk;
        const double c = cos(theta[i]), s = sin(theta[i]);
        const int j = pj[i], l = pl[i];
        double acc = 0.0;
        for (int b = 0; b < kk; ++b) {
            const double bj = Bcur[j * kk + b], bl = Bcur[l * kk + b];
            acc = acc + Lam[j * kk + b] * (-s * bj - c * bl) + Lam[l * kk + b] * (c * bj - s * bl);
        }
        dtheta[i] = acc;
        givens_rows(Lam, kk, j, l, c, s);   /* Lam_{i+1} = G_i Lam_i */
    }
}

/* ------------------------------------------------------------------------ */
/* The steps of one stage, one at a time (Sec. 2.3: the clusters' searches
 * are independent, and the blocked update needs every cluster's rotations).
 * They let a test run the stage split over several processes, each with a
 * part of the clusters, and compare the merged result with or_factor.  The
 * arithmetic is or_factor's own: these only call its functions.            */

int or_step_clusters(int64_t n, const double *coords, int dim, int64_t s, const int32_t *act,
                      int p, const or_params *prm, int64_t *m_out, int64_t *coff,
                      int32_t *members, int64_t *e) {
    uint32_t *q = NULL;
    if (coords) {
        q = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n * dim));
        if (!q) return OR_ERR_OOM;
        or_quantize(n, coords, dim, q);
    }
    int32_t *cl = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *loc = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int64_t mm = 0, *c = NULL, *ee = NULL;
    int32_t *mem = NULL;
    int st = (cl && loc) ? stage_clusters(q, dim, coords != NULL, s, act, p, prm, &mm, &c, &mem,
                                          &ee, cl, loc)
                         : OR_ERR_OOM;
    if (st == OR_OK) {
        *m_out = mm;
        memcpy(coff, c, sizeof(int64_t) * (size_t)(mm + 1));
        memcpy(members, mem, sizeof(int32_t) * (size_t)s);
        memcpy(e, ee, sizeof(int64_t) * (size_t)mm);
    }
    free(q); free(cl); free(loc); free(c); free(mem); free(ee);
    return st;
}

/* The rotation search of the clusters own[0..nown) of a stage (Alg. 2), each
 * with its own ordinal in the random draws: the Gram of a cluster reads only
 * its members' rows, so rows of other clusters may be empty.  Outputs, the
 * owned clusters' rotations in order (step order inside a cluster): cluster
 * ordinal, tuple size, tuple (K slots), block (K*K slots), eliminated id. */
int or_step_search(int64_t n, const int64_t *rowptr, const int32_t *col, const double *val,
                    int64_t m, const int64_t *coff, const int32_t *members, const int64_t *e,
                    int64_t nown, const int32_t *own, int p, const or_params *prm, int32_t *rcl,
                    int32_t *rk, int32_t *ridx, double *rO, int32_t *relim) {
    ostage st;
    memset(&st, 0, sizeof(st));
    st.m = m;
    st.coff = (int64_t *)coff;
    st.members = (int32_t *)members;
    st.rcl = rcl;
    st.rk = rk;
    st.ridx = ridx;
    st.rO = rO;
    st.relim = relim;
    int64_t cmax = 0;
    for (int64_t a = 0; a < nown; ++a) {
        const int64_t u = own[a];
        if (u < 0 || u >= m) return OR_ERR_INVALID_ARG;
        if (coff[u + 1] - coff[u] > cmax) cmax = coff[u + 1] - coff[u];
    }
    double *G = (double *)malloc(sizeof(double) * (size_t)(cmax > 0 ? cmax * cmax : 1));
    double *M = (double *)malloc(sizeof(double) * (size_t)(cmax > 0 ? cmax * cmax : 1));
    if (!G || !M) { free(G); free(M); return OR_ERR_OOM; }
    int64_t rpos = 0;
    int status = OR_OK;
    for (int64_t a = 0; a < nown && status == OR_OK; ++a) {
        const int64_t u = own[a];
        const int64_t cu = coff[u + 1] - coff[u];
        or_gram(n, rowptr, col, val, cu, members + coff[u], G, M);
        status = find_rotations(&st, u, e[u], G, M, prm, p, prm->k, &rpos);
    }
    free(G); free(M);
    return status;
}

/* out[r] = in[r] Q^T for the rows ids[0..nrows) (CSR rowptr/col/val over
 * those rows, columns global ids): every cluster's rotations of the stage
 * (roff[m + 1] into rk / ridx (global ids) / rO, step order) applied to the
 * row's entries in that cluster, exact zeros dropped, columns ascending.
 * orowptr[nrows + 1] always receives the output's offsets; ocol / oval only
 * when *needed (the output's entry count) fits cap. */
int or_step_transform(int64_t n, int64_t nrows, const int64_t *rowptr, const int32_t *col,
                       const double *val, int64_t m, const int64_t *coff, const int32_t *members,
                       const int64_t *roff, const int32_t *rk, const int32_t *ridx,
                       const double *rO, int K, int64_t *orowptr, int32_t *ocol, double *oval,
                       int64_t cap, int64_t *needed) {
    ostage st;
    memset(&st, 0, sizeof(st));
    st.m = m;
    st.coff = (int64_t *)coff;
    st.members = (int32_t *)members;
    st.roff = (int64_t *)roff;
    st.rk = (int32_t *)rk;
    st.ridx = (int32_t *)ridx;
    st.rO = (double *)rO;
    int32_t *cl = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *loc = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    orow *in = (orow *)calloc((size_t)(nrows ? nrows : 1), sizeof(orow));
    orow *out = (orow *)calloc((size_t)(nrows ? nrows : 1), sizeof(orow));
    int64_t cmax = 1;
    if (!cl || !loc || !in || !out) { free(cl); free(loc); free(in); free(out); return OR_ERR_OOM; }
    for (int64_t u = 0; u < m; ++u) {
        if (coff[u + 1] - coff[u] > cmax) cmax = coff[u + 1] - coff[u];
        for (int64_t l = coff[u]; l < coff[u + 1]; ++l) {
            cl[members[l]] = (int32_t)u;
            loc[members[l]] = (int32_t)(l - coff[u]);
        }
    }
    for (int64_t r = 0; r < nrows; ++r) {
        in[r].len = rowptr[r + 1] - rowptr[r];
        in[r].col = (int32_t *)(col + rowptr[r]);
        in[r].val = (double *)(val + rowptr[r]);
    }
    int status = transform_rows(&st, cl, loc, K, nrows, cmax, n, in, NULL, out);
    int64_t tot = 0;
    orowptr[0] = 0;
    for (int64_t r = 0; r < nrows; ++r) {
        tot += out[r].len;
        orowptr[r + 1] = tot;
    }
    *needed = tot;
    if (status == OR_OK && tot <= cap)
        for (int64_t r = 0; r < nrows; ++r) {
            memcpy(ocol + orowptr[r], out[r].col, sizeof(int32_t) * (size_t)out[r].len);
            memcpy(oval + orowptr[r], out[r].val, sizeof(double) * (size_t)out[r].len);
        }
    rows_free(out, nrows);
    free(in); free(cl); free(loc);
    return status;
}

/* ------------------------------------------------------------------------ */
/* The literal reading of the Gram's rows (R2 variant PMMF_ROWS_ALL): the
 * columns of Alg. 2 are the full n-row columns, so the matrix is never
 * compacted: every stage rotates all n rows and columns (a rotation acts on
 * its active coordinates; the rows and columns of coordinates eliminated
 * earlier are carried along), each cluster's Gram sums over all n rows, and
 * d(x) = G_xx - A_xx^2 uses the full column norm.  Dense n x n storage (small
 * n only).  H = the diagonal entries at elimination (later rotations never
 * touch them) and the final active block; the error is the Frobenius norm of
 * everything else in the final matrix (orthogonal invariance), and stage p's
 * contribution the change of that sum with S_p taken as the core.          */

static double off_structure(const double *D, int64_t n, const int8_t *act) {
    double s = 0.0;
    for (int64_t x = 0; x < n; ++x)
        for (int64_t y = 0; y < n; ++y)
            if (x != y && !(act[x] && act[y])) s = s + D[x * n + y] * D[x * n + y];
    return s;
}

or_fact *or_factor_rows_all(int64_t n, const int64_t *rowptr, const int32_t *col,
                            const double *val, const double *coords, int dim,
                            const or_params *prm) {
    or_fact *f = (or_fact *)calloc(1, sizeof(or_fact));
    if (!f) return NULL;
    f->n = n;
    f->K = prm->k;
    if (n < 1 || prm->k < 2 || prm->k > KMAX || !(prm->eta > 0.0 && prm->eta < 1.0) ||
        prm->cluster_size < prm->k || prm->core_size < 1 || prm->core_size > n ||
        (coords && (dim < 1 || dim > 3))) {
        f->status = OR_ERR_INVALID_ARG;
        return f;
    }
    f->status = validate(n, rowptr, col, val);
    if (f->status) return f;
    const int K = prm->k;
    double *D = (double *)calloc((size_t)(n * n), sizeof(double));
    double *T = (double *)calloc((size_t)(n * n), sizeof(double));
    int32_t *actl = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *cl = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *loc = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int8_t *isact = (int8_t *)malloc((size_t)n);
    uint32_t *q = coords ? (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n * dim)) : NULL;
    f->hdiag = (double *)calloc((size_t)n, sizeof(double));
    if (!D || !T || !actl || !cl || !loc || !isact || !f->hdiag || (coords && !q)) goto oom;
    double nrm = 0.0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
            D[i * n + col[e]] = val[e];
            nrm = nrm + val[e] * val[e];
        }
    f->norm_a = sqrt(nrm);
    if (coords) or_quantize(n, coords, dim, q);
    for (int64_t i = 0; i < n; ++i) { actl[i] = (int32_t)i; isact[i] = 1; }
    int64_t s = n;
    double prev = 0.0;
    int p = 0;
    while (s > prm->core_size && (prm->max_stages <= 0 || p < prm->max_stages)) {
        ++p;
        if (f->nst == f->cap) {
            int nc = f->cap ? 2 * f->cap : 16;
            ostage *ns = (ostage *)realloc(f->st, sizeof(ostage) * (size_t)nc);
            if (!ns) goto oom;
            f->st = ns;
            f->cap = nc;
        }
        ostage *st = &f->st[f->nst++];
        memset(st, 0, sizeof(*st));
        st->s = s;
        int64_t mm = 0, esum = 0;
        int64_t *e = NULL;
        int cs = stage_clusters(q, dim, coords != NULL, s, actl, p, prm, &mm, &st->coff,
                                &st->members, &e, cl, loc);
        if (cs == OR_ERR_INVALID_ARG) { f->status = cs; goto done; }
        if (cs != OR_OK) goto oom;
        st->m = mm;
        for (int64_t u = 0; u < mm; ++u) esum += e[u];
        st->nrot = esum;
        st->roff = (int64_t *)calloc((size_t)(mm + 1), sizeof(int64_t));
        st->rcl = (int32_t *)malloc(sizeof(int32_t) * (size_t)(esum + 1));
        st->rk = (int32_t *)malloc(sizeof(int32_t) * (size_t)(esum + 1));
        st->ridx = (int32_t *)malloc(sizeof(int32_t) * (size_t)((esum + 1) * K));
        st->relim = (int32_t *)malloc(sizeof(int32_t) * (size_t)(esum + 1));
        st->rO = (double *)malloc(sizeof(double) * (size_t)((esum + 1) * K * K));
        if (!st->roff || !st->rcl || !st->rk || !st->ridx || !st->relim || !st->rO) { free(e); goto oom; }
        int64_t cmax = 1;
        for (int64_t u = 0; u < mm; ++u) {
            st->roff[u + 1] = st->roff[u] + e[u];
            if (st->coff[u + 1] - st->coff[u] > cmax) cmax = st->coff[u + 1] - st->coff[u];
        }
        /* search: Grams over all n rows (R9 order: ascending row index) */
        double *G = (double *)malloc(sizeof(double) * (size_t)(cmax * cmax));
        double *M = (double *)malloc(sizeof(double) * (size_t)(cmax * cmax));
        if (!G || !M) { free(G); free(M); free(e); goto oom; }
        int status = OR_OK;
        for (int64_t u = 0; u < mm && status == OR_OK; ++u) {
            const int64_t cu = st->coff[u + 1] - st->coff[u];
            const int32_t *mem = st->members + st->coff[u];
            for (int64_t a = 0; a < cu; ++a)
                for (int64_t b = a; b < cu; ++b) {
                    double acc = 0.0;
                    for (int64_t r = 0; r < n; ++r)
                        acc = fma(D[(int64_t)mem[a] * n + r], D[(int64_t)mem[b] * n + r], acc);
                    const double mv = D[(int64_t)(mem[a] < mem[b] ? mem[a] : mem[b]) * n +
                                        (mem[a] < mem[b] ? mem[b] : mem[a])];
                    G[a * cu + b] = G[b * cu + a] = acc;
                    M[a * cu + b] = M[b * cu + a] = mv;
                }
            int64_t rpos = st->roff[u];
            status = find_rotations(st, u, e[u], G, M, prm, p, K, &rpos);
        }
        free(G); free(M); free(e);
        if (status != OR_OK) { f->status = status; goto done; }
        /* update of the whole matrix: D <- (D Q^T)^T Q^T (R13), every row */
        double *dense = (double *)malloc(sizeof(double) * (size_t)cmax);
        if (!dense) goto oom;
        for (int pass = 0; pass < 2; ++pass) {
            for (int64_t r = 0; r < n; ++r) {
                double *row = D + r * n;
                for (int64_t u = 0; u < mm; ++u) {
                    const int64_t base = st->coff[u], cu = st->coff[u + 1] - base;
                    for (int64_t l = 0; l < cu; ++l) dense[l] = row[st->members[base + l]];
                    for (int64_t t = st->roff[u]; t < st->roff[u + 1]; ++t) {
                        const int kk = st->rk[t];
                        double vin[KMAX], vout[KMAX];
                        int64_t Tl[KMAX];
                        for (int a = 0; a < kk; ++a) {
                            Tl[a] = loc[st->ridx[t * K + a]];
                            vin[a] = dense[Tl[a]];
                        }
                        for (int a = 0; a < kk; ++a) vout[a] = rot_row(st->rO + t * K * K, kk, a, vin);
                        for (int a = 0; a < kk; ++a) dense[Tl[a]] = vout[a];
                    }
                    for (int64_t l = 0; l < cu; ++l) row[st->members[base + l]] = dense[l];
                }
            }
            for (int64_t x = 0; x < n; ++x)
                for (int64_t y = 0; y < n; ++y) T[y * n + x] = D[x * n + y];
            double *sw = D; D = T; T = sw;
        }
        free(dense);
        /* eliminations: H's diagonal; the active set shrinks, nothing is dropped */
        for (int64_t t = 0; t < st->nrot; ++t) {
            const int32_t x = st->relim[t];
            f->hdiag[x] = D[(int64_t)x * n + x];
            isact[x] = 0;
        }
        int64_t ns = 0;
        for (int64_t r = 0; r < s; ++r)
            if (isact[actl[r]]) actl[ns++] = actl[r];
        s = ns;
        const double now = off_structure(D, n, isact);
        st->contrib = now - prev;
        prev = now;
    }
    f->ncore = s;
    f->core_idx = (int32_t *)malloc(sizeof(int32_t) * (size_t)(s ? s : 1));
    f->core = (double *)calloc((size_t)(s > 0 ? s * s : 1), sizeof(double));
    if (!f->core_idx || !f->core) goto oom;
    for (int64_t a = 0; a < s; ++a) {
        f->core_idx[a] = actl[a];
        for (int64_t b = 0; b < s; ++b) f->core[a * s + b] = D[(int64_t)actl[a] * n + actl[b]];
        f->hdiag[actl[a]] = D[(int64_t)actl[a] * n + actl[a]];
    }
    f->err = f->norm_a > 0.0 ? sqrt(prev) / f->norm_a : 0.0;
    goto done;
oom:
    f->status = OR_ERR_OOM;
done:
    free(D); free(T); free(actl); free(cl); free(loc); free(isact); free(q);
    return f;
}
