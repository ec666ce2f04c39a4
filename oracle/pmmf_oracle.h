/*
 * pmmf_oracle.h -- plain, slow FP64 CPU reference of parallel MMF (pMMF).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  The CUDA library
 * never links, includes or calls it, and it includes nothing from the CUDA
 * library.
 *
 * It follows the paper step by step: Algorithm 1 (stages: cluster, reblock,
 * per-cluster rotation search, blocked update, H), Algorithm 2 (per-cluster
 * randomized greedy Givens / k-point rotation search with the Gram recursion
 * of Sec. 2 and the elimination rule of Sec. 2.2), the matrix-free product and
 * inverse of Sec. 2.4 and the preconditioned CG of Sec. 4.  The places where the
 * paper is silent or garbled are resolved by fixed readings stated next to the
 * code that uses them.
 */
#ifndef PMMF_ORACLE_H
#define PMMF_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    OR_OK = 0,
    OR_ERR_INVALID_ARG = 1,
    OR_ERR_NOT_SYMMETRIC = 2,
    OR_ERR_NONFINITE = 3,
    OR_ERR_OOM = 4,
    OR_ERR_NOT_SPD = 6,
    OR_ERR_NOT_CONVERGED = 8
};

enum { OR_OP_A = 0, OR_OP_A_INV = 1, OR_OP_U = 2, OR_OP_UT = 3, OR_OP_H = 4, OR_OP_H_INV = 5,
       OR_OP_A_INV_SQRT = 6, OR_OP_H_INV_SQRT = 7 };

typedef struct {
    int k;              /* rotation order, 2..8 (Sec. 2, k-point rotations) */
    double eta;         /* fraction of a cluster eliminated per stage (Alg. 2) */
    int cluster_size;   /* target cluster size c (Sec. 2.1) */
    int core_size;      /* stop once |S| <= core_size (delta_L, Sec. 2) */
    uint64_t seed;      /* seed of the counter-based random pick of Alg. 2 */
    int max_stages;     /* <= 0: no limit */
    int lloyd_iters;    /* Lloyd iterations of the clustering step */
    const int32_t *labels;   /* optional stage-1 clusters: label per coordinate in
                                [0, num_labels) (e.g. grid bricks), or NULL */
    int64_t num_labels;
} or_params;

typedef struct or_fact or_fact;

/* Factor a symmetric CSR matrix (rows' columns ascending, no exact zeros).
 * coords: n x dim points used by the clustering step, or NULL for one
 * cluster per stage.  record != 0 keeps every stage's compacted A_p.
 * Never returns NULL for an allocation-free failure: check or_status(). */
or_fact *or_factor(int64_t n, const int64_t *rowptr, const int32_t *col, const double *val,
                   const double *coords, int dim, const or_params *p, int record);
void or_free(or_fact *f);
int or_status(const or_fact *f);

int or_num_stages(const or_fact *f);
int64_t or_stage_active(const or_fact *f, int p);          /* |S_{p-1}| */
int64_t or_stage_clusters(const or_fact *f, int p);        /* m_p */
void or_stage_cluster_offsets(const or_fact *f, int p, int64_t *out);   /* m_p + 1 */
void or_stage_members(const or_fact *f, int p, int32_t *out);           /* |S_{p-1}| */
int64_t or_stage_rotations(const or_fact *f, int p);
/* per rotation in (cluster, step) order: cluster ordinal, tuple size,
 * tuple (global ids, k slots, unused = -1), k x k block (row-major, k*k slots),
 * eliminated global id */
void or_stage_rotation_data(const or_fact *f, int p, int32_t *cluster, int32_t *kk,
                            int32_t *idx, double *O, int32_t *elim);
double or_stage_contrib(const or_fact *f, int p);
int64_t or_stage_nnz(const or_fact *f, int p);              /* nnz of A_p[S_p,S_p] */
/* recorded A_p[S_p, S_p] (record != 0): CSR over global ids, rows of S_p */
int64_t or_stage_matrix(const or_fact *f, int p, int64_t *rowptr_n1, int32_t *col, double *val);

double or_error(const or_fact *f);          /* ||A - U^T H U||_F / ||A||_F */
int or_threads(void);                        /* host threads a factorization uses */

/* The variant PMMF_ROWS_ALL of the Gram's rows (the literal reading of the
 * n-row columns of Alg. 2): the matrix is kept whole, every Gram sums over
 * all n rows and every stage rotates all n rows and columns.  Dense storage,
 * small n; p->labels and p->max_stages as for or_factor.  The accessors and
 * or_apply work on the result; each stage's contrib is the change of the
 * off-structure sum with that stage's survivors as the core. */
or_fact *or_factor_rows_all(int64_t n, const int64_t *rowptr, const int32_t *col,
                            const double *val, const double *coords, int dim,
                            const or_params *p);

/* The steps of one stage one at a time, for running a stage split over
 * several processes (each with a part of the clusters) in tests:
 *   or_step_clusters    stage p's clusters of the active set act[s] and their
 *                       rotation counts: *m, coff[m + 1] (capacity s + 1),
 *                       members[s], e[m] (capacity s);
 *   or_step_search      the search of the clusters own[nown] (rotations in
 *                       order: cluster, tuple size, tuple, block, eliminated);
 *   or_step_transform   out = in Q^T for a set of rows with every cluster's
 *                       rotations of the stage (offsets always, entries when
 *                       they fit cap; *needed = the entry count). */
int or_step_clusters(int64_t n, const double *coords, int dim, int64_t s, const int32_t *act,
                      int p, const or_params *prm, int64_t *m_out, int64_t *coff,
                      int32_t *members, int64_t *e);
int or_step_search(int64_t n, const int64_t *rowptr, const int32_t *col, const double *val,
                    int64_t m, const int64_t *coff, const int32_t *members, const int64_t *e,
                    int64_t nown, const int32_t *own, int p, const or_params *prm, int32_t *rcl,
                    int32_t *rk, int32_t *ridx, double *rO, int32_t *relim);
int or_step_transform(int64_t n, int64_t nrows, const int64_t *rowptr, const int32_t *col,
                       const double *val, int64_t m, const int64_t *coff, const int32_t *members,
                       const int64_t *roff, const int32_t *rk, const int32_t *ridx,
                       const double *rO, int K, int64_t *orowptr, int32_t *ocol, double *oval,
                       int64_t cap, int64_t *needed);
double or_norm_a(const or_fact *f);
int64_t or_core_size(const or_fact *f);
void or_core(const or_fact *f, int32_t *idx, double *core);
void or_hdiag(const or_fact *f, double *hdiag);
/* x, y: n x nrhs row-major */
int or_apply(const or_fact *f, int op, const double *x, double *y, int64_t nrhs);
int or_pcg(const or_fact *f, int64_t n, const int64_t *rowptr, const int32_t *col,
           const double *val, const double *b, double *x, int64_t nrhs, double rtol,
           int maxit, int32_t *iters, double *relres);
/* xi = 1/2: CG on W A W y = W b, W = (U^T H U)^{-1/2}, x = W y. */
int or_pcg_sym(const or_fact *f, int64_t n, const int64_t *rowptr, const int32_t *col,
               const double *val, const double *b, double *x, int64_t nrhs, double rtol,
               int maxit, int32_t *iters, double *relres);

/* Gradient of L = sum <g, op(x)> for op = OR_OP_A or OR_OP_A_INV with the
 * selections fixed: dx (n x nrhs), dO (K*K slots per rotation in stage, step
 * order; stride kk inside), dtheta (per rotation; k = 2 angle with
 * (c, s) = (cos, sin), 0 for larger blocks), dhdiag (n, 0 on core coordinates),
 * dcore (core_size^2; for OR_OP_A_INV on the lower triangle, which is what the
 * inverse reads).  Any output may be NULL. */
int64_t or_total_rotations(const or_fact *f);
int or_apply_grad(const or_fact *f, int op, const double *x, const double *g, int64_t nrhs,
                  double *dx, double *dO, double *dtheta, double *dhdiag, double *dcore);
int or_set_rotation(or_fact *f, int p, int64_t t, const double *O);
int or_set_h(or_fact *f, const double *hdiag, const double *core);

/* building blocks, exposed for the pins */
uint64_t or_splitmix64_next(uint64_t *state);
uint64_t or_draw(uint64_t seed, int64_t p, int64_t u, int64_t t);
int64_t or_pick(uint64_t r, int64_t count);
void or_jacobi2(double a, double b, double d, double *c, double *s);
int or_jacobik(int k, const double *g, double *O);

/* Angle parameterisation of a kk x kk orthogonal block (k-point rotations'
 * derivative): Givens elimination column by column (j = 0..kk-2, l > j) gives
 * theta[kk(kk-1)/2] and D[kk] (+-1) with O = G_1^T .. G_P^T D;
 * or_block_from_angles rebuilds O; or_block_angle_grad maps dL/dO to
 * dL/dtheta at theta (D fixed). */
int or_block_angles(int kk, const double *O, double *theta, double *D);
void or_block_from_angles(int kk, const double *theta, const double *D, double *O);
void or_block_angle_grad(int kk, const double *theta, const double *D, const double *dO,
                         double *dtheta);
void or_sym_rotate(double *X, int64_t ld, int64_t nn, int kk, const int64_t *T, const double *O);
void or_gram(int64_t n, const int64_t *rowptr, const int32_t *col, const double *val,
             int64_t cu, const int32_t *members, double *G, double *M);
int or_partition(int64_t n, const double *coords, int dim, int64_t s, const int32_t *active,
                 int64_t m, int iters, int32_t *label);
void or_quantize(int64_t n, const double *coords, int dim, uint32_t *q);

#ifdef __cplusplus
}
#endif
#endif
