/*
 * pmmf.h -- C-ABI of the GB300 (sm_103a) implementation of parallel
 * Multiresolution Matrix Factorization (pMMF).
 *
 * Paper: R. Kondor, N. Teneva, P. K. Mudrakarta, "Parallel MMF: a Multiresolution
 * Approach to Matrix Computation", arXiv 1507.04396.  The factorization is
 *     A ~= Q_1^T ... Q_L^T H Q_L ... Q_1            (Eq. 1, Sec. 2)
 * with the rotations grouped into stages Qbar_p that share one clustering
 * (Sec. 2.1, Algorithm 1) and found by the randomized greedy search of
 * Algorithm 2 (Sec. 2.2).  H is core-diagonal (Sec. 2, condition 3).
 *
 * Conventions shared by every entry point
 *   - Every function returns pmmf_status and never throws or aborts.  On a
 *     non-OK status pmmf_last_error() returns a message for the calling thread.
 *   - Floating point data is IEEE binary64 (double); indices are int32
 *     (global coordinate ids) and int64 (offsets).
 *   - Pointers are caller-owned unless stated; the library never frees them.
 *     Device pointers must be CUDA device memory of the current device.
 *   - "stream" is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Work is ordered on that stream.  pmmf_factor synchronizes that stream
 *     internally (it reads stage sizes back to size buffers); pmmf_apply is
 *     asynchronous; pmmf_solve_precond synchronizes once per CG iteration.
 *   - Rotations use the convention x_i' = c x_i - s x_j, x_j' = s x_i + c x_j
 *     for a Givens rotation on (i, j) (Sec. 2; the printed entries are garbled).
 */
#ifndef PMMF_H
#define PMMF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PMMF_OK = 0,
    PMMF_ERR_INVALID_ARG = 1,     /* a parameter is out of range or a pointer is NULL */
    PMMF_ERR_NOT_SYMMETRIC = 2,   /* A is not exactly symmetric (structure or bits) */
    PMMF_ERR_NONFINITE = 3,       /* A holds NaN or Inf */
    PMMF_ERR_OOM = 4,             /* device or host allocation failed; nothing leaked */
    PMMF_ERR_CUDA = 5,            /* a CUDA runtime call failed */
    PMMF_ERR_NOT_SPD = 6,         /* H is not positive definite (inverse requested) */
    PMMF_ERR_SINGULAR_CORE = 7,
    PMMF_ERR_NOT_CONVERGED = 8,   /* CG reached maxit, or a k x k Jacobi did not converge */
    PMMF_ERR_TIMEOUT = 9,
    PMMF_ERR_UNSUPPORTED = 10     /* valid input outside what this build handles */
} pmmf_status;

enum { PMMF_HOST = 0, PMMF_DEVICE = 1 };
enum { PMMF_CSR = 0, PMMF_DENSE = 1 };

/* Operations of pmmf_apply (Sec. 2.4, matrix-free arithmetic):
 *   PMMF_OP_A      y = U^T H U x          (the factorized matrix A~)
 *   PMMF_OP_A_INV  y = U^T H^{-1} U x     (its inverse; wavelet diagonal
 *                                          inverted, core inverted)
 *   PMMF_OP_U      y = U x,   U = Qbar_P ... Qbar_1
 *   PMMF_OP_UT     y = U^T x
 *   PMMF_OP_H      y = H x
 *   PMMF_OP_H_INV  y = H^{-1} x
 *   PMMF_OP_A_INV_SQRT  y = U^T H^{-1/2} U x   (A~^{-1/2}, the symmetric
 *                                          preconditioner of Sec. 4 with
 *                                          xi = 1/2; wavelet entries
 *                                          1/sqrt(H_ii), core^{-1/2})
 *   PMMF_OP_H_INV_SQRT  y = H^{-1/2} x
 * The core enters the inverse ops through its lower triangle (mirrored). */
enum { PMMF_OP_A = 0, PMMF_OP_A_INV = 1, PMMF_OP_U = 2, PMMF_OP_UT = 3, PMMF_OP_H = 4,
       PMMF_OP_H_INV = 5, PMMF_OP_A_INV_SQRT = 6, PMMF_OP_H_INV_SQRT = 7 };

/* A symmetric n x n matrix (Sec. 2: "a symmetric matrix A").
 *   PMMF_CSR:   rowptr[n+1] (int64), colidx[nnz] (int32, strictly ascending
 *               inside each row), val[nnz].  Stored exact zeros are allowed
 *               and ignored.
 *   PMMF_DENSE: val is n x ld row-major (ld >= n); rowptr/colidx unused.
 * location says whether the arrays live in host or device memory.
 * Symmetry must be exact: entry (i, j) and (j, i) carry identical bits. */
typedef struct {
    int64_t n;
    int format;
    int location;
    const int64_t *rowptr;
    const int32_t *colidx;
    const double *val;
    int64_t ld;
} pmmf_matrix;

/* Parameters, named as in the paper.
 *   k             rotation order (Sec. 2, k-point rotations), 2 <= k <= 8:
 *                 k = 2 Givens rotations (Algorithm 2), k >= 3 k-point
 *                 rotations diagonalizing the k x k Gram sub-block.
 *   eta           compression ratio of Algorithm 2: floor(eta c_u) rotations
 *                 (one elimination each) per cluster per stage, 0 < eta < 1.
 *   cluster_size  typical cluster size c (Sec. 2.1), >= k; a stage with s
 *                 active coordinates uses m = max(1, round(s / c)) clusters.
 *   core_size     delta_L: stages run while more than core_size coordinates
 *                 are active (1 <= core_size <= n).
 *   seed          seed of the counter-based random pick of Algorithm 2.
 *   max_stages    stop after this many stages (<= 0: no limit).
 *   lloyd_iters   Lloyd iterations of the clustering step (0 -> 10).
 *   coords        optional n x coord_dim row-major points (coord_dim 1..3)
 *                 that the clustering step (Algorithm 1, "cluster") groups by
 *                 k-means; NULL -> one cluster per stage.
 *   coords_location  PMMF_HOST or PMMF_DEVICE for coords.
 *   labels        optional given clusters for stage 1: labels[x] in
 *                 [0, num_labels) for every coordinate x (e.g. the bricks of
 *                 a structured grid); clusters are the nonempty labels in
 *                 ascending order, members ascending.  Later stages use the
 *                 clustering rule.  NULL -> the clustering rule at stage 1
 *                 too.  A label outside [0, num_labels) -> INVALID_ARG.
 *   labels_location  PMMF_HOST or PMMF_DEVICE for labels.
 *   num_labels    number of label values (>= 1 when labels is set).
 *   record_stages nonzero keeps a device copy of every stage's compacted
 *                 A_p (for inspection with pmmf_stage_matrix).
 *   precision     PMMF_PREC_FP64 (0): every Gram entry in FP64 (the oracle's
 *                 arithmetic, bit for bit).  PMMF_PREC_TF32 / PMMF_PREC_BF16:
 *                 dense inputs only (PMMF_DENSE with n <= 24576; anything
 *                 else returns UNSUPPORTED): the Gram matrices are formed on
 *                 the tensor cores from TF32 / BF16 copies with FP32
 *                 accumulation and serve only to shortlist partners; every
 *                 shortlisted partner is re-scored, and every angle, Gram
 *                 diagonal and rotation computed, in FP64 from the FP64 rows
 *                 (the shortlist keeps every candidate that a certified error
 *                 bound cannot rule out, so the choice is the FP64 choice up to
 *                 rounding of the FP64 scores).  Not bit-identical to FP64
 *                 mode; pmmf_get_precision_stats reports the shortlists. */
typedef struct {
    int k;
    double eta;
    int cluster_size;
    int core_size;
    uint64_t seed;
    int max_stages;
    int lloyd_iters;
    const double *coords;
    int coord_dim;
    int coords_location;
    int record_stages;
    int precision;
    const int32_t *labels;
    int labels_location;
    int64_t num_labels;
} pmmf_params;

enum { PMMF_PREC_FP64 = 0, PMMF_PREC_TF32 = 1, PMMF_PREC_BF16 = 2 };

typedef struct pmmf_handle pmmf_handle;

typedef struct {
    int64_t n;
    int32_t stages;
    int64_t core_size;        /* |S_L| */
    int64_t rotations;        /* total number of rotations (= n - |S_L|) */
    int64_t nnz_input;
    double norm_a;            /* ||A||_F */
    double error;             /* ||A - U^T H U||_F / ||A||_F (residual of Sec. 2) */
} pmmf_info;

typedef struct {
    int64_t active;           /* |S_{p-1}| at the start of the stage */
    int64_t clusters;         /* m_p */
    int64_t rotations;
    int64_t nnz_after;        /* nnz of A_p[S_p, S_p] */
    int32_t max_levels;       /* depth of the stage's rotation dependency graph */
    double contrib;           /* this stage's share of ||A - A~||_F^2 */
} pmmf_stage_info;

/* Factor A (Algorithm 1).  On PMMF_OK *out receives a handle owning every
 * device buffer of the factorization (rotations, H); free it with pmmf_free.
 * On error *out is NULL and no memory is leaked.  The input is only read. */
pmmf_status pmmf_factor(const pmmf_matrix *A, const pmmf_params *p, pmmf_handle **out,
                        void *stream);

/* Matrix-free product with the factorization (Sec. 2.4), O(k p n) work.
 * x and y are DEVICE pointers to n x nrhs row-major blocks with leading
 * dimension ld >= nrhs; x == y (in place) is allowed.  Asynchronous.
 * PMMF_OP_A_INV / PMMF_OP_H_INV return PMMF_ERR_NOT_SPD when a wavelet
 * diagonal entry of H is <= 0 or the core is not positive definite; that check
 * runs on the first inverse request and synchronizes the stream once.  The
 * inverse square root ops form core^{-1/2} on their first request by the
 * coupled Newton-Schulz iteration (dense products, at most 100 steps,
 * synchronizing once per step); PMMF_ERR_NOT_SPD when it diverges or stalls
 * (an eigenvalue <= 0, or numerically so). */
pmmf_status pmmf_apply(const pmmf_handle *f, int op, const double *x, double *y, int64_t nrhs,
                       int64_t ld, void *stream);

/* Allocation-free variant of pmmf_apply (the paper has no counterpart; this
 * is a deployment aid).  Same arguments, semantics and results as pmmf_apply,
 * but it never allocates device or host memory: no cudaMalloc / cudaFree and
 * no allocating library routine.  It is for callers that must not allocate
 * inside their loop -- e.g. a solver or serving path running with a fixed
 * memory budget, or code whose allocator is owned by another framework --
 * because an allocation there can fail, synchronize, or fragment memory.
 *   Scratch: the core slice of the vectors (core_size * nrhs doubles) lives
 *   in one library-owned device array of 1,048,576 doubles (8 MiB), held by
 *   every GPU that loads the library until the process exits.  Calls with
 *   core_size * nrhs > 1,048,576 for the H-using ops (all but U and UT)
 *   return PMMF_ERR_UNSUPPORTED with a message naming the limit.
 *   Set-up: the first call on a device (the calling thread's current device)
 *   looks up the array's device address; make that first call before any
 *   stream capture.
 *   Sharing: every call uses the same array, which keeps the previous call's
 *   contents; nothing in it needs to start at zero (each call writes every
 *   entry it reads).  Calls that overlap on the GPU (different streams, or
 *   host threads) race on the array and must be serialized by the caller.
 *   Inverse ops need the core inverse (inverse square root ops: the core's
 *   inverse square root), which pmmf_apply / pmmf_solve_precond /
 *   pmmf_solve_precond_sym form (and allocate) on their first request;
 *   before that this function returns PMMF_ERR_INVALID_ARG. */
pmmf_status pmmf_apply_noalloc(const pmmf_handle *f, int op, const double *x, double *y,
                               int64_t nrhs, int64_t ld, void *stream);

/* Preconditioned conjugate gradients for A x = b with M^{-1} = A~^{-1}
 * (Sec. 4, xi = 1), every column of b independently, x_0 = 0.  A is the
 * system matrix (any location; CSR or dense); b and x are DEVICE n x nrhs
 * row-major (ld = nrhs).  Stops a column when ||r||/||b|| <= rtol (recurrence
 * residual).  iters[nrhs] and relres[nrhs] (HOST) receive the iteration count
 * and the true residual ||b - A x|| / ||b|| at exit.  Returns
 * PMMF_ERR_NOT_CONVERGED if a column did not reach rtol in maxit steps. */
pmmf_status pmmf_solve_precond(const pmmf_handle *f, const pmmf_matrix *A, const double *b,
                               double *x, int64_t nrhs, double rtol, int maxit, int32_t *iters,
                               double *relres, void *stream);

/* Symmetrically preconditioned conjugate gradients (Sec. 4, xi = 1/2): plain
 * CG on W A W y = W b with W = A~^{-1/2} = U^T H^{-1/2} U applied matrix-free,
 * then x = W y; every column independently, y_0 = 0.  Same arguments as
 * pmmf_solve_precond; a column stops when the split system's recurrence
 * residual satisfies ||r|| / ||W b|| <= rtol.  relres is the true residual
 * ||b - A x|| / ||b|| at exit.  In exact arithmetic the iterates equal those
 * of pmmf_solve_precond.  PMMF_ERR_NOT_SPD when H has no real inverse square
 * root; PMMF_ERR_NOT_CONVERGED as for pmmf_solve_precond. */
pmmf_status pmmf_solve_precond_sym(const pmmf_handle *f, const pmmf_matrix *A, const double *b,
                                   double *x, int64_t nrhs, double rtol, int maxit,
                                   int32_t *iters, double *relres, void *stream);

/* ---- batches of independent matrices ---------------------------------------
 * Many independent symmetric matrices factored together (the paper factors
 * one matrix; a batch is many of its problems at once).  Matrix b is factored
 * exactly as pmmf_factor would factor it alone with one cluster per stage
 * (params.coords = NULL) and seed params.seed + b: per stage
 * e = max(1, min(floor(eta c), c - core_size)) rotations for its c active
 * coordinates, until at most core_size remain, which become its core block.
 * All matrices advance through the stages together, so each stage is one
 * launch per kernel kind over every matrix, the longest searches first.
 *
 * pmmf_factor_blockdiag: the batch as ONE block-diagonal matrix A (any format
 * and location accepted by pmmf_factor) whose diagonal block b spans the
 * coordinates block_off[b] .. block_off[b+1]-1 (block_off: HOST, nmat + 1
 * entries, strictly increasing from 0 to n).  An entry outside its diagonal
 * block gives INVALID_ARG.  params.coords must be NULL and max_stages 0;
 * params.cluster_size is not used (each matrix is one cluster) but must still
 * be >= k.
 * The handle acts on the whole block-diagonal operator: pmmf_apply and
 * pmmf_solve_precond take n x nrhs vectors (the matrices' vectors stacked).
 * pmmf_get_h then returns core_idx[nmat * core_stride] (unused slots -1) and
 * core[nmat * core_stride^2]: block b's core at core + b * core_stride^2,
 * row stride core_stride (see pmmf_get_batch).  pmmf_apply_backward is not
 * available on a batch handle (UNSUPPORTED). */
pmmf_status pmmf_factor_blockdiag(const pmmf_matrix *A, int64_t nmat, const int64_t *block_off,
                                  const pmmf_params *p, pmmf_handle **out, void *stream);

/* Convenience form: nmat separate HOST CSR matrices A[0..nmat-1], stacked
 * into one block-diagonal matrix on the host and factored as above. */
pmmf_status pmmf_factor_batched(int64_t nmat, const pmmf_matrix *A, const pmmf_params *p,
                                pmmf_handle **out, void *stream);

/* Shortlist counters of a reduced-precision factorization (HOST outputs, any
 * may be NULL): candidates re-scored in FP64 over all steps, steps whose
 * shortlist held more than 64 candidates, rotation search steps, and the
 * largest shortlist.  All zero in FP64 mode. */
pmmf_status pmmf_get_precision_stats(const pmmf_handle *f, int64_t *rescored, int64_t *fallbacks,
                                     int64_t *steps, int64_t *max_shortlist);

/* Batch layout (HOST outputs, any may be NULL): nmat, core_stride (slot
 * stride of the core blocks), block_off[nmat + 1], errors[nmat] (each
 * matrix's ||A_b - U_b^T H_b U_b||_F / ||A_b||_F) and core_dim[nmat] (each
 * core block's size).  A single factorization reports nmat = 1. */
pmmf_status pmmf_get_batch(const pmmf_handle *f, int64_t *nmat, int64_t *core_stride,
                           int64_t *block_off, double *errors, int32_t *core_dim);

/* ---- differentiation of the factorized operator ----------------------------
 * With the greedy selections held fixed, A~ = U^T H U is a smooth function of
 * x, of H (its wavelet diagonal and its dense core) and of every k = 2
 * rotation's angle theta ((c, s) = (cos theta, sin theta); Sec. 2's Givens
 * rotations).  The paper defines the product and inverse (Sec. 2.4) but no
 * derivative; these calls add one.
 *
 * pmmf_apply_backward: for L = sum over entries of g * op(x), op = PMMF_OP_A
 * (y = A~ x) or PMMF_OP_A_INV (y = A~^{-1} x), writes
 *   dx[n x nrhs] (row-major, ld)   dL/dx
 *   dtheta[rotations]              dL/dtheta, stages in order and (cluster,
 *                                  step) order inside a stage (the order of
 *                                  pmmf_get_stage_rotations); for k >= 3 the
 *                                  rotations are parameterised by their block
 *                                  O (x_T' = O x_T) and dtheta[rotations *
 *                                  k * k] receives dL/dO, k * k slots per
 *                                  rotation, entry (a, b) of a kk x kk block
 *                                  at slot a * kk + b, the others 0
 *   dhdiag[n]                      dL/dH_xx on wavelet coordinates, 0 on core
 *                                  coordinates
 *   dcore[core_size^2]             dL/dcore (row-major; for A_INV the core
 *                                  inverse is formed from the lower triangle,
 *                                  so the gradient sits there: entries above
 *                                  the diagonal are 0)
 * All arrays are DEVICE memory; outputs are overwritten and any of them may be
 * NULL.  The stage-start state of [x | g] is checkpointed per stage and each
 * stage is replayed once, so the cost is about three applies.  Asynchronous on
 * stream (except the first A_INV call, which forms the core inverse).  Errors:
 * INVALID_ARG (op, sizes, NULL x or g), UNSUPPORTED (a batch handle, or a
 * cluster too large for one CTA's shared memory), NOT_SPD (A_INV with H not
 * SPD), OOM. */
pmmf_status pmmf_apply_backward(const pmmf_handle *f, int op, const double *x, const double *g,
                                int64_t nrhs, int64_t ld, double *dx, double *dtheta,
                                double *dhdiag, double *dcore, void *stream);

/* Angles of every rotation into the DEVICE array theta, rotations in the
 * order above.  k = 2: theta[rotations], theta = atan2(s, c).  k >= 3 (the
 * angle parameterisation of a k-point block, not in the paper): P = k(k-1)/2
 * slots per rotation, the Givens elimination of the kk x kk block column by
 * column (j = 0..kk-2, l = j+1..kk-1; theta = atan2(A_lj, A_jj), rows (j, l)
 * <- (c row j + s row l, -s row j + c row l)), which leaves signs D =
 * diag(+-1) with O = G_1^T .. G_P^T D; slots beyond kk(kk-1)/2 are 0.  The
 * signs are formed on the first call (of this function, pmmf_set_angles or
 * pmmf_block_angle_grad) and kept in the handle.  UNSUPPORTED for a batch. */
pmmf_status pmmf_get_angles(const pmmf_handle *f, double *theta, void *stream);

/* Replace every rotation from the DEVICE array theta (layout above): k = 2
 * (cos theta, sin theta); k >= 3 O = G_1^T .. G_P^T D with the kept signs.
 * The selections (tuples, levels, eliminations) are kept; pmmf_get_info's
 * error still describes the factorization as computed. */
pmmf_status pmmf_set_angles(pmmf_handle *f, const double *theta, void *stream);

/* k >= 3: dL/dtheta[rotations * k(k-1)/2] (layout of pmmf_get_angles) from
 * dL/dO[rotations * k * k] (the output of pmmf_apply_backward) at the
 * handle's current blocks, by the chain rule through O = G_1^T .. G_P^T D
 * (D fixed).  DEVICE arrays.  UNSUPPORTED for k = 2 (the backward returns
 * angle gradients directly) and for a batch. */
pmmf_status pmmf_block_angle_grad(const pmmf_handle *f, const double *dO, double *dtheta,
                                  void *stream);

/* Replace H: hdiag[n] (its core entries are not used) and/or
 * core[core_size^2], DEVICE arrays, either may be NULL.  The cached core
 * inverse is dropped and formed again on the next inverse request. */
pmmf_status pmmf_set_h(pmmf_handle *f, const double *hdiag, const double *core, void *stream);

/* ---- one stage's steps as separate calls (a stage split over GPUs) --------
 * Sec. 2.3 runs the clusters' searches independently and the blocked update
 * block by block, redistributing the matrix between stages.  These calls are
 * the steps of pmmf_factor's stage (same kernels, same bits) for a caller that
 * spreads the clusters of every stage over several GPUs and moves rows and
 * rotations between them itself (paper_1507_04396_gb300/shard.py does, over
 * torch.distributed).  All arrays are DEVICE memory unless marked HOST; ids
 * are global coordinate ids; stage is 1-based (it enters the random draws).
 *
 * pmmf_shard_create: per-factorization state: the parameters (pmmf_params as
 *   for pmmf_factor; coords and labels copied), the quantized points.
 * pmmf_shard_clusters: stage's clusters of the active set act[s] (ascending)
 *   and their rotation counts (Algorithm 1 "cluster", the schedule):
 *   *m (HOST), coff[m + 1] (capacity s + 1), members[s], e[m] (capacity s).
 * pmmf_shard_search: Algorithm 2 for the clusters own[nown] (ascending
 *   ordinals of coff / members): rowptr/col/val is a CSR over the whole active
 *   set in act order in which at least these clusters' members' rows are
 *   filled (the others may be empty); outputs, the owned clusters' rotations
 *   in order (sum of e over own entries): cluster ordinal, tuple size, tuple
 *   (k slots, -1 unused), block (k * k slots), eliminated id.
 * pmmf_shard_transform: out = R Q^T for the rows R (ids[nrows], CSR) with the
 *   rotations of every cluster of the stage (in the layout of
 *   pmmf_shard_search's outputs, ordered by cluster ordinal), exact zeros
 *   dropped, columns ascending.  account != 0 adds the stage's accounting: an
 *   eliminated row writes hdiag[id] (its diagonal) and adds its other
 *   entries' squares to contrib[0]; an entry at an eliminated column adds its
 *   square and is dropped; only the surviving rows are kept.  *out_rows and
 *   *out_nnz (HOST) receive the result's size; pmmf_shard_result copies it
 *   (ids[out_rows], rowptr[out_rows + 1], col / val[out_nnz], any may be
 *   NULL) into caller buffers, until the next transform.
 * pmmf_shard_sumsq: the sum of squares of val[nnz] into *out (HOST), for the
 *   norm ||A||_F of the relative error; synchronizes the stream.
 * Errors: INVALID_ARG, OOM, CUDA, UNSUPPORTED (a cluster or row too large for
 * the kernels), NOT_CONVERGED (a k x k Jacobi). */
typedef struct pmmf_shard pmmf_shard;
pmmf_status pmmf_shard_create(int64_t n, const pmmf_params *p, pmmf_shard **out, void *stream);
pmmf_status pmmf_shard_clusters(pmmf_shard *sh, int64_t stage, int64_t s, const int32_t *act,
                                int64_t *m, int64_t *coff, int32_t *members, int64_t *e,
                                void *stream);
pmmf_status pmmf_shard_search(pmmf_shard *sh, int64_t stage, int64_t s, const int32_t *act,
                              const int64_t *rowptr, const int32_t *col, const double *val,
                              int64_t m, const int64_t *coff, const int32_t *members,
                              const int64_t *e, int64_t nown, const int32_t *own,
                              int32_t *rcluster, int32_t *rkk, int32_t *ridx, double *rO,
                              int32_t *relim, void *stream);
pmmf_status pmmf_shard_transform(pmmf_shard *sh, int64_t stage, int account, int64_t nrows,
                                 const int32_t *ids, const int64_t *rowptr, const int32_t *col,
                                 const double *val, int64_t s, int64_t m, const int64_t *coff,
                                 const int32_t *members, int64_t nrot, const int32_t *rcluster,
                                 const int32_t *rkk, const int32_t *ridx, const double *rO,
                                 const int32_t *relim, double *hdiag, double *contrib,
                                 int64_t *out_rows, int64_t *out_nnz, void *stream);
pmmf_status pmmf_shard_result(const pmmf_shard *sh, int32_t *ids, int64_t *rowptr, int32_t *col,
                              double *val, void *stream);
pmmf_status pmmf_shard_sumsq(const double *val, int64_t nnz, double *out, void *stream);
void pmmf_shard_free(pmmf_shard *sh);

/* Release a handle (NULL-safe). */
void pmmf_free(pmmf_handle *f);

/* Message of the last failed call on this thread ("" if none). */
const char *pmmf_last_error(void);

/* ---- inspection (copies into HOST buffers; synchronous) ------------------ */

pmmf_status pmmf_get_info(const pmmf_handle *f, pmmf_info *info);
pmmf_status pmmf_get_stage_info(const pmmf_handle *f, int p, pmmf_stage_info *info);

/* Clustering of stage p (0-based): offsets[clusters + 1] into members[active];
 * each cluster's members are global ids in ascending order. */
pmmf_status pmmf_get_stage_clusters(const pmmf_handle *f, int p, int64_t *offsets,
                                    int32_t *members);

/* Rotations of stage p in (cluster, step) order, the order Algorithm 2 finds
 * them: cluster[r], kk[r] (tuple size), idx[r*k + a] global ids of the tuple
 * (i first, then partners by decreasing score; unused slots -1),
 * O[r*k*k + a*kk + b] the kk x kk block acting as x_T' = O x_T (for kk = 2:
 * [[c, -s], [s, c]]), elim[r] the eliminated global id. */
pmmf_status pmmf_get_stage_rotations(const pmmf_handle *f, int p, int32_t *cluster, int32_t *kk,
                                     int32_t *idx, double *O, int32_t *elim);

/* H (core-diagonal, Sec. 2): hdiag[n] is the diagonal of H (core diagonal
 * included), core_idx[core_size] the ascending global ids of S_L and
 * core[core_size^2] the dense core block H[S_L, S_L] row-major. */
pmmf_status pmmf_get_h(const pmmf_handle *f, double *hdiag, int32_t *core_idx, double *core);

/* Recorded A_p[S_p, S_p] of stage p (params.record_stages != 0) as CSR over
 * global ids: rowptr_n1[n + 1] (rows outside S_p empty), col[nnz], val[nnz].
 * Pass NULL arrays to query nnz only. */
pmmf_status pmmf_get_stage_matrix(const pmmf_handle *f, int p, int64_t *rowptr_n1, int32_t *col,
                                  double *val, int64_t *nnz);

/* ---- launch tuning (no counterpart in the paper) ---------------------------
 * Launch shapes an offline sweep may choose per cluster-size bucket
 * (paper_1507_04396_gb300/autotune.py writes them to a JSON file that the
 * Python binding applies at load time).  param: PMMF_TUNE_ROWS_WARPS (warps
 * per block of the blocked-update row kernel, 1..8), PMMF_TUNE_GRAM_WARPS
 * (warps per block of the Gram kernel, 1..8), PMMF_TUNE_SELECT_WARPS (warps
 * per cluster of the k = 2 rotation search, 8 or 16; without a setting the
 * search uses 8; clusters above 512 coordinates always use 16),
 * PMMF_TUNE_PASS1_ESTIMATE (the first stage allocates the blocked update's
 * intermediate for this many times the input's entries, 1..32, default 8;
 * later stages scale the previous stage's size; a short estimate costs a
 * second pass, never a wrong result; use max_size 1), PMMF_TUNE_REACH_CLUSTERS
 * (the blocked update's counting passes take each row segment's fill pattern
 * from per-cluster reach sets when the stage has at least this many clusters,
 * default 64, else they run the rotation levels on the pattern; both give the
 * same counts; 1..2^31-1, use max_size 1), PMMF_TUNE_ROWS_KERNEL (the blocked
 * update's kernel: 1 = one warp per row running every rotation level of the
 * segment's cluster (the default), 2 = one thread per row, applying to each
 * row segment only the rotations that reach its pattern (clusters of up to
 * 1,024 coordinates); both give the same bits), PMMF_TUNE_DENSE_TILES (the
 * dense update: 1 = the block in cluster order moved in TMA tiles, each CTA
 * staging one cluster's rotations (clusters whose tiles do not fit shared
 * memory fall back to 2), 2 = one CTA per row applying every cluster's
 * rotations (the default); both give the same bits), PMMF_TUNE_SELECT_DSM
 * (the k = 2 rotation search: 1 = one CTA per cluster with G and M in
 * global memory (the default), 2 = a thread-block cluster of 8 CTAs per
 * cluster holding G and M in their shared memory, row-sliced, for stages
 * whose clusters have up to ~318 coordinates (larger ones use 1); both give
 * the same bits), PMMF_TUNE_APPLY_FUSED (the rotation passes of the
 * matrix-free apply: 1 = one launch per stage (the default), 2 = one
 * cooperative launch per pass with a grid barrier between stages, where the
 * device supports cooperative launches and the right-hand sides fit one pass
 * (else 1); both give the same bits; max_size is the largest cluster of the
 * factorization), PMMF_TUNE_SELECT_BLOCKS (CTAs of the k = 2 search's
 * 256-thread kernel per SM, 2, 3 or 4, its registers capped to fit; without
 * a setting 4 for clusters of up to 256 coordinates and 3 up to 512 when a
 * stage has at least 4 and 6 times as many clusters as SMs, else 2; all give
 * the same bits), PMMF_TUNE_MIXED_ACTIVE (with a reduced-precision mode, the
 * stages with at least this many clusters use the reduced-precision Gram and
 * shortlist, the others the FP64 Gram and search; 0 = every stage; default
 * 12), PMMF_TUNE_TC_GRAM (the reduced-precision Gram: 2 = tcgen05 MMAs with
 * the accumulators in tensor memory and TMA-loaded operands (the default),
 * 1 = warp-level mma.sync; the same 16-term FP32 chunks and compensated sums,
 * so the same certified bound).
 * A value
 * applies to launches whose largest cluster has at most max_size coordinates
 * and no smaller bucket matches; shared-memory limits still halve the row and
 * Gram warps when needed.  Process wide; INVALID_ARG for an unknown param or
 * a value outside 1..32 (outside {8, 16} for the search warps, {1, 2} for the
 * kernel choices, 2..4 for the search's CTAs per SM, 0..32 for the
 * reduced-precision threshold; any positive value for the reach threshold). */
enum { PMMF_TUNE_ROWS_WARPS = 0, PMMF_TUNE_GRAM_WARPS = 1, PMMF_TUNE_SELECT_WARPS = 2,
       PMMF_TUNE_PASS1_ESTIMATE = 3, PMMF_TUNE_REACH_CLUSTERS = 4, PMMF_TUNE_ROWS_KERNEL = 5,
       PMMF_TUNE_DENSE_TILES = 6, PMMF_TUNE_SELECT_DSM = 7,
       PMMF_TUNE_APPLY_FUSED = 8, PMMF_TUNE_SELECT_BLOCKS = 9, PMMF_TUNE_MIXED_ACTIVE = 10,
       PMMF_TUNE_TC_GRAM = 11 };
pmmf_status pmmf_set_tuning(int param, int64_t max_size, int value);
void pmmf_clear_tuning(void);

/* Number of GPU kernel launches this process has issued through the library. */
uint64_t pmmf_launch_count(void);

/* Number of device allocations this process has requested through the
 * library (every device buffer it owns, transient or kept, is one request).
 * A diagnostic with no counterpart in the paper: a caller can check that a
 * call it expects to be allocation-free (pmmf_apply_noalloc) made none. */
uint64_t pmmf_alloc_count(void);

/* FP64 FMA throughput of the current device in TFLOP/s (HOST output), the
 * denominator of the roofline fraction of the FP64-bound kernels.  A
 * measurement aid with no counterpart in the paper: every SM runs 8 CTAs of
 * 256 threads, each thread 8 independent chains of 4,096 dependent fmas;
 * the best of three timed launches (CUDA events on stream, after one
 * warm-up launch) counts 2 flops per fma.  Synchronizes the stream. */
pmmf_status pmmf_probe_fp64(double *tflops, void *stream);

/* The reduced-precision Gram matrix of the shortlist search (the tensor-core
 * screen of pattern (1) on the local Grams of Sec. 2.1) for one set of rows,
 * a diagnostic that exposes the kernel the factorization uses: X is a HOST
 * rows x s FP64 row-major matrix (1 <= rows <= 4096, 1 <= s <= 2^24), G a HOST
 * rows x rows FP32 output (row-major, symmetric) receiving
 * G~ = hi hi^T + hi lo^T + lo hi^T for the split x = hi + lo of every entry
 * (precision PMMF_PREC_TF32: hi, lo TF32, rounded to nearest with ties away;
 * PMMF_PREC_BF16: BF16, to nearest even), summed in FP32 chunks of 16 terms
 * that are added into compensated FP32 sums; the kernel follows
 * PMMF_TUNE_TC_GRAM.  |G~_ij - (X X^T)_ij| stays within the shortlist's
 * certified bound eps sqrt(G_ii G_jj).  INVALID_ARG for NULL buffers, sizes
 * out of range or precision PMMF_PREC_FP64; TIMEOUT if a bounded wait of the
 * tensor-core pipeline ran out.  The caller owns both buffers; synchronizes
 * the stream. */
pmmf_status pmmf_gram_reduced(const double *X, int64_t rows, int64_t s, int precision, float *G,
                              void *stream);

/* ---- profiling (measurement aid; no counterpart in the paper) -------------
 * Kernel families: 0 partition (k-means assignment), 1 Gram, 2 rotation
 * search, 3 blocked-update row kernels, 4 matrix-free apply, 5 other.
 * pmmf_profile_begin(mask) brackets every later launch of the families in mask
 * with two CUDA events recorded on that launch's stream, together with the
 * launch's algorithmic bytes and flops (compulsory traffic and arithmetic, as
 * documented at each launch site).  pmmf_profile_end synchronizes the device
 * and fills ms[6], launches[6], bytes[6], flops[6] (host arrays, one slot per
 * family), then disables profiling. */
pmmf_status pmmf_profile_begin(unsigned family_mask);
pmmf_status pmmf_profile_end(double *ms, int64_t *launches, double *bytes, double *flops);
/* The launches recorded since pmmf_profile_begin, one by one in launch order
 * (HOST arrays of cap entries; cap may be 0 to query the count): family,
 * duration (ms), algorithmic bytes and flops.  Synchronizes the device; the
 * records stay until pmmf_profile_end or the next pmmf_profile_begin. */
pmmf_status pmmf_profile_records(int64_t cap, int32_t *family, double *ms, double *bytes,
                                 double *flops, int64_t *count);

#ifdef __cplusplus
}
#endif
#endif
