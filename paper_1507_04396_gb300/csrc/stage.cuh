// stage.cuh -- per-stage data passed between the kernels of one pMMF stage
// (internal to the library).
#pragma once

#include "common.cuh"

namespace pmmf {

struct PartitionIn {
    int64_t n = 0, s = 0;
    int dim = 0;
    const int32_t *q = nullptr;       // n x dim quantized points (null: one cluster)
    const int32_t *morder = nullptr;  // n global ids in Morton order
    const int32_t *pos = nullptr;     // n: row of a global id in the active list, -1 if inactive
    const int32_t *act = nullptr;     // s active global ids, ascending
    int32_t *cl = nullptr;            // n: cluster ordinal of a global id (output)
    int32_t *loc = nullptr;           // n: index inside its cluster (output)
};

struct StageClusters {
    int64_t m = 0;            // clusters (an upper bound while count_d is set)
    DBuf<int64_t> coff;       // m + 1
    DBuf<int32_t> members;    // s, cluster by cluster, ascending global id
    DBuf<int64_t> count_d;    // exact cluster count on the device (k-means),
                              // read with the stage schedule
};

// A CSR block over the active rows: row r is global id act[r].
struct Csr {
    int64_t rows = 0, nnz = 0;    // nnz: entries allocated (>= rowptr[rows])
    bool nnz_exact = true;        // false: the count is rowptr[rows] on the device
    DBuf<int64_t> rowptr;
    DBuf<int32_t> col;        // global ids
    DBuf<double> val;
};

// Rotations of one stage, in the two orders the kernels need.
struct StageRotations {
    int64_t nrot = 0;
    int32_t max_levels = 0;
    int K = 2;                // rotation order k
    DBuf<int64_t> roff;       // m + 1: cluster u owns [roff[u], roff[u+1])
    DBuf<int32_t> lvl_off;    // cluster u: entries [roff[u] + u, roff[u] + u + nlev_u + 1)
    DBuf<int32_t> nlev;       // m
    // k = 2
    DBuf<RotRec> rec;         // step order (export)
    DBuf<Rot2> lvl;           // grouped by dependency level inside each cluster
    // k >= 3, step order: tuple (local indices, K slots, -1 unused), kk x kk
    // block (K*K slots, stride kk inside), tuple size, eliminated local index,
    // level; lvlidx = the step-order rotation at each level-grouped slot
    DBuf<int32_t> kidx, kk, kel, klvl, lvlidx;
    DBuf<double> kO;
    DBuf<double> kD;          // k >= 3: the blocks' Givens signs (K per rotation), once formed
    bool kD_ready = false;
};

pmmf_status quantize_points(const double *coords, int64_t n, int dim, int32_t *q, uint64_t *code,
                            unsigned *status, cudaStream_t st);
pmmf_status partition_stage(const PartitionIn &in, int64_t m, int iters, StageClusters &out,
                            cudaStream_t st);
pmmf_status one_cluster(const int32_t *act, int64_t s, StageClusters &out, int32_t *cl,
                        int32_t *loc, cudaStream_t st);
// Given clusters (labels[x] in [0, m) for every coordinate x): the nonempty
// labels in ascending order, members ascending.  check_labels sets
// ST_BAD_LABEL for a label outside [0, m).
pmmf_status check_labels(const int32_t *labels, int64_t n, int64_t m, unsigned *status,
                         cudaStream_t st);
pmmf_status partition_from_labels(const PartitionIn &in, const int32_t *labels, int64_t m,
                                  StageClusters &out, cudaStream_t st);
// host_out[5]: total rotations, one-cluster fallback flag, largest cluster,
// sum of squared cluster sizes (the two last for the fallback's one cluster
// when the flag is set), number of clusters.  mm_dev (may be NULL): the exact
// cluster count on the device, mm then an upper bound.
pmmf_status schedule_stage(const int64_t *coff, int64_t mm, const int64_t *mm_dev, int64_t s,
                           int64_t core, double eta, DBuf<int64_t> &e, DBuf<int64_t> &roff,
                           int64_t *host_out, cudaStream_t st);
// The same in two halves: schedule_launch enqueues the kernel on st (its
// results go to the host mailbox's MB_SCHED slots); schedule_read copies them
// out once the host has waited for st (or an event recorded after the launch).
pmmf_status schedule_launch(const int64_t *coff, int64_t mm, const int64_t *mm_dev, int64_t s,
                            int64_t core, double eta, DBuf<int64_t> &e, DBuf<int64_t> &roff,
                            cudaStream_t st);
void schedule_read(int64_t *host_out);

// Gram G^u and symmetric local block M^u of every cluster (dense c_u x c_u,
// row-major at goff[u]) and the rotation search of Algorithm 2.
// order (optional): launch position -> cluster, e.g. longest first; useed
// (optional): per-cluster seeds, the draws then use cluster ordinal 0 (each
// cluster searched as if it were the only cluster of its own factorization).
// Dense per-cluster Gram and local blocks: block u (c_u x c_u, row-major) at
// goff[u] of G and M.
struct GramBlocks {
    int64_t total = 0;
    DBuf<int64_t> goff;       // m + 1
    DBuf<double> G, M;
};
// total: sum of c_u^2 when the caller knows it (-1: read it back).
pmmf_status gram_blocks(const StageClusters &cls, GramBlocks &gb, cudaStream_t st,
                        int64_t total = -1);
// Rotation search of every cluster on formed Gram blocks.
// ords (optional): per cluster the ordinal its random draws use (default the
// cluster's own index): a subset of a stage's clusters, renumbered, searched
// exactly as in the whole stage.
pmmf_status select_stage(const StageClusters &cls, int64_t cmax, GramBlocks &gb, uint64_t seed,
                         int64_t stage, StageRotations &rot, int32_t *elimflag, cudaStream_t st,
                         const int32_t *order = nullptr, const uint64_t *useed = nullptr,
                         unsigned *status = nullptr, const int32_t *ords = nullptr);

// rot.K selects Givens (2) or k-point (>= 3) rotations; status receives
// ST_NOT_CONVERGED when a k x k Jacobi did not converge.  nmem (optional): the
// clusters' member count when they cover only part of A's rows (the other
// rows empty, their cl -1); ords as for select_stage.
pmmf_status gram_and_select(const Csr &A, const int32_t *act, const int32_t *pos,
                            const int32_t *cl, const int32_t *loc, const StageClusters &cls,
                            int64_t cmax, uint64_t seed, int64_t stage, StageRotations &rot,
                            int32_t *elimflag, cudaStream_t st, const int32_t *order = nullptr,
                            const uint64_t *useed = nullptr, unsigned *status = nullptr,
                            int64_t gram_total = -1, const int32_t *ords = nullptr,
                            int64_t nmem = -1);
// The k >= 3 search on Gram blocks already formed (selectk.cu).
pmmf_status select_kpoint(const StageClusters &cls, int64_t cmax, const int64_t *goff, double *G,
                          double *M, uint64_t seed, int64_t stage, StageRotations &rot,
                          int32_t *elimflag, cudaStream_t st, const int32_t *order,
                          const uint64_t *useed, unsigned *status, const int32_t *ords = nullptr);

// Blocked update A_p = (A Q^T)^T Q^T, residual accounting, H diagonal and
// compaction to the surviving coordinates.
struct UpdateOut {
    Csr next;                 // A_p[S_p, S_p]
    double *contrib = nullptr;   // device accumulator (added to)
    int64_t w_hint = 0;       // in: estimate of pass 1's output (0: 8 nnz(A))
    int64_t w_nnz = 0;        // out: pass 1's output size (upper bound of V's entries)
};
// The survivors S_p of a stage (one elimination per rotation, so nrot fewer
// than the active rows): flag per active row, their new row numbers (an
// exclusive scan of the flags) and S_p ascending.
struct Survivors {
    DBuf<int32_t> flag, act;
    DBuf<int64_t> newrow;
    int64_t count = 0;
};
pmmf_status survivors_stage(const int32_t *act, int64_t s, int64_t nrot, const int32_t *elimflag,
                            int64_t stage, Survivors &sv, cudaStream_t st);
pmmf_status update_stage(const Csr &A, const int32_t *act, int64_t n, const int32_t *pos,
                         const int32_t *cl, const int32_t *loc, const StageClusters &cls,
                         int64_t cmax, const StageRotations &rot, const int32_t *elimflag,
                         int64_t stage, const Survivors &sv, double *hdiag, double *contrib,
                         UpdateOut &out, unsigned *status, cudaStream_t st,
                         double *contrib_cl = nullptr);

// out = R Q^T for the rows of R (row r is global id ids[r]) with every
// cluster's rotations of a stage, exact zeros dropped, columns ascending (the
// blocked update's second pass on a set of rows).  stage >= 0 adds the
// accounting of that stage's eliminations (elimflag[x] == stage): an
// eliminated row gives hdiag[id] (its diagonal) and adds its other entries'
// squares to *contrib, an entry at an eliminated column adds its square and is
// dropped, and out (rows out_ids) holds the surviving rows only.  stage < 0:
// every row and entry is kept.  Synchronizes st (output sizes).
pmmf_status transform_stage(const Csr &R, const int32_t *ids, const int32_t *cl, const int32_t *loc,
                            const StageClusters &cls, int64_t cmax, const StageRotations &rot,
                            const int32_t *elimflag, int32_t stage, double *hdiag,
                            double *contrib, Csr &out, DBuf<int32_t> &out_ids,
                            unsigned *status, cudaStream_t st);

pmmf_status set_positions(const int32_t *act, int64_t s, int32_t *pos, cudaStream_t st);
pmmf_status extract_core(const Csr &A, const int32_t *pos, int64_t s, double *core, double *hdiag,
                         const int32_t *act, cudaStream_t st);

}  // namespace pmmf
