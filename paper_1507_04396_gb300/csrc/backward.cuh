// backward.cuh -- gradient of the factorized operator (internal).
#pragma once

#include <vector>

#include "apply.cuh"

namespace pmmf {

// dL/dx, dL/dtheta (per rotation, stages in order, (cluster, step) order
// inside; for k-point rotations dL/dO, K*K slots per rotation), dL/d(diagonal
// of H) (0 on core coordinates) and dL/dcore for L = sum(g * U^T M U x),
// M = H or H^{-1}.  Outputs are overwritten; any may be NULL.  recs[p] =
// stage p's step-order rotation records (k = 2), klvls[p] = its rotations'
// levels (k >= 3).
pmmf_status apply_backward(const ApplyStages &S, const std::vector<const RotRec *> &recs,
                           const std::vector<const int32_t *> &klvls, const HData &H,
                           bool inverse, const double *x, const double *g, int64_t nrhs,
                           int64_t ld, double *dx, double *dtheta, double *dhdiag, double *dcore,
                           cudaStream_t st);

// k-point blocks (K*K slots each, kk x kk used) <-> Givens angles (P = K(K-1)/2
// slots per rotation) and signs D (K slots), and dL/dO -> dL/dtheta at theta.
// D may be NULL in block_angles.
pmmf_status block_angles(int64_t nrot, int K, const int32_t *kkv, const double *kO,
                         double *theta, double *D, cudaStream_t st);
pmmf_status block_from_angles(int64_t nrot, int K, const int32_t *kkv, const double *theta,
                              const double *D, double *kO, cudaStream_t st);
pmmf_status block_angle_grad(int64_t nrot, int K, const int32_t *kkv, const double *theta,
                             const double *D, const double *dO, double *dtheta, cudaStream_t st);

// theta[t] = atan2(s_t, c_t) for one stage's records.
pmmf_status get_angles(const RotRec *rec, int64_t nrot, double *theta, cudaStream_t st);

// (c_t, s_t) = (cos theta_t, sin theta_t) in one stage's records and the
// level-grouped copies.
pmmf_status set_angles(const ApplyStage &a, RotRec *rec, Rot2 *lvlrot, const double *theta,
                       cudaStream_t st);

}  // namespace pmmf
