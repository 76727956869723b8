/* Flat "GMM J=n" variant of HGMM registration (Sec. 5, variant 3).
 *
 * The ablation that removes the tree: a single-level GMM of J components,
 * every point associated with every component (Eq. 3 over all J, O(NJ) per
 * round instead of Algorithm 1's logarithmic descent), and the same PCA
 * M-step (Eq. 8-16) and pose update as the tree.
 *
 * The paper does not say how the J components are obtained.  Here they come
 * from a built GMM tree (hgmm.h): the leaves of the tree cut at a level (every
 * live node of that level and every live node of a shallower level without a
 * live child), each weighted by the product of the within-parent mixing
 * weights on its path, normalised to one; hgmm_flat_fit then optionally
 * refines them by plain EM over all J components.
 *
 * Conventions are those of hgmm.h: device pointers (d_*) are device memory
 * of the current device, points are n x float4 (x, y, z, ignored), poses
 * 4x4 row-major float64; calls are asynchronous on `stream` (NULL = legacy
 * default stream) unless marked synchronous; every function returns HGMM_OK
 * or a negative HGMM_E* code; device-side problems (non-finite input,
 * singular normal equations) are reported by hgmm_flat_sync.
 */
#ifndef HGMM_FLAT_H
#define HGMM_FLAT_H

#include <stdint.h>

#include "hgmm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hgmm_flat hgmm_flat;

/* A flat model for clouds of up to max_points points and up to
 * max_components components, on the current device; owns all of its
 * scratch (no allocation after this call).  Errors: HGMM_EINVAL,
 * HGMM_ENOMEM. */
int hgmm_flat_create(int64_t max_points, int32_t max_components, hgmm_flat** out);
void hgmm_flat_destroy(hgmm_flat* f);

/* Components from the last build of tree t, cut at `level` (0-based;
 * -1 = the tree's deepest level): the live nodes of that level and the live
 * nodes of shallower levels that have no live child, ordered by level then
 * by index; pi_j = product of the within-parent weights pi along the node's
 * path, normalised to sum to one; mu_j, Sigma_j and the eigen-decomposition
 * as in the tree; eps (the covariance floor) is the tree's.  Errors:
 * HGMM_EINVAL (no build, level out of range), HGMM_ECAPACITY (the tree cut
 * has more nodes than max_components). */
int hgmm_flat_from_tree(hgmm_flat* f, const hgmm_tree* t, int32_t level, void* stream);

/* em_iters iterations of EM over all components on d_points (n points):
 * Eq. 3 posteriors of every point over all J, then pi_j = S0_j / n,
 * mu_j = S1_j / S0_j, Sigma_j = S2_j / S0_j - mu_j mu_j^T + eps I; a
 * component below n_min expected points dies (it keeps its parameters and
 * gets weight 0).  FP32 E-step with compensated moment sums, FP64 M-step and
 * eigen-decomposition.  em_iters = 0 is valid (no change).  Errors:
 * HGMM_EINVAL (no components yet, n < 1, unaligned pointer),
 * HGMM_ECAPACITY (n > max_points). */
int hgmm_flat_fit(hgmm_flat* f, const float* d_points, int64_t n, int32_t em_iters, float n_min,
                  void* stream);

/* EM registration of source d_src (n points) to the flat model (Eq. 1):
 * `iters` rounds of z' = R z + t, Eq. 3 posteriors over all components,
 * M0_j = sum_i gamma_ij and M1_j = sum_i gamma_ij z'_i (Eq. 8), the Eq. 9-16
 * normal equations in FP64 (eigenvalues floored at eps) and T <- dT T.
 * d_T_init: 16 float64 (NULL = identity); d_T_out: 16 float64 or NULL;
 * d_T_hist: iters x 16 float64 (the pose after every round) or NULL.
 * Errors: HGMM_EINVAL, HGMM_ECAPACITY. */
int hgmm_flat_register(hgmm_flat* f, const float* d_src, int64_t n, const double* d_T_init,
                       int32_t iters, void* stream, double* d_T_out, double* d_T_hist);

/* The Eq. 11 objective of the last round of the last registration,
 * sum_j pi*_j (mu_j - mu*_j)^T P_j (mu_j - mu*_j) at the pose that round
 * started from (1 float64 to d_obj). */
int hgmm_flat_objective(const hgmm_flat* f, double* d_obj, void* stream);

/* Synchronous.  *h_count = J; then min(J, cap) components of 10 float64 each
 * to h_out: pi, mu (3), Sigma upper (xx xy xz yy yz zz); and, if h_node is
 * not NULL, 2 int32 per component: the tree level and the index within that
 * level of the node it was made from. */
int hgmm_flat_export(hgmm_flat* f, double* h_out, int64_t cap, int32_t* h_count, int32_t* h_node);

/* Synchronous.  Moments of the last round of the last registration, 4
 * float64 per component (M0, M1 x, y, z; M1 as sum gamma z'), min(J, cap)
 * components; *h_count = J. */
int hgmm_flat_debug_moments(hgmm_flat* f, double* h_out, int64_t cap, int32_t* h_count);

/* Synchronise `stream` and return the first device-side error recorded
 * since the last call (HGMM_ENONFINITE, HGMM_EDEGENERATE) or HGMM_OK; clears
 * it. */
int hgmm_flat_sync(hgmm_flat* f, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* HGMM_FLAT_H */
