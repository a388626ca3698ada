/*
 * dtwgb_proposal.h -- k-medoids over exact DTW with learned proposals.
 *
 * The paper's k-medoids (Mathematical background, last paragraph) needs only
 * some DTW distances ("it does not compute all DTW distances", Performance
 * comparison); these entry points compute exactly those, on the GPU, and take
 * their proposals from embeddings (dtwgb_encoder.h) whose distances follow DTW:
 *
 *   proposal_kmeanspp   initial medoids by k-means++ seeding (Arthur &
 *                       Vassilvitskii 2007) in embedding space;
 *   kmedoids_lazy_fit   alternate k-medoids (the rules of kmedoids_fit) whose
 *                       assignment computes DTW(medoid, point) for every point
 *                       and whose update evaluates, per cluster, only
 *                       `candidates` proposals -- the current medoid and the
 *                       members nearest to the cluster's embedding centroid --
 *                       by their exact DTW sums over the cluster's members.
 *                       With candidates <= 0 (or emb == NULL) every member is a
 *                       candidate and the sweeps are exactly those of
 *                       kmedoids_fit on the full matrix D.
 * Every accepted assignment, medoid and cost is an exact DTW value.
 */
#ifndef DTWGB_PROPOSAL_H
#define DTWGB_PROPOSAL_H

#include <stdint.h>

#include "dtwgb.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * k distinct medoids from embeddings emb [n][dim] (device float32): the first
 * is index splitmix64(seed) mod n, each next one is drawn with probability
 * proportional to the squared embedding distance to the nearest chosen one,
 * using uniforms u_i = (splitmix64 output >> 11) * 2^-53 of the same stream.
 * out_medoids: int32 [k] device.  Asynchronous.  Errors: DTW_EINVAL for n < 1,
 * k outside [1, n], dim < 1, NULL pointers.
 */
int proposal_kmeanspp(const float *emb, int32_t n, int32_t dim, int32_t k, uint64_t seed,
                      int32_t *out_medoids, void *stream);

/*
 * Lazy alternate k-medoids over the set (values, offsets, n series; band as
 * dtw_pairwise with `window` and `flags`).
 *
 *   emb           float32 [n][dim] device embeddings, or NULL
 *   candidates    proposals per cluster and sweep (current medoid included);
 *                 <= 0: all members
 *   init_medoids  int32 [k] device, distinct, in [0, n)
 *   out_medoids   int32 [k] device; out_labels int32 [n] device
 *   out_cost      HOST double: sum_j DTW(j, M_{label_j}) in float64; may be NULL
 *   out_iters     HOST int32: update sweeps performed; may be NULL
 *   out_pairs     HOST int64: DTW pairs evaluated in total; may be NULL
 *
 * Synchronous (reads cluster sizes and a convergence flag every sweep).
 * Errors: as kmedoids_fit, plus DTW_EINVAL for emb != NULL with dim outside
 * [1, 1024], and the errors of dtw_pairs for the set.
 */
int kmedoids_lazy_fit(const float *values, const int64_t *offsets, int32_t n, int32_t window,
                      uint32_t flags, const float *emb, int32_t dim, int32_t k,
                      const int32_t *init_medoids, int32_t candidates, int32_t max_iter,
                      int32_t *out_medoids, int32_t *out_labels, double *out_cost,
                      int32_t *out_iters, int64_t *out_pairs, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* DTWGB_PROPOSAL_H */
