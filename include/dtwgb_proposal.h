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
 *   proposal_kmeans     initial medoids from Lloyd's k-means in embedding
 *                       space (restarts from k-means++ seedings): the member
 *                       nearest to each centroid of the best restart;
 *   kmedoids_lazy_fit   alternate k-medoids (the rules of kmedoids_fit) whose
 *                       assignment computes DTW(medoid, point) for every point
 *                       and whose update evaluates, per cluster, only a short
 *                       candidate list -- the current medoid, the members
 *                       nearest to the cluster's embedding centroid, and the
 *                       members of least DTW sum to a sample of the cluster --
 *                       by their exact DTW sums over the cluster's members.
 *                       Without proposals every member is a candidate and the
 *                       sweeps are exactly those of kmedoids_fit on the full
 *                       matrix D.
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
 * out_medoids: int32 [k] device.  If every remaining squared distance is zero
 * the smallest index not chosen yet is taken.  Asynchronous.  Errors:
 * DTW_EINVAL for n < 1, k outside [1, n], dim < 1, NULL pointers.
 */
int proposal_kmeanspp(const float *emb, int32_t n, int32_t dim, int32_t k, uint64_t seed,
                      int32_t *out_medoids, void *stream);

/*
 * k distinct medoid proposals from Lloyd's k-means over emb [n][dim]:
 * restart r (0 <= r < restarts) starts from the k-means++ centres of seed
 * seed + r and alternates assignment (squared Euclidean distance, ties to the
 * smaller centre) and centroid update (an empty cluster keeps its centroid)
 * for at most `iters` assignments, stopping early when no label changes.  The
 * restart of least inertia (sum of squared distances to the final centroids,
 * float64; the first on ties) is kept; the proposal of each of its clusters is
 * the member nearest to the centroid (ties to the smaller index); an empty
 * cluster takes the nearest point not taken by another cluster.
 *   out_medoids   int32 [k] device
 *   out_inertia   HOST double, the kept restart's inertia; may be NULL
 * Synchronous (reads a label-change flag per assignment).  Errors: DTW_EINVAL
 * for n < 1, dim outside [1, 1024], k outside [1, n], restarts < 1, iters < 0,
 * NULL pointers.
 */
int proposal_kmeans(const float *emb, int32_t n, int32_t dim, int32_t k, int32_t restarts,
                    int32_t iters, uint64_t seed, int32_t *out_medoids, double *out_inertia,
                    void *stream);

/*
 * Lazy alternate k-medoids over the set (values, offsets, n series; band as
 * dtw_pairwise with `window` and `flags`).  Each sweep: assignment as
 * kmedoids_fit (k*n DTW pairs); then, per cluster c with members C_c in index
 * order, the candidate list
 *   base      the current medoid, then (with emb != NULL and candidates > 1)
 *             the min(candidates, |C_c|) - 1 other members nearest to the
 *             centroid of the members' embeddings, by (squared distance,
 *             index);
 *   screened  (screen_sample > 0) with s = min(screen_sample, |C_c|) and the
 *             sample Q = { C_c[floor(q |C_c| / s)] : q < s }, every member i is
 *             scored sum_{j in Q} DTW(i, j) (float64, j in order) and the
 *             min(screen_keep, |C_c|) members of least score (ties to the
 *             smaller index) are appended, repeats of base members included;
 * and the new medoid is the candidate of least exact DTW sum over C_c, a tie
 * keeping the current medoid, else going to the smaller index.  With
 * candidates <= 0 (or emb == NULL) and screen_sample == 0 every member is a
 * candidate: the sweeps of kmedoids_fit.  Sweeps stop when no medoid moves.
 *
 *   emb           float32 [n][dim] device embeddings, or NULL
 *   candidates    base list length (current medoid included); <= 0: see above
 *   screen_sample sampled members per cluster, 0 <= screen_sample <= 4096
 *   screen_keep   screened members kept, >= 1 when screen_sample > 0
 *   init_medoids  int32 [k] device, distinct, in [0, n)
 *   out_medoids   int32 [k] device; out_labels int32 [n] device
 *   out_cost      HOST double: sum_j DTW(j, M_{label_j}) in float64; may be NULL
 *   out_iters     HOST int32: update sweeps performed; may be NULL
 *   out_pairs     HOST int64: DTW pairs evaluated in total; may be NULL
 *
 * Synchronous (reads cluster sizes and a convergence flag every sweep).
 * Errors: as kmedoids_fit, plus DTW_EINVAL for emb != NULL with dim outside
 * [1, 1024] or screening arguments out of range, and the errors of dtw_pairs
 * for the set.
 */
int kmedoids_lazy_fit(const float *values, const int64_t *offsets, int32_t n, int32_t window,
                      uint32_t flags, const float *emb, int32_t dim, int32_t k,
                      const int32_t *init_medoids, int32_t candidates, int32_t screen_sample,
                      int32_t screen_keep, int32_t max_iter, int32_t *out_medoids,
                      int32_t *out_labels, double *out_cost, int32_t *out_iters,
                      int64_t *out_pairs, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* DTWGB_PROPOSAL_H */
