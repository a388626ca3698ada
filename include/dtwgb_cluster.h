/*
 * dtwgb_cluster.h -- cluster-quality reporting over the DTW matrix D.
 *
 * The paper's software reports "the silhouette score and elbow score for the
 * clusters in order to aid the user decision on how many clusters, k, to
 * include" (Overview, item 6) without defining them.  This library reads the
 * silhouette as Rousseeuw's (1987) definition over the same distances the
 * clustering uses (the DTW costs in D, no square root):
 *
 *   a(i) = sum_{j in C(i), j != i} D[i][j] / (|C(i)| - 1)
 *   b(i) = min over clusters C' != C(i), C' non-empty, of sum_{j in C'} D[i][j] / |C'|
 *   s(i) = (b(i) - a(i)) / max(a(i), b(i)),   s(i) = 0 if |C(i)| = 1 or max = 0
 *
 * and the silhouette score as the mean of s(i).  The elbow curve is the
 * k-medoids cost as a function of k (repeated kmedoids_fit calls; see the
 * Python helper paper_2307_04904_gb300.quality.elbow).
 *
 * kmedoids_pam refines (or builds) medoids with PAM's swap search (Kaufman &
 * Rousseeuw 1990), another reading of the paper's unspecified k-medoids: one
 * swap at a time, the one that lowers the total deviation most.
 *
 * All pointers are device pointers owned by the caller unless marked host.
 */
#ifndef DTWGB_CLUSTER_H
#define DTWGB_CLUSTER_H

#include <stdint.h>

#include "dtwgb.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Silhouette of a clustering: D float32 [n][n] (symmetric, zero diagonal, as
 * dtw_pairwise writes it), labels int32 [n] in [0, k).
 *   out_s     float32 [n] device, s(i); may be NULL
 *   out_mean  HOST double, the mean of s(i) (float64 sums in a fixed order)
 * Cluster sums are Kahan-compensated float32 (float64 in the fallback for
 * n * k > 2^26), taken over each cluster's members in index order, so the
 * result is deterministic.  Synchronous.  Errors: DTW_EINVAL for n < 2,
 * k < 2 or k > 4096, a label outside [0, k), fewer than two non-empty
 * clusters, NULL D or out_mean.
 */
int kmedoids_silhouette(const float *D, int32_t n, const int32_t *labels, int32_t k,
                        float *out_s, double *out_mean, void *stream);

/*
 * PAM on D float32 [n][n].  With init_medoids == NULL, BUILD: the first
 * medoid has the least row sum, each next one lowers TD = sum_j min_c
 * D[M_c][j] the most (ties to the smaller index).  Then SWAP passes: for every
 * non-medoid o and medoid i the change delta(o, i) of TD when o replaces
 * medoid i, all k at once in one pass over the points from the nearest and
 * second-nearest medoid distances (Schubert & Rousseeuw 2019, FastPAM1),
 * Kahan-compensated float32 sums over each cluster's members in index order
 * (relative error about 1e-7 of the summed magnitudes); the least delta
 * (ties: smaller o, then smaller i) is applied while it is negative, at most
 * max_swaps times.
 *   init_medoids  int32 [k] device, distinct, in [0, n); or NULL
 *   out_medoids   int32 [k] device; out_labels int32 [n] device (nearest medoid,
 *                 ties to the smaller position, a medoid labels itself)
 *   out_cost      HOST double TD; out_swaps HOST int32 swaps applied (may be NULL)
 * Synchronous.  Each pass reads D once (n^2 floats).  Errors: DTW_EINVAL for
 * n < 1, k outside [1, min(n, 64)], max_swaps < 0, invalid init, NULL pointers.
 */
int kmedoids_pam(const float *D, int32_t n, int32_t k, const int32_t *init_medoids,
                 int32_t max_swaps, int32_t *out_medoids, int32_t *out_labels, double *out_cost,
                 int32_t *out_swaps, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* DTWGB_CLUSTER_H */
