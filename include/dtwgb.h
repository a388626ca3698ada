/*
 * dtwgb.h -- C ABI of the GB300 (sm_103a) library for all-pairs windowed DTW
 * and k-medoids clustering, after "Fast dynamic time warping and clustering
 * in C++" (arXiv 2307.04904).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Pointers are DEVICE pointers owned by the caller unless a flag or the
 *    argument's comment says "host".  The library never frees them and never
 *    keeps them after the call returns.
 *  - `stream` is a cudaStream_t passed as void*; NULL means the legacy default
 *    stream.  Kernels are enqueued on `stream`.  Where a call has to read data
 *    on the host (offsets, initial medoids, a convergence flag) it
 *    synchronises `stream` and says so below.
 *  - A set of p time series is passed as `values` (all series concatenated,
 *    float32) and `offsets` (int64, p+1 entries, non-decreasing): series i is
 *    values[offsets[i] .. offsets[i+1]).  The paper allows series of
 *    differing lengths (Mathematical background, problem statement).
 *  - Return value: DTW_OK (0) or a negative DTW_E* code.  The message of the
 *    last failure on the calling thread is returned by dtw_last_error().
 *    Argument errors are detected before anything is launched; then no output
 *    is written.
 *
 * What is computed (Mathematical background, the equation for c_{i,j}):
 *     c_{i,j} = (x_i - y_j)^2 + min(c_{i-1,j-1}, c_{i-1,j}, c_{i,j-1})
 * with c_{0,0} = 0 and c_{i,0} = c_{0,j} = +inf; the DTW distance of x
 * (length n) and y (length m) is c_{n,m}, in float32.  No square root is
 * taken.  The Sakoe-Chiba band (Introduction, window example; Overview of
 * method, item 2) admits cell (i,j) iff |i-j| <= w.  window < 0 means no
 * band.  For n != m the band is widened to max(w, |n-m|) so that c_{n,m} is
 * reachable, unless DTW_BAND_STRICT is set, in which case a pair with
 * |n-m| > w gets +INFINITY (not an error).
 */
#ifndef DTWGB_H
#define DTWGB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DTW_OK 0
#define DTW_EINVAL (-1)       /* bad argument (sizes, offsets, medoids, non-finite values) */
#define DTW_ENOMEM (-2)       /* device or host allocation failed */
#define DTW_ECUDA (-3)        /* a CUDA runtime call or kernel launch failed */
#define DTW_ETIMEOUT (-4)     /* a bounded device-side wait gave up */
#define DTW_EUNSUPPORTED (-5) /* valid request the compiled kernels cannot run (e.g. band too wide) */

/* flags for dtw_pairwise / dtw_query */
#define DTW_BAND_STRICT 0x1u      /* keep the band at w for n != m (see above) */
#define DTW_OUT_PACKED_UPPER 0x2u /* dtw_pairwise: out holds p(p-1)/2 values, pair (i<j) in
                                     row-major upper-triangle order, no diagonal */
#define DTW_HOST_IO 0x4u          /* every array argument is HOST memory; the library stages
                                     it through device memory and synchronises `stream` */
#define DTW_CHECK_FINITE 0x8u     /* scan the values first; a NaN or Inf is DTW_EINVAL */
#define DTW_WINDOW_PERMILLE 0x10u /* `window` is per mille of the longer series of each pair:
                                     w = floor(window * max(n, m) / 1000) per pair */
#define DTW_OFFSETS_HOST 0x20u    /* dtw_pairwise / dtw_query: `offsets` is a HOST array (the
                                     other arrays stay device memory), so the call neither
                                     reads offsets back nor synchronises `stream`; the library
                                     copies them to the device on `stream` (an asynchronous
                                     copy: leave the array unchanged until `stream` has
                                     passed the call) */

/* Message of the last failure on this thread ("" if none).  Never NULL. */
const char *dtw_last_error(void);

/* Library version as "major.minor.patch". */
const char *dtw_version(void);

/*
 * dtw_pairwise -- the distance matrix D of the paper (Mathematical
 * background, the paragraph on D): d_{ij} = DTW(series i, series j).
 *
 *   values    float32 [offsets[p]]       the series, concatenated
 *   offsets   int64   [p+1]              non-decreasing; every series non-empty
 *   p         number of series, >= 1
 *   window    w of the band; < 0 = unconstrained
 *   flags     DTW_BAND_STRICT | DTW_OUT_PACKED_UPPER | DTW_HOST_IO | DTW_CHECK_FINITE
 *   out_D     float32 [p*p] row-major, symmetric, zero diagonal; or [p(p-1)/2]
 *             with DTW_OUT_PACKED_UPPER
 *   stream    see above
 *
 * Synchronises `stream` once to read `offsets` on the host (unless
 * DTW_HOST_IO or DTW_OFFSETS_HOST); the DP kernels run asynchronously after
 * that.  Every pair is
 * computed once (i < j) and written to both d_{ij} and d_{ji}: the DP is
 * exactly symmetric in float arithmetic.
 * Bands of up to dtw_max_band_cells() cells per row run on the rotated-band
 * kernels; wider bands (and unconstrained long series) on the column-strip
 * kernel; the cheaper of the two is chosen from the set's lengths and window.
 * Errors: DTW_EINVAL for p < 1, decreasing offsets, an empty series, NULL
 * pointers, or (with DTW_CHECK_FINITE) a non-finite value.
 */
int dtw_pairwise(const float *values, const int64_t *offsets, int32_t p, int32_t window,
                 uint32_t flags, float *out_D, void *stream);

/*
 * dtw_query -- one query against a resident set: one row of D,
 * out[i] = DTW(query, series i).  Same DP, band and flags as dtw_pairwise
 * (DTW_OUT_PACKED_UPPER is ignored).
 *
 *   query     float32 [qlen], qlen >= 1
 *   values, offsets, p   the set, as for dtw_pairwise
 *   out       float32 [p]
 */
int dtw_query(const float *query, int32_t qlen, const float *values, const int64_t *offsets,
              int32_t p, int32_t window, uint32_t flags, float *out, void *stream);

/*
 * dtw_pairs -- DTW of an explicit list of pairs of one set: out[t] =
 * DTW(series pair_a[t], series pair_b[t]) (entries of D, the paragraph on D).
 * Same DP, band and flags as dtw_pairwise (DTW_OUT_PACKED_UPPER is ignored).
 *
 *   values, offsets, p   the set, as for dtw_pairwise
 *   pair_a, pair_b       int32 [npairs] device, indices in [0, p)
 *   npairs               >= 0
 *   out                  float32 [npairs]
 *
 * Synchronises `stream` once to read offsets and the pair indices on the host
 * (validation).  Errors: DTW_EINVAL for an index outside [0, p), p < 1, NULL
 * pointers, or invalid offsets.
 */
int dtw_pairs(const float *values, const int64_t *offsets, int32_t p, const int32_t *pair_a,
              const int32_t *pair_b, int64_t npairs, int32_t window, uint32_t flags, float *out,
              void *stream);

/* Widest band (2*w_eff+1 cells per DP row) the rotated-band kernels hold in
 * registers; wider bands use the column-strip kernel. */
int32_t dtw_max_band_cells(void);

/*
 * dtw_describe_shape -- the kernel and shape dtw_pairwise would run for a set
 * whose series lengths lie in [minlen, maxlen] (minlen == maxlen: one length)
 * with `window` and `flags`, as text in buf (at most buflen bytes, always
 * NUL-terminated), e.g. "dtw_tworow_kernel<H=13,MT=1> G=4".  Host only: no
 * device work.  The DTWGB_SHAPE environment variable, which forces a shape,
 * is honoured as in dtw_pairwise.  Errors: DTW_EINVAL for an invalid length
 * range or buffer, DTW_EUNSUPPORTED as dtw_pairwise.
 */
int dtw_describe_shape(int32_t minlen, int32_t maxlen, int32_t window, uint32_t flags, char *buf,
                       int32_t buflen);

/*
 * kmedoids_fit -- k-medoids clustering over D (the paper's iterative
 * alternative to the MIP, Mathematical background, last paragraph).  The
 * paper gives no algorithm; this is the alternate (Voronoi-iteration)
 * k-medoids of Park & Jun (2009):
 *   assign: label_j = argmin_c D[j, M_c], ties to the smallest c; a medoid
 *           always labels itself;
 *   update: M_c = argmin over members i of sum_{j in cluster c} D[i, j]
 *           (relative error about n 2^-53, as a float64 sum: TwoSum-
 *           compensated float32 pairs, added in float64); a tie keeps the
 *           current medoid if it is among the minima, else the smallest index;
 *   repeat while a medoid changes, at most max_iter update sweeps; the labels
 *   returned are the assignment to the final medoids.
 *
 *   D             float32 [n*n] row-major, symmetric (as written by dtw_pairwise)
 *   n             number of points, >= 1
 *   k             number of clusters, 1 <= k <= n
 *   init_medoids  int32 [k] device, distinct, each in [0, n)
 *   max_iter      >= 1
 *   out_medoids   int32 [k] device
 *   out_labels    int32 [n] device
 *   out_cost      HOST double: sum_j D[j, M_{label_j}] summed in float64 (the
 *                 clustering cost of the paper's Overview, item 5); may be NULL
 *   out_iters     HOST int32: update sweeps performed; may be NULL
 *
 * Synchronous: reads init_medoids on the host to validate them and reads a
 * convergence flag after every sweep; returns after the final results are
 * written.  Scratch (row sums, flags) is allocated stream-ordered and
 * released before returning.
 * Errors: DTW_EINVAL for n < 1, k outside [1, n], max_iter < 1, NULL
 * pointers, or duplicate / out-of-range initial medoids.
 */
int kmedoids_fit(const float *D, int32_t n, int32_t k, const int32_t *init_medoids,
                 int32_t max_iter, int32_t *out_medoids, int32_t *out_labels, double *out_cost,
                 int32_t *out_iters, void *stream);

/*
 * kmedoids_fit_noalloc -- kmedoids_fit without any device allocation.  The
 * paper has no counterpart; this entry point exists for callers that must not
 * allocate device memory during a call: for example an application whose
 * allocator reserves the GPU's memory up front (a library allocation could
 * fail or fragment its pool), or a loop with a hard latency budget that cannot
 * risk an allocation growing a pool at an unpredictable moment.
 *
 * Arguments, results, errors and synchronisation are those of kmedoids_fit,
 * with one more limit: n <= 65536 and k <= 1024, else DTW_EINVAL with a
 * message.  The scratch is a static device array of about 0.5 MB compiled into
 * the library; every GPU that loads the library's k-medoids kernels holds it
 * until the process exits.  The CUDA runtime loads kernels lazily by default
 * (CUDA_MODULE_LOADING=LAZY), so the array is placed on a device, with device
 * memory of its own, when a k-medoids kernel is first used there: a caller
 * whose allocator reserves the GPU's memory up front should make one call
 * (a 1 x 1 matrix will do) before reserving it, or run with
 * CUDA_MODULE_LOADING=EAGER.  That first call on each device also looks up the
 * array's device address (cudaGetSymbolAddress) and caches it, so it should
 * come before any stream capture.  The cached address belongs to the context
 * current at that first call: the library does not support cudaDeviceReset
 * between calls, nor more than one context per device.  All calls share that
 * one array and leave the last call's contents in it: calls that overlap on
 * the GPU (from several streams, threads or processes sharing the context)
 * race and must be serialised by the caller.  Host-side the call uses a stack
 * buffer only.
 */
int kmedoids_fit_noalloc(const float *D, int32_t n, int32_t k, const int32_t *init_medoids,
                         int32_t max_iter, int32_t *out_medoids, int32_t *out_labels,
                         double *out_cost, int32_t *out_iters, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* DTWGB_H */
