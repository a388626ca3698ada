/*
 * dtwgb_batch.h -- batched DTW work: many ragged sets and queries, planned
 * once, run as cost-sorted persistent work queues captured in a CUDA graph.
 *
 * The paper computes its distance matrix D pair by pair, in parallel over
 * pairs, for series that may differ in length (Mathematical background,
 * problem statement and the paragraph on D).  A batch applies the same DP and
 * band readings as dtw_pairwise / dtw_query (see dtwgb.h) to several jobs at
 * once:
 *
 *   plan (dtw_batch_create, host side, once):
 *     - enumerate every pair of every job (all pairs i < j of a set, or the
 *       query against every series), compute its band and its cost;
 *     - give every pair a kernel shape: a rotated-band shape (K slots per lane,
 *       G lanes per pair) when the band row fits in registers, else a
 *       column-strip shape (one warp per pair, 32*K columns per strip); the
 *       shape comes from an instruction-count model or, with
 *       DTW_BATCH_AUTOTUNE, from timing candidate shapes on sampled pairs of
 *       each length/band bucket;
 *     - one work queue per shape class, sorted by estimated cost, largest
 *       first, uploaded to the device;
 *     - with DTW_BATCH_GRAPH, capture one run (queue resets, staging of every
 *       job's series, one persistent launch per class on parallel graph
 *       branches, diagonals) into a CUDA graph.
 *   run (dtw_batch_run, every time): replay the graph (or enqueue the same
 *       launches) on `stream`.  The jobs' buffers are read and written at run
 *       time, so new data in the same buffers is picked up by each run.
 *
 * Ownership: the batch keeps device pointers of the jobs (values, offsets,
 * query, out); they must stay valid at the same addresses until
 * dtw_batch_destroy.  Host offsets are read only by dtw_batch_create.
 */
#ifndef DTWGB_BATCH_H
#define DTWGB_BATCH_H

#include <stdint.h>

#include "dtwgb.h"

#ifdef __cplusplus
extern "C" {
#endif

/* flags for dtw_batch_create */
#define DTW_BATCH_GRAPH 0x1u    /* capture the run into a CUDA graph; runs replay it */
#define DTW_BATCH_AUTOTUNE 0x2u /* time candidate shapes per bucket at plan time (runs the
                                   kernels on the jobs' data, writing correct values) */
#define DTW_BATCH_UNSORTED 0x4u /* keep enumeration order in each queue (for comparison) */
#define DTW_BATCH_POOLED 0x8u   /* one-shot use: device buffers come from the library's
                                   stream-ordered pool on `stream` and are released
                                   stream-ordered by dtw_batch_destroy, every class runs on
                                   the run's stream, and neither create nor destroy
                                   synchronises (runs must use the create stream); excludes
                                   DTW_BATCH_GRAPH and DTW_BATCH_AUTOTUNE */

typedef struct dtw_job {
    const float *values;         /* device: series of the set, concatenated */
    const int64_t *offsets;      /* device: p+1 offsets into values */
    const int64_t *offsets_host; /* host copy of the same offsets (read at plan time only) */
    int32_t p;                   /* number of series, >= 1 */
    const float *query;          /* device query series for a 1-vs-p job; NULL: all pairs */
    int32_t qlen;                /* query length (>= 1 when query != NULL) */
    int32_t window;              /* band half-width w; < 0: no band */
    int32_t window_permille;     /* > 0: per pair w = floor(window_permille * max(n,m) / 1000),
                                    replacing `window` */
    uint32_t flags;              /* DTW_BAND_STRICT | DTW_OUT_PACKED_UPPER (sets) */
    float *out;                  /* device: p*p (or p(p-1)/2 packed) for a set, p for a query */
} dtw_job;

typedef struct dtw_batch dtw_batch;

typedef struct dtw_batch_info {
    int64_t pairs;     /* work items: pairs of sets plus query rows */
    int64_t cells;     /* in-band DP cells over all items (the work of one run) */
    int32_t classes;   /* shape classes, one persistent launch each */
    int32_t graph;     /* 1 if runs replay a captured CUDA graph */
    int32_t buckets_tuned; /* length/band buckets timed by the autotuner (0 without it) */
    int32_t jobs;
} dtw_batch_info;

/*
 * Plan a batch of `njobs` jobs.  Synchronises `stream` (autotuning and graph
 * capture run on it).  Errors: DTW_EINVAL for an invalid job (as for
 * dtw_pairwise / dtw_query: p < 1, empty series, decreasing offsets, NULL
 * pointers, qlen < 1 with a query); DTW_ENOMEM; DTW_ECUDA.  On error *out is
 * NULL and nothing is kept.
 */
int dtw_batch_create(const dtw_job *jobs, int32_t njobs, uint32_t flags, void *stream,
                     dtw_batch **out);

/* Enqueue one run on `stream` (asynchronous). */
int dtw_batch_run(dtw_batch *batch, void *stream);

/* Totals of a planned batch. */
int dtw_batch_get_info(const dtw_batch *batch, dtw_batch_info *info);

/*
 * Plan, run once and release a batch on `stream` with DTW_BATCH_POOLED: the
 * jobs' DTW values are written to their `out` buffers when `stream` reaches
 * the end of the enqueued work; nothing on the device is synchronised (the
 * planning itself runs on the host before the call returns).  For servers that
 * pack the jobs that arrive together into one set of persistent launches.
 * flags: 0 or DTW_BATCH_UNSORTED.  Errors: as dtw_batch_create.
 */
int dtw_batch_run_once(const dtw_job *jobs, int32_t njobs, uint32_t flags, void *stream);

/* Shape class i (0 <= i < classes): kind 0 = rotated band (K slots, G lanes
 * per pair), kind 1 = column strip (one warp per pair, strips of 32*K
 * columns), kind 2 = transposed strip (G lanes per pair hold the shorter
 * series, K values each, and walk the longer one's rows), kind 3 = two-row
 * rotated band (K = 2H slots per lane in two halves one row apart, G lanes);
 * number of items and estimated cells in its queue. */
int dtw_batch_get_class(const dtw_batch *batch, int32_t i, int32_t *kind, int32_t *K, int32_t *G,
                        int64_t *items, int64_t *cells);

/* Release everything the batch owns (synchronises the device the batch was
 * planned on).  NULL is ignored. */
void dtw_batch_destroy(dtw_batch *batch);

#ifdef __cplusplus
}
#endif

#endif /* DTWGB_BATCH_H */
