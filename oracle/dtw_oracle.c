/*
 * dtw_oracle.c -- plain, slow CPU oracle for the DTW distance matrix and the
 * k-medoids sweeps of "Fast dynamic time warping and clustering in C++"
 * (arXiv 2307.04904).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this file:
 * only the tests, __graft_entry__.smoke() and the CPU-baseline leg of bench.py
 * load it.  It shares no code, header, table or constant with the CUDA path.
 *
 * Notation follows the paper's "Mathematical background" section: series
 * x = (x_1..x_n) and y = (y_1..y_m), cumulative cost c_{i,j} (Eq. for c),
 * window w of the Sakoe-Chiba band, distance matrix D (p x p), k clusters.
 *
 * Readings of the paper (it is silent or ambiguous on each of these):
 *  - pointwise cost is the squared difference (x_i - y_j)^2 of the equation
 *    for c_{i,j}; no square root is taken of c_{n,m} (the text calls c_{n,m}
 *    the total cost);
 *  - boundary: c_{0,0} = 0 and c_{i,0} = c_{0,j} = +inf for i, j >= 1, which
 *    makes the first and last elements matched and the path continuous;
 *  - band (Introduction, window example; "Overview of method", item 2): cell
 *    (i,j) is admissible iff |i-j| <= w.  w < 0 means no band.  For n != m the
 *    default widens the band to max(w, |n-m|) so that c_{n,m} is reachable;
 *    with strict = 1 the band stays w and c_{n,m} = +inf when |n-m| > w.
 *
 * Precision: every DP runs in double on float inputs widened exactly, except
 * oracle_dtw_f32_mirror, which runs the same recurrence in float with a
 * fused multiply-add per cell so that a float implementation that performs
 * the same operations can be compared bit for bit.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_INF HUGE_VAL

/* Band half-width actually used for a pair of lengths n, m; -1 = no band. */
static int64_t band_of(int64_t n, int64_t m, int64_t w, int strict)
{
    if (w < 0) return -1;
    if (strict) return w;
    int64_t d = n > m ? n - m : m - n;
    return w > d ? w : d;
}

static double min3d(double a, double b, double c)
{
    double r = a < b ? a : b;
    return r < c ? r : c;
}

/*
 * c_{n,m} of the recurrence
 *     c_{i,j} = (x_i - y_j)^2 + min(c_{i-1,j-1}, c_{i-1,j}, c_{i,j-1})
 * in double, keeping only the previous row as the paper does ("Mathematical
 * background", the paragraph after the equation).  Cells outside the band
 * are +inf.  `work` must hold 2*(m+1) doubles.
 */
double oracle_dtw_f64_ws(const float *x, int64_t n, const float *y, int64_t m,
                         int64_t w, int strict, double *work)
{
    double *prev = work, *cur = work + (m + 1);
    int64_t band = band_of(n, m, w, strict);
    prev[0] = 0.0; /* c_{0,0} */
    for (int64_t j = 1; j <= m; ++j) prev[j] = ORACLE_INF; /* c_{0,j} */
    for (int64_t i = 1; i <= n; ++i) {
        for (int64_t j = 0; j <= m; ++j) cur[j] = ORACLE_INF; /* c_{i,0}, out-of-band */
        int64_t lo = 1, hi = m;
        if (band >= 0) {
            if (i - band > lo) lo = i - band;
            if (i + band < hi) hi = i + band;
        }
        for (int64_t j = lo; j <= hi; ++j) {
            double d = (double)x[i - 1] - (double)y[j - 1];
            cur[j] = d * d + min3d(prev[j - 1], prev[j], cur[j - 1]);
        }
        double *t = prev; prev = cur; cur = t;
    }
    return prev[m];
}

double oracle_dtw_f64(const float *x, int64_t n, const float *y, int64_t m,
                      int64_t w, int strict)
{
    double *work = (double *)malloc(sizeof(double) * 2 * (size_t)(m + 1));
    if (!work) return NAN;
    double r = oracle_dtw_f64_ws(x, n, y, m, w, strict, work);
    free(work);
    return r;
}

/*
 * The same recurrence evaluated in float: d = x_i - y_j rounded to float,
 * then c = fmaf(d, d, min(min(c_diag, c_up), c_left)).  min is exact, so the
 * result does not depend on how the three-way minimum is grouped.
 */
float oracle_dtw_f32_mirror(const float *x, int64_t n, const float *y, int64_t m,
                            int64_t w, int strict)
{
    float *prev = (float *)malloc(sizeof(float) * 2 * (size_t)(m + 1));
    if (!prev) return NAN;
    float *cur = prev + (m + 1), *base = prev;
    int64_t band = band_of(n, m, w, strict);
    prev[0] = 0.0f;
    for (int64_t j = 1; j <= m; ++j) prev[j] = INFINITY;
    for (int64_t i = 1; i <= n; ++i) {
        for (int64_t j = 0; j <= m; ++j) cur[j] = INFINITY;
        int64_t lo = 1, hi = m;
        if (band >= 0) {
            if (i - band > lo) lo = i - band;
            if (i + band < hi) hi = i + band;
        }
        for (int64_t j = lo; j <= hi; ++j) {
            float d = x[i - 1] - y[j - 1];
            float b = fminf(fminf(prev[j - 1], prev[j]), cur[j - 1]);
            cur[j] = fmaf(d, d, b);
        }
        float *t = prev; prev = cur; cur = t;
    }
    float r = prev[m];
    free(base);
    return r;
}

/* Number of admissible cells of the band, i.e. the DP work of one pair. */
int64_t oracle_band_cells(int64_t n, int64_t m, int64_t w, int strict)
{
    int64_t band = band_of(n, m, w, strict), cells = 0;
    for (int64_t i = 1; i <= n; ++i) {
        int64_t lo = 1, hi = m;
        if (band >= 0) {
            if (i - band > lo) lo = i - band;
            if (i + band < hi) hi = i + band;
        }
        if (hi >= lo) cells += hi - lo + 1;
    }
    return cells;
}

/*
 * Distance matrix D (p x p, row major): d_{ij} = c_{n,m} of series i against
 * series j ("Mathematical background", the matrix D paragraph).  Series i is
 * values[offsets[i] .. offsets[i+1]).  The upper triangle is computed and
 * mirrored; the diagonal is computed too (it is 0 for any series).
 */
void oracle_pairwise_f64(const float *values, const int64_t *offsets, int64_t p,
                         int64_t w, int strict, double *D, int threads)
{
    int64_t maxlen = 0;
    for (int64_t i = 0; i < p; ++i) {
        int64_t l = offsets[i + 1] - offsets[i];
        if (l > maxlen) maxlen = l;
    }
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#else
    (void)threads;
#endif
#pragma omp parallel
    {
        double *work = (double *)malloc(sizeof(double) * 2 * (size_t)(maxlen + 1));
#pragma omp for schedule(dynamic, 16)
        for (int64_t i = 0; i < p; ++i) {
            for (int64_t j = i; j < p; ++j) {
                const float *x = values + offsets[i], *y = values + offsets[j];
                int64_t n = offsets[i + 1] - offsets[i], m = offsets[j + 1] - offsets[j];
                double c = oracle_dtw_f64_ws(x, n, y, m, w, strict, work);
                D[i * p + j] = c;
                D[j * p + i] = c;
            }
        }
        free(work);
    }
}

/* d for an explicit list of pairs (a[t], b[t]); used to sample large matrices. */
void oracle_pairs_f64(const float *values, const int64_t *offsets, const int64_t *a,
                      const int64_t *b, int64_t count, int64_t w, int strict,
                      double *out, int threads)
{
    int64_t maxlen = 0;
    for (int64_t t = 0; t < count; ++t) {
        int64_t l1 = offsets[a[t] + 1] - offsets[a[t]], l2 = offsets[b[t] + 1] - offsets[b[t]];
        if (l1 > maxlen) maxlen = l1;
        if (l2 > maxlen) maxlen = l2;
    }
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#else
    (void)threads;
#endif
#pragma omp parallel
    {
        double *work = (double *)malloc(sizeof(double) * 2 * (size_t)(maxlen + 1));
#pragma omp for schedule(dynamic, 16)
        for (int64_t t = 0; t < count; ++t) {
            const float *x = values + offsets[a[t]], *y = values + offsets[b[t]];
            int64_t n = offsets[a[t] + 1] - offsets[a[t]], m = offsets[b[t] + 1] - offsets[b[t]];
            out[t] = oracle_dtw_f64_ws(x, n, y, m, w, strict, work);
        }
        free(work);
    }
}

/* d(a[t], b[t]) in double with a window of its own for every pair. */
void oracle_pairs_w_f64(const float *values, const int64_t *offsets, const int64_t *a,
                        const int64_t *b, const int64_t *w, int64_t count, int strict,
                        double *out, int threads)
{
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#else
    (void)threads;
#endif
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < count; ++t) {
        const float *x = values + offsets[a[t]], *y = values + offsets[b[t]];
        int64_t n = offsets[a[t] + 1] - offsets[a[t]], m = offsets[b[t] + 1] - offsets[b[t]];
        out[t] = oracle_dtw_f64(x, n, y, m, w[t], strict);
    }
}

/* float mirror over a list of pairs (same pairing as oracle_pairs_f64). */
void oracle_pairs_f32_mirror(const float *values, const int64_t *offsets, const int64_t *a,
                             const int64_t *b, int64_t count, int64_t w, int strict,
                             float *out, int threads)
{
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#else
    (void)threads;
#endif
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < count; ++t) {
        const float *x = values + offsets[a[t]], *y = values + offsets[b[t]];
        int64_t n = offsets[a[t] + 1] - offsets[a[t]], m = offsets[b[t] + 1] - offsets[b[t]];
        out[t] = oracle_dtw_f32_mirror(x, n, y, m, w, strict);
    }
}

/* float mirror over a list of pairs, each with a window of its own (same
 * pairing as oracle_pairs_w_f64). */
void oracle_pairs_w_f32_mirror(const float *values, const int64_t *offsets, const int64_t *a,
                               const int64_t *b, const int64_t *w, int64_t count, int strict,
                               float *out, int threads)
{
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#else
    (void)threads;
#endif
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < count; ++t) {
        const float *x = values + offsets[a[t]], *y = values + offsets[b[t]];
        int64_t n = offsets[a[t] + 1] - offsets[a[t]], m = offsets[b[t] + 1] - offsets[b[t]];
        out[t] = oracle_dtw_f32_mirror(x, n, y, m, w[t], strict);
    }
}

/* One query q (length nq) against every series of a set: one row of D. */
void oracle_query_f64(const float *q, int64_t nq, const float *values, const int64_t *offsets,
                      int64_t p, int64_t w, int strict, double *out, int threads)
{
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#else
    (void)threads;
#endif
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < p; ++i) {
        int64_t m = offsets[i + 1] - offsets[i];
        out[i] = oracle_dtw_f64(q, nq, values + offsets[i], m, w, strict);
    }
}

/* ------------------------------------------------------------------------ */
/* k-medoids ("Mathematical background", last paragraph; the paper gives no
 * algorithm).  Reading: the alternate (Voronoi-iteration) k-medoids of
 * Park & Jun (2009), run on the supplied D in double:
 *   assign : label_j = argmin_c D[j, M_c]; ties go to the smallest c; a
 *            medoid always labels itself, so no cluster is empty;
 *   update : for each cluster c, S_i = sum_{j in C_c} D[i, j] over members i;
 *            M_c <- argmin S_i; a tie keeps the current medoid if it is among
 *            the minima, otherwise the smallest index wins;
 *   repeat while any medoid changes, for at most max_iter update sweeps.
 * The returned labels are the assignment to the final medoids and the cost is
 * sum_j D[j, M_{label_j}] (the clustering cost, the MIP objective evaluated at
 * the k-medoids answer).
 *
 * min_margin reports the smallest relative gap met between the best and the
 * second-best candidate of any assign or update decision; a gap below ~1e-6
 * means a float implementation may legitimately decide differently.
 */
static void km_assign(const double *D, int64_t p, int64_t k, const int64_t *M,
                      int64_t *labels, double *margin)
{
    for (int64_t j = 0; j < p; ++j) {
        int64_t own = -1;
        for (int64_t c = 0; c < k; ++c)
            if (M[c] == j) { own = c; break; }
        if (own >= 0) { labels[j] = own; continue; }
        int64_t best = 0;
        double bd = D[j * p + M[0]], second = ORACLE_INF;
        for (int64_t c = 1; c < k; ++c) {
            double d = D[j * p + M[c]];
            if (d < bd) { second = bd; bd = d; best = c; }
            else if (d < second) second = d;
        }
        labels[j] = best;
        if (k > 1 && margin) {
            double scale = fabs(second) > 0 ? fabs(second) : 1.0;
            double g = (second - bd) / scale;
            if (g < *margin) *margin = g;
        }
    }
}

static int km_update(const double *D, int64_t p, int64_t k, const int64_t *M,
                     const int64_t *labels, int64_t *Mnew, double *margin)
{
    int changed = 0;
    for (int64_t c = 0; c < k; ++c) {
        double bestS = ORACLE_INF, second = ORACLE_INF, curS = ORACLE_INF;
        int64_t best = -1;
        for (int64_t i = 0; i < p; ++i) {
            if (labels[i] != c) continue;
            double S = 0.0;
            for (int64_t j = 0; j < p; ++j)
                if (labels[j] == c) S += D[i * p + j];
            if (i == M[c]) curS = S;
            if (S < bestS) { second = bestS; bestS = S; best = i; }
            else if (S < second) second = S;
        }
        /* tie: keep the current medoid when it reaches the minimum */
        int64_t chosen = (curS == bestS) ? M[c] : best;
        Mnew[c] = chosen;
        if (chosen != M[c]) changed = 1;
        if (margin && second < ORACLE_INF) {
            double scale = fabs(second) > 0 ? fabs(second) : 1.0;
            double g = (second - bestS) / scale;
            if (g < *margin) *margin = g;
        }
    }
    return changed;
}

int oracle_kmedoids(const double *D, int64_t p, int64_t k, const int64_t *init,
                    int64_t max_iter, int64_t *medoids, int64_t *labels,
                    double *cost, int64_t *iters, double *min_margin)
{
    int64_t *M = (int64_t *)malloc(sizeof(int64_t) * (size_t)k);
    int64_t *Mn = (int64_t *)malloc(sizeof(int64_t) * (size_t)k);
    if (!M || !Mn) { free(M); free(Mn); return -1; }
    memcpy(M, init, sizeof(int64_t) * (size_t)k);
    double margin = ORACLE_INF;
    int64_t it = 0;
    for (int64_t s = 1; s <= max_iter; ++s) {
        km_assign(D, p, k, M, labels, &margin);
        int changed = km_update(D, p, k, M, labels, Mn, &margin);
        it = s;
        if (!changed) break;
        memcpy(M, Mn, sizeof(int64_t) * (size_t)k);
    }
    km_assign(D, p, k, M, labels, &margin);
    double total = 0.0;
    for (int64_t j = 0; j < p; ++j) total += D[j * p + M[labels[j]]];
    memcpy(medoids, M, sizeof(int64_t) * (size_t)k);
    *cost = total;
    *iters = it;
    if (min_margin) *min_margin = margin;
    free(M);
    free(Mn);
    return 0;
}

/* Clustering cost of a given labelling: sum_j D[j, M_{label_j}]. */
double oracle_cluster_cost(const double *D, int64_t p, const int64_t *M, const int64_t *labels)
{
    double total = 0.0;
    for (int64_t j = 0; j < p; ++j) total += D[j * p + M[labels[j]]];
    return total;
}
