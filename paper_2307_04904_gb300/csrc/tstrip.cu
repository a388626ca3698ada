// tstrip.cu -- DTW of pairs whose shorter series fits in one lane group: the
// pair's DP is a single strip with the shorter series across the lanes and the
// longer one down the rows.
//
// The column-strip kernel (strip.cu) puts the shorter series on the rows and
// cuts the longer one into strips of 32 K columns: a pair of lengths n <= m
// costs ceil(m / 32K) strips of n + 31 steps, and with short n the 31-step skew
// of every strip dominates (n = 64: under 2.5 TCUPS).  DTW is symmetric, so the
// same value comes from the transposed DP: G lanes (a power of two with
// G K >= n) own the n columns of the shorter series, K each, in registers for
// the whole pair, and the warp's wavefront walks the m rows of the longer one
// once: m + G - 1 steps, no boundary column, several pairs per warp when G < 32.
//
// Lane l owns columns [lK + 1, lK + K] and works on row T - l at step T.  Its
// left and diagonal values come from lane l - 1 (shuffle up: that lane's last
// column of the same row, computed one step earlier); lane 0's left is column
// 0, +inf (added as a mask), and its diagonal c_{0,0} = 0 on the first row.
// Columns beyond n read the +inf padding and stay +inf.  Blocks of steps in
// which every cell of every lane lies inside the band and the pair's rows run
// without the band mask (warp-uniform test); in the others a cell outside the
// band becomes +inf by adding the block's edge mask.  Each lane holds the row values
// of its current block of steps and loads the next block's a block ahead.
#include <algorithm>

#include "tstrip.cuh"

namespace dtwgb {

constexpr int kTsBlock = 8;  // steps per predicate-free block

template <int K, bool CHECK>
__device__ __forceinline__ void tstrip_step(const int s, const int i, const int m,
                                            const bool have, const int G, const float xi,
                                            const float (&yv)[K], float (&prev)[K], float &left,
                                            float &diag, const float lmask,
                                            float (&mk)[K], const unsigned d0, const unsigned w2)
{
    const bool active = !CHECK || (have && i >= 1 && i <= m);
    if (active) {
        float dg = diag, lf = left;
#pragma unroll
        for (int t = 0; t < K; ++t) {
            const float up = prev[t];
            float v = dtw_cell(xi, yv[t], fmin3(dg, up, lf));
            if (CHECK) v = __fadd_rn(v, mk[t]);  // +inf outside the band
            dg = up;
            prev[t] = v;
            lf = v;
        }
    }
    if (CHECK) edge_masks_next<K>(d0, w2, s, mk);
    // next row: lane l-1's last column of that row (computed this step) is our left
    const float lin = __shfl_up_sync(0xffffffffu, prev[K - 1], 1, G);
    diag = left;
    left = __fadd_rn(lin, lmask);
}

// the row values of the kTsBlock steps starting at row r (padding beyond the series)
__device__ __forceinline__ void load_rows(const float *rowp, int r, float (&x)[kTsBlock])
{
#pragma unroll
    for (int s = 0; s < kTsBlock; ++s) x[s] = __ldg(rowp + r + s);
}

template <int K, typename Src>
__global__ void __launch_bounds__(256, 2) dtw_tstrip_kernel(const Src src)
{
    const float INF = finf();
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int G = src.G;
    const int l = lane & (G - 1);
    const int gpw = 32 >> src.log2G;
    const unsigned gmask = (G == 32) ? FULL : (((1u << G) - 1u) << (lane & ~(G - 1)));
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t ngroups = nwarps * gpw;
    const float lmask = (l == 0) ? INF : 0.f;
    const int jl = l * K + 1;

    int64_t cursor = warp * gpw + (lane >> src.log2G) - ngroups;
    int job = 0;
    int64_t pair = 0;
    PairGeom g;
    float yv[K], prev[K];
    float xc[kTsBlock], xn[kTsBlock];  // row values of this block and of the next (loaded a block ahead)
    float left = INF, diag = INF;
    const float *rowp = nullptr;
    bool have = false;
    int n = 0, m = 0, w = 0, blk = 0, nblk = 0, i = 0;

    while (true) {
        if (!have) {
            while (next_item(src, cursor, ngroups, gmask, l, job, pair)) {
                pair_geometry(src.job(job), pair, g);
                if (!g.trivial) { have = true; break; }
                if (l == 0) write_result(src.job(job), pair, g, INF);
            }
            if (have) {
                // columns: the shorter series (g.x, n values); rows: the longer (g.y, m)
                n = g.n;
                m = g.m;
                w = g.w;
#pragma unroll
                for (int t = 0; t < K; ++t) {
                    yv[t] = __ldg(g.x + (jl + t - 1));  // padding gives +inf beyond n
                    prev[t] = INF;                       // row 0
                }
                rowp = g.y - 1;  // rowp[r] = row r of the longer series
                i = 1 - l;       // lane l reaches row 1 at step l + 1
                load_rows(rowp, i, xc);
                load_rows(rowp, i + kTsBlock, xn);
                left = INF;
                diag = (l == 0) ? 0.f : INF;  // c_{0,0} = 0 for lane 0's first row
                blk = 0;
                nblk = (m + G - 1 + kTsBlock - 1) / kTsBlock;
            }
        }
        if (__all_sync(FULL, !have)) break;

        const int ib = i + kTsBlock - 1;
        const bool clean = have && i >= 1 && ib <= m && ib - jl <= w && jl + K - 1 - i <= w;
        float mk[K];
        const unsigned d0 = (unsigned)(i - jl + w), w2 = 2u * (unsigned)w;
        if (__all_sync(FULL, clean)) {
#pragma unroll
            for (int s = 0; s < kTsBlock; ++s, ++i)
                tstrip_step<K, false>(s, i, m, true, G, xc[s], yv, prev, left, diag, lmask, mk, d0, w2);
        } else {
            edge_masks_init<K>(d0, w2, mk);
#pragma unroll
            for (int s = 0; s < kTsBlock; ++s, ++i)
                tstrip_step<K, true>(s, i, m, have, G, xc[s], yv, prev, left, diag, lmask, mk, d0, w2);
        }
        // rows of the next block are in xn; fetch the block after it
#pragma unroll
        for (int s = 0; s < kTsBlock; ++s) xc[s] = xn[s];
        if (have) load_rows(rowp, i + kTsBlock, xn);

        if (have && ++blk == nblk) {
            // every lane has passed row m; c_{m,n} = c_{n,m} sits in column n
            const int lr = (n - 1) / K, tr = (n - 1) - lr * K;
            float r = prev[0];
#pragma unroll
            for (int t = 1; t < K; ++t)
                if (t == tr) r = prev[t];
            if (l == lr) write_result(src.job(job), pair, g, r);
            have = false;
        }
    }
}

int launch_tstrip_queue(const QueueSrc &src, int K, cudaStream_t st)
{
    switch (K) {
    case 4: return launch_kernel(dtw_tstrip_kernel<4, QueueSrc>, src, src.n_items, src.G, st);
    case 8: return launch_kernel(dtw_tstrip_kernel<8, QueueSrc>, src, src.n_items, src.G, st);
    case 16: return launch_kernel(dtw_tstrip_kernel<16, QueueSrc>, src, src.n_items, src.G, st);
    default: set_error("internal: no transposed strip kernel for K=%d", K); return DTW_EUNSUPPORTED;
    }
}

// Lanes per pair for a shorter series of n values at K columns per lane: the
// smallest power of two with G K >= n (at least 2), or 0 if n > 32 K.
int tstrip_lanes(int n, int K)
{
    int G = 2;
    while (G * K < n && G < 32) G *= 2;
    return G * K >= n ? G : 0;
}

// Warp-instructions per pair: G lanes x (m + G - 1) steps x (3 per cell + the
// exchange, mask and next-row load), plus a mask addition per cell and the
// block's K + 7 masks in the blocks the band's edges cross: rows past w + 1 (the lower edge meets column 1) and rows
// before G K - w (the upper edge meets the last column).
double cost_tstrip(int n, int m, int w, int K)
{
    const int G = tstrip_lanes(n, K);
    if (!G) return 1e300;
    const double steps = m + G - 1;
    const double edge = std::min<double>(m, std::max(0, m - w - 1) + std::max(0, G * K - w) +
                                                2.0 * kTsBlock + G);
    return G * (steps * (3.0 * K + 5.0) + edge * (K + 3.0 * (K + kTsBlock - 1) / kTsBlock)) / 32.0;
}

}  // namespace dtwgb
