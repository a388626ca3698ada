// strip.cu -- DTW for bands too wide for the rotated kernel: one warp per pair,
// original coordinates, vertical strips of 32*K columns.
//
// Lane l of the warp owns columns [j0 + lK, j0 + lK + K) of the current strip
// (their y values stay in registers for the whole strip) and works on row
// r0 + T - l at step T.  Per cell (i, j) the predecessors are (i-1, j-1),
// (i-1, j), (i, j-1): the lane's own previous row supplies the first two, the
// current row the third; the first slot's left and diagonal values come from
// lane l-1 (shuffle up, one step earlier) or, at lane 0, from the column
// buffer `bnd`, where the previous strip's last lane left c_{i, j0-1}.  The last
// lane writes c_{i, j0+32K-1} into `bnd` for the next strip, always behind the
// row lane 0 reads, so one buffer per warp serves in place.
//
// Each strip only visits the rows that meet the band, [j0-w, j0+32K-1+w].
// Blocks of steps in which every cell of every lane is inside the band and
// inside the strip's rows run without any mask or predicate (warp-uniform
// decision).  In the others a cell outside the band becomes +inf by adding the
// block's edge mask.  With the wavefront skewed one row per lane and the band
// edges at 45 degrees, lane l meets an edge K + 1 steps after lane l - 1, so
// each edge keeps the warp in masked blocks for about 32(K + 1) steps of every
// strip it crosses: a large part of a wide pair, at one addition per cell.
// Columns beyond m read the +inf padding of the staged series and stay +inf.
#include "tstrip.cuh"

namespace dtwgb {

constexpr int kStripBlock = 8;  // steps per predicate-free block

template <int K, bool CHECK>
__device__ __forceinline__ void strip_step(const int l, const int s, const int i,
                                           const int r_start, const int r_end,
                                           const float (&yv)[K], float (&prev)[K], float &xi,
                                           float &xnext, float &left, float &diag,
                                           float &bnext, const float *xrow, float *bnd,
                                           float (&mk)[K], const unsigned d0, const unsigned w2)
{
    const unsigned FULL = 0xffffffffu;
    const bool active = !CHECK || (i >= r_start && i <= r_end);
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
        if (l == 31) bnd[i] = prev[K - 1];
    }
    if (CHECK) edge_masks_next<K>(d0, w2, s, mk);
    // next row: lane l-1's last slot of row i+1 (computed this step) is our left
    const float lin = __shfl_up_sync(FULL, prev[K - 1], 1);
    diag = left;
    left = (l == 0) ? bnext : lin;
    // x rows outside [1, n] read the +inf padding of the staged series
    xi = xnext;
    xnext = __ldg(xrow + i + 2);  // x_{i+2}: the row after next
    // lane 0 only reads boundary rows that exist (in the ramp-out it runs past r_end)
    if (l == 0 && (!CHECK || i + 2 <= r_end)) bnext = bnd[i + 2];
}

template <int K, typename Src>
__global__ void __launch_bounds__(256) dtw_strip_kernel(const Src src, float *bnd_all,
                                                        int64_t bnd_stride)
{
    const float INF = finf();
    const int l = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    float *bnd = bnd_all + warp * bnd_stride;  // bnd[i] = c_{i, j0-1}, i in [0, n+3]
    constexpr int WS = 32 * K;

    int64_t cursor = warp - nwarps, pair = 0;
    int job = 0;
    while (next_item(src, cursor, nwarps, 0xffffffffu, l, job, pair)) {
        const BandArgs &A = src.job(job);
        PairGeom g;
        pair_geometry(A, pair, g);
        if (g.trivial) {
            if (l == 0) write_result(A, pair, g, INF);
            continue;
        }
        const int n = g.n, m = g.m, w = g.w;
        for (int i = l; i <= n + 3; i += 32) bnd[i] = INF;  // c_{i,0} = +inf
        __syncwarp();
        float result = INF;
        for (int j0 = 1; j0 <= m; j0 += WS) {
            const int jl = j0 + l * K;
            float yv[K], prev[K];
#pragma unroll
            for (int t = 0; t < K; ++t) {
                yv[t] = __ldg(g.y + (jl + t - 1));  // padding gives +inf beyond m
                prev[t] = INF;                        // the row above the strip's rows
            }
            const int r_start = j0 - w > 1 ? j0 - w : 1;
            const int r_end = j0 + WS - 1 + w < n ? j0 + WS - 1 + w : n;
            // Lane 0 starts from the column buffer: diag = c_{r_start-1, j0-1} (row 0
            // holds c_{0,0} = 0 only at column 0), left = c_{r_start, j0-1}.  Lane l >= 1
            // receives its values by shuffle from lane l-1, which is inactive (+inf)
            // until its own first row; its own predecessors above r_start lie outside
            // the band (or in row 0), so both start at +inf.
            float diag = INF, left = INF, bnext = INF;
            if (l == 0) {
                diag = (r_start == 1) ? (j0 == 1 ? 0.f : INF) : bnd[r_start - 1];
                left = bnd[r_start];
                bnext = bnd[r_start + 1];
            }
            // lane l starts at row r_start - l (inactive until its first row); x rows
            // outside [1, n] read the padding
            const float *xrow = g.x - 1;  // xrow[r] = x_r
            int i = r_start - l;
            float xi = __ldg(xrow + i), xnext = __ldg(xrow + i + 1);
            const int nsteps = r_end - r_start + 1 + 31;
            const unsigned w2 = 2u * (unsigned)w;
            for (int T0 = 0; T0 < nsteps; T0 += kStripBlock) {
                // rows of this lane in the block: [i, i + B - 1]
                const int ib = i + kStripBlock - 1;
                const bool clean = i >= r_start && ib <= r_end && jl >= ib - w &&
                                   jl + K - 1 <= i + w && T0 + kStripBlock <= nsteps;
                float mk[K];
                const unsigned d0 = (unsigned)(i - jl + w);
                if (__all_sync(0xffffffffu, clean)) {
#pragma unroll
                    for (int s = 0; s < kStripBlock; ++s, ++i)
                        strip_step<K, false>(l, s, i, r_start, r_end, yv, prev, xi, xnext, left,
                                             diag, bnext, xrow, bnd, mk, d0, w2);
                } else {
                    edge_masks_init<K>(d0, w2, mk);
#pragma unroll
                    for (int s = 0; s < kStripBlock; ++s, ++i)
                        strip_step<K, true>(l, s, i, r_start, r_end, yv, prev, xi, xnext, left,
                                            diag, bnext, xrow, bnd, mk, d0, w2);
                }
            }
            // c_{n,m} lies in the strip holding column m, in the row n every lane ended on
            if (m < j0 + WS) {
                const int lm = (m - j0) / K, tm = (m - j0) - lm * K;
                float r = prev[0];
#pragma unroll
                for (int t = 1; t < K; ++t)
                    if (t == tm) r = prev[t];
                if (l == lm) result = r;
            }
            __syncwarp();
        }
        const int lm = ((m - 1) % WS) / K;
        if (l == lm) write_result(A, pair, g, result);
        __syncwarp();
    }
}

template <typename Src>
int launch_strip_src(const Src &src, int K, float *bnd, int64_t bnd_stride, int64_t warps,
                     cudaStream_t st)
{
    const int64_t blocks = warps / (kThreads / 32);
    switch (K) {
    case 4: dtw_strip_kernel<4, Src><<<(unsigned)blocks, kThreads, 0, st>>>(src, bnd, bnd_stride); break;
    case 8: dtw_strip_kernel<8, Src><<<(unsigned)blocks, kThreads, 0, st>>>(src, bnd, bnd_stride); break;
    case 16: dtw_strip_kernel<16, Src><<<(unsigned)blocks, kThreads, 0, st>>>(src, bnd, bnd_stride); break;
    default: set_error("internal: no strip kernel for K=%d", K); return DTW_EUNSUPPORTED;
    }
    DTWGB_CUDA(cudaGetLastError());
    return DTW_OK;
}

int launch_strip(const BandArgs &A, int K, float *bnd, int64_t bnd_stride, int64_t warps,
                 cudaStream_t st)
{
    StaticSrc src{A, 32, 5};
    return launch_strip_src(src, K, bnd, bnd_stride, warps, st);
}

int launch_strip_queue(const QueueSrc &src, int K, float *bnd, int64_t bnd_stride,
                       int64_t warps, cudaStream_t st)
{
    return launch_strip_src(src, K, bnd, bnd_stride, warps, st);
}

int strip_warps(int K, int64_t n_pairs, int64_t *warps)
{
    int dev = 0, sms = 0, per_sm = 0;
    DTWGB_CUDA(cudaGetDevice(&dev));
    DTWGB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    cudaError_t e;
    switch (K) {
    case 4: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dtw_strip_kernel<4, QueueSrc>, kThreads, 0); break;
    case 8: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dtw_strip_kernel<8, QueueSrc>, kThreads, 0); break;
    default: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dtw_strip_kernel<16, QueueSrc>, kThreads, 0); break;
    }
    if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
    if (per_sm < 1) per_sm = 1;
    const int64_t wmax = (int64_t)sms * per_sm * (kThreads / 32);
    int64_t w = n_pairs < wmax ? (n_pairs > 0 ? n_pairs : 1) : wmax;
    *warps = (w + 7) / 8 * 8;
    return DTW_OK;
}

}  // namespace dtwgb
