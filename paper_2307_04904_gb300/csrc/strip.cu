// strip.cu -- DTW for bands too wide for the rotated kernel: one warp per pair,
// original coordinates, vertical strips of 32*K columns.
//
// Lane l of the warp owns columns [j0 + lK, j0 + lK + K) of the current strip
// (their y values stay in registers for the whole strip) and works on row
// R0 + T - l at step T.  Per cell (i, j) the predecessors are (i-1, j-1),
// (i-1, j), (i, j-1): the lane's own previous row supplies the first two, the
// current row the third; the first slot's left and diagonal values come from
// lane l-1 (shuffle up, one step earlier) or, at lane 0, from the column
// buffer `bnd`, where the previous strip's last lane left c_{i, j0-1}.  The last
// lane writes c_{i, j0+32K-1} into `bnd` for the next strip, always behind the
// row lane 0 reads, so one buffer per warp serves in place.
//
// Band edges.  Outside the band |i - j| <= w every cell must be +inf.  Only the
// cells just outside it, at j - i = w + 1 (upper edge U) and i - j = w + 1
// (lower edge L), are read by cells inside; every cell farther out reads only
// cells that are themselves outside, so once the two edge cells of each row are
// +inf, every cell beyond them comes out +inf by itself (fma(d, d, +inf) with
// finite d).  With the wavefront skewed one row per lane, lane l's U edge cell
// sits at slot T + C - l(K+1) (C = R0 + w + 1 - j0) and its L edge cell at
// slot T + C' - l(K+1) (C' = R0 - w - 1 - j0): consecutive lanes are K + 1
// steps apart, so at any step at most one lane has an edge cell among its K
// slots.  Blocks of P = K + 1 steps that start where T + C (or T + C') is a
// multiple of P therefore put that edge cell in slot s at step s, of the one
// lane l* = (T + C) / P: one addition of a per-lane +0/+inf per step marks the
// whole edge.  Blocks are
//   clean    every lane inside both edges: no masks;
//   edge     one edge crossing, phase-aligned: slot s of lane l* gets +inf;
//   general  alignment prefixes, blocks both edges cross and the last partial
//            block: a K-entry window of +0/+inf masks from the band test
//            |i - j| <= w, moved one slot per step.
// Rows outside the strip's range need no test: rows above it lie beyond the U
// edge and rows below beyond the L edge (or outside [1, n], where the +inf
// padding of x makes every cell +inf; cells past column m may become NaN, and
// no cell at or before column m reads them).  The last strip stops at the step
// in which the lane holding column m reaches row n.
#include "tstrip.cuh"

namespace dtwgb {

enum StripMode { kStripClean = 0, kStripEdge = 1, kStripGeneral = 2 };

template <int K, int MODE>
__device__ __forceinline__ void strip_step(const int l, const int s, const int i,
                                           const float (&yv)[K], float (&prev)[K], float &xi,
                                           float &xnext, float &left, float &diag, float &bnext,
                                           const float *xrow, float *bnd, float (&mk)[K],
                                           const float em, const unsigned d0, const unsigned w2)
{
    const unsigned FULL = 0xffffffffu;
    float dg = diag, lf = left;
#pragma unroll
    for (int t = 0; t < K; ++t) {
        const float up = prev[t];
        float v = dtw_cell(xi, yv[t], fmin3(dg, up, lf));
        if (MODE == kStripGeneral) v = __fadd_rn(v, mk[t]);  // +inf outside the band
        if (MODE == kStripEdge && t == s) v = __fadd_rn(v, em);  // the crossing lane's edge cell
        dg = up;
        prev[t] = v;
        lf = v;
    }
    if (l == 31) bnd[i] = prev[K - 1];
    if (MODE == kStripGeneral) edge_masks_next<K>(d0, w2, s, mk);
    // next row: lane l-1's last slot of row i+1 (computed this step) is our left
    const float lin = __shfl_up_sync(FULL, prev[K - 1], 1);
    diag = left;
    left = (l == 0) ? bnext : lin;
    xi = xnext;
    xnext = __ldg(xrow + i + 2);  // x_{i+2}: the row after next
    if (l == 0) bnext = bnd[i + 2];
}

// Resident blocks per SM the register budget is set for: 64, 80 and 128
// registers a thread for K = 4, 8, 16.
template <int K>
constexpr int strip_min_blocks()
{
    return K <= 4 ? 4 : (K <= 8 ? 3 : 2);
}

template <int K, typename Src>
__global__ void __launch_bounds__(256, strip_min_blocks<K>()) dtw_strip_kernel(const Src src, float *bnd_all,
                                                        int64_t bnd_stride)
{
    constexpr int P = K + 1;
    // clean blocks need no phase: 8 steps for every K keeps the unrolled loop
    // small; general blocks run at most 8 steps (a prefix that ends short of an
    // edge block's phase is completed by the next block)
    constexpr int BC = 8;
    constexpr int BG = P < 8 ? P : 8;
    const float INF = finf();
    const int l = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    float *bnd = bnd_all + warp * bnd_stride + 32;  // bnd[i] = c_{i, j0-1}, i in [-32, n+35]
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
        for (int i = l; i <= n + 35; i += 32) bnd[i] = INF;  // c_{i,0} = +inf
        __syncwarp();
        float result = INF;
        const int lm = ((m - 1) % WS) / K;  // lane of column m in the last strip
        for (int j0 = 1; j0 <= m; j0 += WS) {
            const int jl = j0 + l * K;
            float yv[K], prev[K];
#pragma unroll
            for (int t = 0; t < K; ++t) {
                yv[t] = __ldg(g.y + (jl + t - 1));  // padding gives +inf beyond m
                prev[t] = INF;                        // the row above the strip's rows
            }
            const int R0 = j0 - w > 1 ? j0 - w : 1;
            const int r_end = j0 + WS - 1 + w < n ? j0 + WS - 1 + w : n;
            const bool last = m < j0 + WS;
            // the last strip ends when lane lm reaches row n (= r_end), the others when
            // lane 31 has written row r_end
            const int nsteps = r_end - R0 + 1 + (last ? lm : 31);
            // Lane 0 starts from the column buffer: diag = c_{R0-1, j0-1} (row 0 holds
            // c_{0,0} = 0 only at column 0), left = c_{R0, j0-1}.  Lane l >= 1 starts
            // above the strip's rows with +inf predecessors.
            float diag = INF, left = INF, bnext = INF;
            if (l == 0) {
                diag = (R0 == 1) ? (j0 == 1 ? 0.f : INF) : bnd[R0 - 1];
                left = bnd[R0];
                bnext = bnd[R0 + 1];
            }
            const float *xrow = g.x - 1;  // xrow[r] = x_r; rows outside [1, n] read the padding
            int i = R0 - l;
            float xi = __ldg(xrow + i), xnext = __ldg(xrow + i + 1);
            const unsigned w2 = 2u * (unsigned)w;
            const int C = R0 + w + 1 - j0, CL = R0 - w - 1 - j0;
            float mk[K];
            for (int T0 = 0; T0 < nsteps;) {
                // block kind, from warp-uniform quantities only
                const bool full = T0 + P <= nsteps;
                const bool u_in = T0 + C - 31 * P >= K;  // every lane inside U all block
                const bool l_clear = T0 + P - 1 + CL < 0 || T0 + CL - 31 * P >= K;
                int kind = kStripGeneral, len = full ? BG : (nsteps - T0 < BG ? nsteps - T0 : BG),
                    lstar = 0;
                if (T0 + BC <= nsteps && u_in && (T0 + BC - 1 + CL < 0 || T0 + CL - 31 * P >= K)) {
                    kind = kStripClean;
                    len = BC;
                } else if (full && l_clear) {
                    const int v = T0 + C;  // >= 1
                    const int ph = v % P;
                    if (ph == 0) { kind = kStripEdge; len = P; lstar = v / P; } else if (P - ph < BG) { len = P - ph; }
                } else if (full && u_in) {
                    const int v = T0 + CL;
                    if (v < 0) {
                        if (-v < BG) len = -v;
                    } else {
                        const int ph = v % P;
                        if (ph == 0) { kind = kStripEdge; len = P; lstar = v / P; } else if (P - ph < BG) { len = P - ph; }
                    }
                }
                const unsigned d0 = (unsigned)(i - jl + w);
                if (kind == kStripClean) {
#pragma unroll
                    for (int s = 0; s < BC; ++s, ++i)
                        strip_step<K, kStripClean>(l, s, i, yv, prev, xi, xnext, left, diag, bnext,
                                                   xrow, bnd, mk, 0.f, d0, w2);
                } else if (kind == kStripEdge) {
                    const float em = (l == lstar) ? INF : 0.f;
#pragma unroll
                    for (int s = 0; s < P; ++s, ++i)
                        strip_step<K, kStripEdge>(l, s, i, yv, prev, xi, xnext, left, diag, bnext,
                                                  xrow, bnd, mk, em, d0, w2);
                } else {
                    edge_masks_init<K>(d0, w2, mk);
#pragma unroll
                    for (int s = 0; s < BG; ++s) {
                        if (s < len) {
                            strip_step<K, kStripGeneral>(l, s, i, yv, prev, xi, xnext, left, diag,
                                                         bnext, xrow, bnd, mk, 0.f, d0, w2);
                            ++i;
                        }
                    }
                }
                T0 += len;
            }
            // c_{n,m}: lane lm ended on row n in the last strip
            if (last) {
                const int tm = (m - j0) - lm * K;
                float r = prev[0];
#pragma unroll
                for (int t = 1; t < K; ++t)
                    if (t == tm) r = prev[t];
                if (l == lm) result = r;
            }
            __syncwarp();
        }
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
