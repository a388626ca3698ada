// band_multirow.cuh -- the R-row rotated-band DTW kernel (R = 3).
//
// The generalisation of the two-row kernel (band_tworow.cuh): lane l of a
// group of G lanes owns the band offsets [lK, lK + K) of a row, K = R*H, split
// into R parts of H slots, and at step T part h works on row r - h with
// r = T - R*l (lanes are skewed by R rows).  Part h's predecessors:
//   * slot 0's left value: for h = 0, lane l-1's last slot of its last part
//     on row r, computed one step earlier (shuffle up); for h > 0, the lane's
//     own last slot of part h-1 on row r - h, computed one step earlier;
//   * the last slot's up value: for h < R-1, slot 0 of part h+1 on row
//     r - h - 1, computed first in this step; for the last part, slot 0 of
//     lane l+1's part 0 on row r - R, computed first in this step (shuffle
//     down);
//   * everything else from the part's own previous row.
// So a step runs R independent chains of H cells.  The y windows of all parts
// advance by one per step and rotate together through an H-entry window; the
// entry leaving slot 0 becomes slot H-1's: part h's value there is part h+1's
// slot-1 value of the step just done (the same y), the last part's is one new
// load.  The x values (x_r, x_{r-1}, ..., x_{r-R+1}) shift by one per step.
// Every cell is d = x - y rounded once, then fma(d, d, min of three): the
// values are bitwise those of the one-row kernel.
#pragma once

#include "band_kernels.cuh"

namespace dtwgb {

constexpr int kMultiRowThreads = 256;

template <int R, int H, int MT, bool CHECK>
__device__ __forceinline__ void multirow_step(const int s, const int T, const int l, const int G,
                                              const bool have, const int n, float (&P)[R][H],
                                              float (&Y)[R][H], const float (&tm)[MT],
                                              const float lmask, const float rmask,
                                              float (&X)[R], float &left0, float &xpre,
                                              float &ypre, const float *qx, const float *qy)
{
    const unsigned FULL = 0xffffffffu;
    constexpr int K = R * H;
    bool act[R];
#pragma unroll
    for (int h = 0; h < R; ++h) {
        const int row = T - R * l - h;
        act[h] = !CHECK || (have && row >= 1 && row <= n);
    }
    // slot 0 of every part (part h > 0 takes the last slot of part h-1 from the last step)
    float c[R];
#pragma unroll
    for (int h = 0; h < R; ++h) {
        const float lf = (h == 0) ? left0 : P[h - 1][H - 1];
        const int u = h * H;  // slot index in the lane's band order
        float v = dtw_cell(X[h], Y[h][s % H], fmin3(P[h][0], P[h][1], lf));
        if (MT == K || u >= K - MT) v = __fadd_rn(v, tm[MT == K ? u : u - (K - MT)]);
        c[h] = (CHECK && !act[h]) ? P[h][0] : v;
    }
#pragma unroll
    for (int h = 0; h < R; ++h) P[h][0] = c[h];
    // lane l+1's part-0 slot 0 (row r - R) is the up value of this lane's last slot
    const float up_last = __fadd_rn(__shfl_down_sync(FULL, c[0], 1, G), rmask);
#pragma unroll
    for (int t = 1; t < H; ++t) {
#pragma unroll
        for (int h = 0; h < R; ++h) {
            const float up = (t + 1 < H) ? P[h][t + 1] : (h + 1 < R ? P[h + 1][0] : up_last);
            const int u = h * H + t;
            float v = dtw_cell(X[h], Y[h][(s + t) % H], fmin3(P[h][t], up, c[h]));
            if (MT == K || u >= K - MT) v = __fadd_rn(v, tm[MT == K ? u : u - (K - MT)]);
            if (CHECK && !act[h]) v = P[h][t];
            P[h][t] = v;
            c[h] = v;
        }
    }
    // lane l-1's last slot (row r + 1 next step) is the left value of part 0's slot 0
    left0 = __fadd_rn(__shfl_up_sync(FULL, P[R - 1][H - 1], 1, G), lmask);
    // rotate the window: slot 0's entry becomes slot H-1's
#pragma unroll
    for (int h = 0; h < R; ++h)
        Y[h][s % H] = (h + 1 < R) ? Y[h + 1][(s + 1) % H] : ypre;
#pragma unroll
    for (int h = R - 1; h > 0; --h) X[h] = X[h - 1];
    X[0] = xpre;
    if (!CHECK || have) {
        xpre = __ldg(qx + T + 2);
        ypre = __ldg(qy + T + 1);
    }
}

template <int R, int H, int MT>
constexpr int multirow_min_blocks()
{
#ifdef DTWGB_MULTIROW_MINB
    return DTWGB_MULTIROW_MINB;
#else
    return 2;
#endif
}

template <int R, int H, int MT, typename Src>
__global__ void __launch_bounds__(kMultiRowThreads, (multirow_min_blocks<R, H, MT>()))
    dtw_multirow_kernel(const Src src)
{
    static_assert(R >= 2 && H >= 2 && MT >= 1 && MT <= R * H, "bad multi-row kernel shape");
    constexpr int K = R * H;
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
    const bool first = (l == 0), last = (l == G - 1);
    const int kbase = l * K;
    const float lmask = first ? INF : 0.f;
    const float rmask = last ? INF : 0.f;

    int64_t cursor = warp * gpw + (lane >> src.log2G) - ngroups;
    int job = 0;
    int64_t pair = 0;
    float P[R][H], Y[R][H], X[R], tm[MT];
    float left0 = INF, xpre = 0.f, ypre = 0.f;
    // qx[T] = x_{T-Rl} (part 0's row at step T); qy[T] = the y entering the last
    // part's last slot after step T
    const float *qx = nullptr, *qy = nullptr;
    bool have = false;
    int n = 0, blk = 0, nblk = 0;

    while (true) {
        if (!have) {
            PairGeom g;
            while (next_item(src, cursor, ngroups, gmask, l, job, pair)) {
                const BandArgs &J = src.job(job);
                pair_geometry(J, pair, g);
                if (!g.trivial) { have = true; break; }
                if (first) write_result(J, pair, g, INF);
            }
            if (have) {
                const int w = g.w;
                // part h slot t at step T reads y_j, j = T - Rl - h + lK + hH + t - w,
                // stored at g.y[j - 1]; row 0 everywhere (c_{0,0} = 0 at band offset w)
                const int base = l * (K - R) - w;
#pragma unroll
                for (int h = 0; h < R; ++h)
#pragma unroll
                    for (int t = 0; t < H; ++t) {
                        P[h][t] = (kbase + h * H + t == w) ? 0.f : INF;
                        Y[h][t] = __ldg(g.y + base + h * (H - 1) + t);
                    }
#pragma unroll
                for (int u = 0; u < MT; ++u)
                    tm[u] = (kbase + (MT == K ? u : K - MT + u) > 2 * w) ? INF : 0.f;
                qx = g.x - R * l - 1;
                qy = g.y + base + (R - 1) * (H - 1) + H - 1;
#pragma unroll
                for (int h = 0; h < R; ++h) X[h] = __ldg(qx + 1 - h);
                left0 = INF;
                xpre = __ldg(qx + 2);
                ypre = __ldg(qy + 1);
                n = g.n;
                blk = 0;
                nblk = (n + R * G - 1 + H - 1) / H;
            }
        }
        if (__all_sync(FULL, !have)) break;

        const int T0 = blk * H;
        // every part of every lane inside its pair for the whole block
        const bool fast = __all_sync(FULL, have && T0 >= R * G - 1 && T0 + H <= n);
        if (fast) {
#pragma unroll
            for (int s = 0; s < H; ++s)
                multirow_step<R, H, MT, false>(s, T0 + s + 1, l, G, true, n, P, Y, tm, lmask,
                                               rmask, X, left0, xpre, ypre, qx, qy);
        } else {
#pragma unroll
            for (int s = 0; s < H; ++s)
                multirow_step<R, H, MT, true>(s, T0 + s + 1, l, G, have, n, P, Y, tm, lmask,
                                              rmask, X, left0, xpre, ypre, qx, qy);
        }

        if (have && ++blk == nblk) {
            // every part of every lane now holds row n; c_{n,m} sits at band offset kres
            const BandArgs &J = src.job(job);
            PairGeom g;
            pair_geometry(J, pair, g);
            const int lres = g.kres / K, tres = g.kres - lres * K;
            float r = P[0][0];
#pragma unroll
            for (int h = 0; h < R; ++h)
#pragma unroll
                for (int t = 0; t < H; ++t)
                    if (h * H + t == tres) r = P[h][t];
            if (l == lres) write_result(J, pair, g, r);
            have = false;
        }
    }
}

// Pads the R-row kernel needs around every staged series: x is read down to
// x_{2-RG} and up to about n + RG + H, y from y_{1-w} to about m + G*K + H.
inline int32_t multirow_pad_left(int64_t wmax, int R, int G)
{
    return (int32_t)((wmax > R * G ? wmax : R * G) + 2);
}
inline int32_t multirow_pad_right(int R, int G, int H) { return G * R * H + R * G + H + 4; }

// Slot counts H of the compiled three-row shapes, and the tail a shape with G*3H
// slots needs for a band row of W cells with every pair of that band.
constexpr int kThreeRowHs[] = {5, 6, 7, 8, 9, 10, 11};
inline int threerow_masked_tail(int H, int G, int W)
{
    const int masked = G * 3 * H - W;
    if (masked <= 1) return 1;
    if (masked <= 4) return 4;
    if (masked <= 8) return 8;
    return 3 * H;
}
inline bool threerow_shape_compiled(int H, int MT)
{
    bool listed = false;
    for (int h : kThreeRowHs) listed = listed || h == H;
    return listed && (MT == 1 || MT == 4 || MT == 8);
}

#define DTWGB_THREEROW_SHAPES(X)                                                                \
    X(5, 1) X(5, 4) X(5, 8) X(6, 1) X(6, 4) X(6, 8) X(7, 1) X(7, 4) X(7, 8) X(8, 1) X(8, 4)    \
        X(8, 8) X(9, 1) X(9, 4) X(9, 8) X(10, 1) X(10, 4) X(10, 8) X(11, 1) X(11, 4) X(11, 8)

// Launch the three-row kernel of shape (H, MT) with A.G lanes per pair (band3r.cu).
int launch_threerow(const BandArgs &A, int H, int MT, cudaStream_t st);

// Instruction-count estimate per pair of a three-row shape (dtw_band.cu).
double cost_threerow(int n, int H, int G, int MT);

}  // namespace dtwgb
