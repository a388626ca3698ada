// band_tworow.cuh -- the two-row rotated-band DTW kernel.
//
// Same rotated band coordinates as band_kernels.cuh (i, k = j - i + w; the
// predecessors of (i, k) are (i-1, k) diagonal, (i-1, k+1) up, (i, k-1)
// left), the same G lanes per pair, and lane l again owns the band offsets
// [lK, lK + K) of a row.  What changes is the schedule inside a lane: its
// slots are split into a lower half A = [lK, lK + H) and an upper half
// B = [lK + H, lK + 2H), and at step T half A works on row r = T - 2l while
// half B works on row r - 1 (lanes are skewed by two rows).  Then
//   * A's slot 0 takes its left value from lane l-1's last B slot of row r,
//     computed one step earlier (shuffle up);
//   * B's slot 0 takes its left value from the lane's own last A slot of row
//     r - 1, computed one step earlier;
//   * A's last slot takes its up value from B's slot 0 of row r - 1, computed
//     first in this step;
//   * B's last slot takes its up value from lane l+1's A slot 0 of row r - 2,
//     computed first in this step (shuffle down).
// So every step runs two independent chains of H cells instead of one chain
// of K = 2H: slot t of A and slot t of B do not depend on each other.  Their
// two subtractions are one packed f32x2 instruction (A in the .x halves, B in
// the .y halves, IEEE per half); the minimum and the fused multiply-add stay
// scalar, so the chains stay apart.  The DP values are bitwise those of the
// one-row kernel: d = x - y rounded once, c = fma(d, d, min of three).
//
// The y window: A's slot t at step T reads y_j with j = T - 2l + lK + t - w,
// B's slot t reads j - 1 + H; both advance by one per step, so the pair
// (yA_t, yB_t) rotates through an H-entry window (an H-step unrolled block).
// After a step the entry of slot 0 becomes the entry of slot H - 1: its A half
// is B's slot-1 value of the step just done, its B half is one new load.
// The x pair is (x_r, x_{r-1}): one new load per step.
#pragma once

#include "band_kernels.cuh"

namespace dtwgb {

// Masked tails of the two-row kernel, in slots of the lane's band order: the
// last MT slots are B's last ones when MT <= H; MT = 2H masks every slot
// (ragged sets, where a pair's band can end anywhere in the lanes).
template <int H, int MT>
struct TwoRowMask {
    static constexpr bool kFull = (MT == 2 * H);
    static constexpr int kN = kFull ? H : MT;  // float2 entries (full) or B-half floats
};

// Threads per block and resident blocks per SM the register allocation aims
// for: two independent chains per lane keep more values live than the
// one-row kernel, so 2 blocks of 256 (128 registers) except for the narrowest
// shape.
#ifndef DTWGB_TWOROW_THREADS
#define DTWGB_TWOROW_THREADS 256
#endif
constexpr int kTwoRowThreads = DTWGB_TWOROW_THREADS;
template <int H, int MT>
constexpr int tworow_min_blocks()
{
#ifdef DTWGB_TWOROW_MINB
    return DTWGB_TWOROW_MINB;
#else
    return (H <= 6 && MT == 1) ? 3 : 2;
#endif
}

// The cell of both halves: d = x - y rounded once per half (one packed
// subtraction), then a separate fused multiply-add per half.  Keeping the two
// multiply-adds apart leaves A's and B's chains independent, so the scheduler
// overlaps them; packing them too saves an instruction per cell pair but ties
// each A link to its B link, which measured slower.
__device__ __forceinline__ float2 tworow_cell(float2 x, float2 y, float2 m)
{
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;"
        : "=l"(r)
        : "l"(*reinterpret_cast<unsigned long long *>(&x)),
          "l"(*reinterpret_cast<unsigned long long *>(&y)));
    const float2 d = *reinterpret_cast<float2 *>(&r);
    return make_float2(__fmaf_rn(d.x, d.x, m.x), __fmaf_rn(d.y, d.y, m.y));
}

template <int H, int MT, bool CHECK>
__device__ __forceinline__ void tworow_step(const int s, const int T, const int l, const int G,
                                            const bool have, const int n, float2 (&P)[H],
                                            float2 (&Y)[H],
                                            const float2 (&tm)[TwoRowMask<H, MT>::kN],
                                            const float lmask, const float rmask, float2 &X,
                                            float &leftA, float &xpre, float &ypre,
                                            const float *qx, const float *qy)
{
    using M = TwoRowMask<H, MT>;
    const unsigned FULL = 0xffffffffu;
    bool actA = true, actB = true;
    if (CHECK) {
        const int r = T - 2 * l;
        actA = have && r >= 1 && r <= n;
        actB = have && r >= 2 && r <= n + 1;
    }
    // slot 0 of both halves (B's left is the lane's last A slot of row r - 1)
    float2 v = tworow_cell(X, Y[s % H],
                       make_float2(fmin3(P[0].x, P[1].x, leftA), fmin3(P[0].y, P[1].y, P[H - 1].x)));
    if (M::kFull) v = __fadd2_rn(v, tm[0]);
    else if (H - MT <= 0) v.y = __fadd_rn(v.y, tm[0].x);
    if (CHECK) {
        v.x = actA ? v.x : P[0].x;
        v.y = actB ? v.y : P[0].y;
    }
    // lane l+1's A slot 0 (row r - 2) is the up value of this lane's last B slot
    const float upB_last = __fadd_rn(__shfl_down_sync(FULL, v.x, 1, G), rmask);
    P[0] = v;
    float2 c = v;
#pragma unroll
    for (int t = 1; t < H; ++t) {
        // A's last slot: up = B's slot 0 of row r - 1, just computed (P[0].y)
        const float upA = (t + 1 < H) ? P[t + 1].x : P[0].y;
        const float upB = (t + 1 < H) ? P[t + 1].y : upB_last;
        float2 u = tworow_cell(X, Y[(s + t) % H],
                           make_float2(fmin3(P[t].x, upA, c.x), fmin3(P[t].y, upB, c.y)));
        if (M::kFull) u = __fadd2_rn(u, tm[t]);
        else if (t >= H - MT) u.y = __fadd_rn(u.y, tm[t - (H - MT)].x);
        if (CHECK) {
            u.x = actA ? u.x : P[t].x;
            u.y = actB ? u.y : P[t].y;
        }
        P[t] = u;
        c = u;
    }
    // lane l-1's last B slot (row r) is the left value of A's slot 0 next step
    leftA = __fadd_rn(__shfl_up_sync(FULL, P[H - 1].y, 1, G), lmask);
    Y[s % H] = make_float2(Y[(s + 1) % H].y, ypre);
    X = make_float2(xpre, X.x);
    if (!CHECK || have) {
        xpre = __ldg(qx + T + 2);
        ypre = __ldg(qy + T + 1);
    }
}

template <int H, int MT, typename Src>
__global__ void __launch_bounds__(kTwoRowThreads, (tworow_min_blocks<H, MT>()))
    dtw_tworow_kernel(const Src src)
{
    static_assert(H >= 2 && (MT == 2 * H || (MT >= 1 && MT <= H)), "bad two-row kernel shape");
    using M = TwoRowMask<H, MT>;
    constexpr int K = 2 * H;
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
    float2 P[H], Y[H], tm[M::kN];
    float2 X = make_float2(0.f, 0.f);
    float leftA = INF, xpre = 0.f, ypre = 0.f;
    // qx[T] = x_{T-2l} (A's row at step T), qy[T] = the y entering B's last slot at step T+1
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
                // row 0 in both halves (c_{0,0} = 0 at band offset w); the window of step 1
                const int base = l * (K - 2) - w;
#pragma unroll
                for (int t = 0; t < H; ++t) {
                    P[t] = make_float2((kbase + t == w) ? 0.f : INF,
                                       (kbase + H + t == w) ? 0.f : INF);
                    Y[t] = make_float2(__ldg(g.y + base + t), __ldg(g.y + base + H - 1 + t));
                }
                if (M::kFull) {
#pragma unroll
                    for (int t = 0; t < H; ++t)
                        tm[t] = make_float2((kbase + t > 2 * w) ? INF : 0.f,
                                            (kbase + H + t > 2 * w) ? INF : 0.f);
                } else {
#pragma unroll
                    for (int u = 0; u < M::kN; ++u)
                        tm[u] = make_float2((kbase + K - MT + u > 2 * w) ? INF : 0.f, 0.f);
                }
                qx = g.x - 2 * l - 1;
                qy = g.y + base + 2 * H - 2;
                X = make_float2(__ldg(qx + 1), __ldg(qx));
                leftA = INF;
                xpre = __ldg(qx + 2);
                ypre = __ldg(qy + 1);
                n = g.n;
                blk = 0;
                nblk = (n + 2 * G - 1 + H - 1) / H;
            }
        }
        if (__all_sync(FULL, !have)) break;

        const int T0 = blk * H;
        const bool fast = __all_sync(FULL, have && T0 >= 2 * G - 1 && T0 + H <= n);
        if (fast) {
#pragma unroll
            for (int s = 0; s < H; ++s)
                tworow_step<H, MT, false>(s, T0 + s + 1, l, G, true, n, P, Y, tm, lmask, rmask, X,
                                          leftA, xpre, ypre, qx, qy);
        } else {
#pragma unroll
            for (int s = 0; s < H; ++s)
                tworow_step<H, MT, true>(s, T0 + s + 1, l, G, have, n, P, Y, tm, lmask, rmask, X,
                                         leftA, xpre, ypre, qx, qy);
        }

        if (have && ++blk == nblk) {
            // both halves of every lane now hold row n; c_{n,m} sits at band offset kres
            const BandArgs &J = src.job(job);
            PairGeom g;
            pair_geometry(J, pair, g);
            const int lres = g.kres / K, tres = g.kres - lres * K;
            float r = P[0].x;
#pragma unroll
            for (int t = 0; t < H; ++t) {
                if (t == tres) r = P[t].x;
                if (t + H == tres) r = P[t].y;
            }
            if (l == lres) write_result(J, pair, g, r);
            have = false;
        }
    }
}

// Padding the two-row kernel needs around every staged series: x is read
// down to x_{2-2G} and up to about n + 2G + H, y from y_{1-w} to about
// m + G*K + H (prefetches included).
inline int32_t tworow_pad_left(int64_t wmax, int G)
{
    return (int32_t)((wmax > 2 * G ? wmax : 2 * G) + 2);
}
inline int32_t tworow_pad_right(int G, int H) { return G * 2 * H + 2 * G + H + 4; }

// Slot-pair counts H compiled for the two-row kernel (static pair stride), and
// the tail it needs for a band row of W cells with every pair of that band.
constexpr int kTwoRowHs[] = {6, 8, 10, 12, 13, 16};
inline int tworow_masked_tail(int H, int G, int W)
{
    const int masked = G * 2 * H - W;
    if (masked <= 1) return 1;
    if (masked <= 4 && H >= 4) return 4;
    return 2 * H;
}
inline bool tworow_shape_compiled(int H, int MT)
{
    bool listed = false;
    for (int h : kTwoRowHs) listed = listed || h == H;
    return listed && (MT == 1 || MT == 4 || (MT == 2 * H && H <= 10));
}

// The work-queue launch (batch.cu) has the same shapes.
inline bool tworow_queue_compiled(int H, int MT) { return tworow_shape_compiled(H, MT); }

#define DTWGB_TWOROW_SHAPES(X)                                                                  \
    X(6, 1) X(6, 4) X(6, 12) X(8, 1) X(8, 4) X(8, 16) X(10, 1) X(10, 4) X(10, 20) X(12, 1)     \
        X(12, 4) X(13, 1) X(13, 4) X(16, 1) X(16, 4)

// Launch the two-row kernel of shape (H, MT) with A.G lanes per pair (band2r.cu), or
// on a work queue of many jobs' pairs (band2rq.cu).
int launch_tworow(const BandArgs &A, int H, int MT, cudaStream_t st);
int launch_tworow_queue(const QueueSrc &src, int H, int MT, cudaStream_t st);

// Instruction-count estimate per pair of a two-row shape (dtw_band.cu).
double cost_tworow(int n, int H, int G, int MT);

}  // namespace dtwgb
