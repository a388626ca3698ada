// band_kernels.cuh -- the rotated-band DTW kernels (shared by band1.cu and band2.cu).
//
// The DP of the paper's equation for c_{i,j} is evaluated in rotated band
// coordinates (i, k = j - i + w): the Sakoe-Chiba band |i - j| <= w becomes a
// rectangle of n rows by 2w+1 columns, and the three predecessors of (i, k)
// are (i-1, k) [diagonal], (i-1, k+1) [up] and (i, k-1) [left].
//
// A group of G lanes (G a power of two, 2..32) owns one pair at a time; lane l
// holds band offsets k in [l*K, l*K+K) of the current row in registers.  Lane
// l works on row T - l at step T (a one-step skew), so within a step:
//   * the left value of its first slot is lane l-1's last slot of the same
//     row, computed one step earlier (shuffle up);
//   * the up value of its last slot is lane l+1's first slot of the previous
//     row, computed earlier in the same step (shuffle down);
//   * the band slides one column per row, so the lane's window of y values
//     shifts by one slot per step (a register rotation over a K-step unrolled
//     block); each lane loads its next x and the one y entering its window.
// Series are staged with +inf padding: cells with j outside [1, m] see
// y = +inf and stay +inf, which also realises c_{i,0} = +inf.  Slots beyond
// 2w (when G*K > 2w+1) are forced to +inf by adding +inf on the last MT slots;
// lane 0's left and lane G-1's up values are forced the same way.
//
// Only the previous row is kept (the paper's previous-row vector), here in
// registers; no shared memory, no per-cell band test.  One float is written
// per pair; the full matrix gets d_ij and d_ji (the DP is exactly symmetric).
#pragma once

#include "common.cuh"

namespace dtwgb {

constexpr int kThreads = 256;  // threads per block of every band kernel

enum : int { SRC_TRIANGLE = 0, SRC_QUERY = 1, SRC_LIST = 2 };
enum : int { OUT_FULL = 0, OUT_PACKED = 1, OUT_ROW = 2, OUT_LIST = 3 };

struct BandArgs {
    const float *padded;     // series staged with PL leading and PR trailing +inf (see stage_kernel)
    const int64_t *offsets;  // offsets of the unpadded set
    int64_t qbase;           // SRC_QUERY: index of the query's x_1 in `padded`
    int64_t qlen;
    int64_t p;        // series in the set
    int64_t n_pairs;  // p(p-1)/2 for the triangle, p for a query
    int32_t window;     // < 0: no band
    int32_t wpermille;  // > 0: the band of a pair is floor(wpermille * max(n, m) / 1000) instead
    int32_t strict;
    int32_t src;
    int32_t out_mode;
    float *out;
    int32_t G, log2G;
    int32_t PL, PR;   // padding of every staged series
    const int32_t *pa, *pb;  // SRC_LIST: pair t is (pa[t], pb[t])
    // SRC_TRIANGLE (full matrix) and SRC_QUERY: the series in visiting order (series
    // perm[k] takes the place of k), or nullptr for 0 .. p-1.  Visiting a set of
    // several lengths in order of length gives the lane groups of a warp pairs of
    // similar lengths.  Outputs keep the original indices.
    const int32_t *perm;
};

struct PairGeom {
    const float *x, *y;  // rows (shorter series) and columns, in the padded buffer
    int32_t n, m, w;     // lengths and the band half-width used
    int32_t kres;        // band offset of c_{n,m}
    int64_t a, b;        // output indices
    bool trivial;        // strict band cannot reach (n, m): result +inf
};

__device__ __forceinline__ void pair_geometry(const BandArgs &A, int64_t t, PairGeom &g)
{
    const float *s0, *s1;
    int64_t n0, n1;
    const int64_t o0 = A.offsets[0], pad = A.PL + A.PR;
    if (A.src != SRC_QUERY) {
        int64_t a, b;
        if (A.src == SRC_TRIANGLE) {
            tri_index(t, A.p, a, b);
            if (A.perm) {
                a = A.perm[a];
                b = A.perm[b];
            }
        } else {
            a = A.pa[t];
            b = A.pb[t];
        }
        g.a = a;
        g.b = b;
        const int64_t oa = A.offsets[a], ob = A.offsets[b];
        s0 = A.padded + (oa - o0) + a * pad + A.PL;
        n0 = A.offsets[a + 1] - oa;
        s1 = A.padded + (ob - o0) + b * pad + A.PL;
        n1 = A.offsets[b + 1] - ob;
    } else {
        const int64_t s = A.perm ? A.perm[t] : t;
        g.a = -1;
        g.b = s;
        const int64_t ob = A.offsets[s];
        s0 = A.padded + A.qbase;
        n0 = A.qlen;
        s1 = A.padded + (ob - o0) + s * pad + A.PL;
        n1 = A.offsets[s + 1] - ob;
    }
    if (n0 <= n1) {
        g.x = s0; g.n = (int32_t)n0; g.y = s1; g.m = (int32_t)n1;
    } else {
        g.x = s1; g.n = (int32_t)n1; g.y = s0; g.m = (int32_t)n0;
    }
    const int32_t diff = g.m - g.n;
    const int32_t wb = A.wpermille > 0 ? (int32_t)((int64_t)A.wpermille * g.m / 1000) : A.window;
    int32_t w;
    if (wb < 0) w = g.m - 1;
    else if (A.strict) w = wb;
    else w = wb > diff ? wb : diff;
    if (w > g.m - 1) w = g.m - 1;  // |i-j| <= m-1 always holds for n <= m
    g.w = w;
    g.trivial = diff > w;
    g.kres = diff + w;
}

__device__ __forceinline__ void write_result(const BandArgs &A, int64_t t, const PairGeom &g,
                                             float r)
{
    if (A.out_mode == OUT_FULL) {
        A.out[g.a * A.p + g.b] = r;
        A.out[g.b * A.p + g.a] = r;
    } else if (A.out_mode == OUT_PACKED || A.out_mode == OUT_LIST) {
        A.out[t] = r;
    } else {
        A.out[g.b] = r;
    }
}

// Work sources of the persistent kernels.  StaticSrc: every pair of one call,
// strided over the lane groups of the grid.  QueueSrc: items (job << 40 | pair)
// of many jobs, sorted by estimated cost (largest first), popped from a shared
// counter by lane 0 of a group and broadcast to the group.
struct StaticSrc {
    static constexpr bool kQueue = false;
    BandArgs A;
    int32_t G, log2G;
    __device__ __forceinline__ const BandArgs &job(int) const { return A; }
};

struct QueueSrc {
    static constexpr bool kQueue = true;
    const BandArgs *jobs;
    const uint64_t *items;
    int64_t n_items;
    unsigned long long *head;
    int32_t G, log2G;
    __device__ __forceinline__ const BandArgs &job(int j) const { return jobs[j]; }
};

constexpr int kItemShift = 40;

// Next (job, pair) of a group; false when the source is exhausted.  `cursor`
// is the group's position in the static stride sequence.  All G lanes of the
// group call it together (gmask names them).
__device__ __forceinline__ bool next_item(const StaticSrc &src, int64_t &cursor, int64_t ngroups,
                                          unsigned, int, int &job, int64_t &t)
{
    cursor += ngroups;
    job = 0;
    t = cursor;
    return cursor < src.A.n_pairs;
}

__device__ __forceinline__ bool next_item(const QueueSrc &src, int64_t &, int64_t, unsigned gmask,
                                          int l, int &job, int64_t &t)
{
    unsigned long long idx = 0;
    if (l == 0) idx = atomicAdd(src.head, 1ull);
    idx = __shfl_sync(gmask, idx, 0, src.G);
    if ((int64_t)idx >= src.n_items) return false;
    const uint64_t it = src.items[idx];
    job = (int)(it >> kItemShift);
    t = (int64_t)(it & ((1ull << kItemShift) - 1));
    return true;
}

// One step T of a group (unrolled position s of a K-step block).  CHECK
// selects the ramp version, in which lanes whose row T-l lies outside [1, n]
// keep their state; without it every lane of the warp is inside its pair.
//
// Boundary values enter as additions of +inf or 0 (lmask: +inf on lane 0,
// rmask: +inf on lane G-1, tmask: +inf on band slots beyond 2w); every value
// is >= +0, so adding +0 is exact and the adds run on the FMA pipe, leaving
// the ALU pipe to the three-input minimum.
//
// Each lane fetches its own next x and y values from the padded series one
// step ahead: px[T'] = x_{T'+1-l} and py[T'] = the y value that enters its
// last slot after step T' (pb* are those pointers advanced to the block).  A
// step lasts hundreds of cycles, enough to cover an L2 hit.
template <int K, int MT, bool CHECK>
__device__ __forceinline__ void band_step(const int s, const int T, const int l, const int G,
                                          const bool have, const int n, float (&prev)[K],
                                          float (&ywin)[K], const float (&tmask)[MT],
                                          const float lmask, const float rmask, float &xr,
                                          float &left_in, float &pxa, float &pya,
                                          const float *pbx, const float *pby)
{
    const unsigned FULL = 0xffffffffu;
    bool active = true;
    if (CHECK) {
        const int row = T - l;
        active = have && row >= 1 && row <= n;
    }
    // first slot: its left value is lane l-1's last slot of this row (last step)
    float v0 = prev[0];
    if (active) {
        v0 = dtw_cell(xr, ywin[s % K], fmin3(prev[0], prev[1], left_in));
        if (MT == K) v0 = __fadd_rn(v0, tmask[0]);
    }
    // lane l+1 just computed (row-1, its first slot): our last slot's up value
    const float up_last = __fadd_rn(__shfl_down_sync(FULL, v0, 1, G), rmask);
    if (active) {
        prev[0] = v0;
        float c = v0;
#pragma unroll
        for (int t = 1; t < K; ++t) {
            const float up = (t + 1 < K) ? prev[t + 1] : up_last;
            float v = dtw_cell(xr, ywin[(s + t) % K], fmin3(prev[t], up, c));
            if (t >= K - MT) v = __fadd_rn(v, tmask[t - (K - MT)]);
            prev[t] = v;
            c = v;
        }
    }
    left_in = __fadd_rn(__shfl_up_sync(FULL, prev[K - 1], 1, G), lmask);
    ywin[s % K] = pya;
    xr = pxa;
    if (!CHECK || have) {
        pya = __ldg(pby + s + 2);
        pxa = __ldg(pbx + s + 2);
    }
}

// Resident blocks per SM the register allocation aims for: 4 (64 registers)
// for the narrow shapes, 3 where 64 registers would spill, 2 for K > 20 (the
// work-queue source holds a few more registers than the static stride).
template <int K, int MT, bool QUEUE>
constexpr int band_min_blocks()
{
#ifdef DTWGB_BAND_MINB
    return DTWGB_BAND_MINB;
#else
    return QUEUE ? (K <= 4 ? 4 : 3) : ((K <= 13 && MT == 1) || K <= 8 ? 4 : (K <= 20 ? 3 : 2));
#endif
}

template <int K, int MT, typename Src>
__global__ void __launch_bounds__(256, (band_min_blocks<K, MT, Src::kQueue>()))
    dtw_band_kernel(const Src src)
{
    static_assert(K >= 2 && MT >= 1 && MT <= K, "bad band kernel shape");
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
    float prev[K], ywin[K], tmask[MT];
    float xr = 0.f, left_in = INF, pxa = 0.f, pya = 0.f;
    // px[T] = x_{T+1-l}, py[T] = y_{T+l(K-1)+K-w}; both advance by K per block
    const float *px = nullptr, *py = nullptr;
    bool have = false;
    int n = 0, blk = 0, nblk = 0;

    while (true) {
        if (!have) {
            // next pair of this group; pairs the strict band cannot join are +inf
            PairGeom g;
            while (next_item(src, cursor, ngroups, gmask, l, job, pair)) {
                const BandArgs &J = src.job(job);
                pair_geometry(J, pair, g);
                if (!g.trivial) { have = true; break; }
                if (first) write_result(J, pair, g, INF);
            }
            if (have) {
                const int w = g.w;
                // row 0: c_{0,0} = 0 (band offset w), every other c_{0,j} = +inf;
                // y window of step 1: y_j for j = 1 + l(K-1) + t - w (padding gives +inf)
#pragma unroll
                for (int t = 0; t < K; ++t) {
                    prev[t] = (kbase + t == w) ? 0.f : INF;
                    ywin[t] = __ldg(g.y + (l * (K - 1) + t - w));
                }
#pragma unroll
                for (int u = 0; u < MT; ++u)
                    tmask[u] = (kbase + K - MT + u > 2 * w) ? INF : 0.f;
                px = g.x - l;
                py = g.y + (l * (K - 1) + K - 1 - w);
                xr = __ldg(px);  // x_{1-l}: the row of step 1
                left_in = INF;
                pxa = __ldg(px + 1);
                pya = __ldg(py + 1);
                n = g.n;
                blk = 0;
                nblk = (n + G - 1 + K - 1) / K;
            }
        }
        if (__all_sync(FULL, !have)) break;

        const int T0 = blk * K;
        const bool fast = __all_sync(FULL, have && T0 >= G - 1 && T0 + K <= n);
        if (fast) {
#pragma unroll
            for (int s = 0; s < K; ++s)
                band_step<K, MT, false>(s, T0 + s + 1, l, G, true, n, prev, ywin, tmask, lmask,
                                        rmask, xr, left_in, pxa, pya, px, py);
        } else {
#pragma unroll
            for (int s = 0; s < K; ++s)
                band_step<K, MT, true>(s, T0 + s + 1, l, G, have, n, prev, ywin, tmask, lmask,
                                       rmask, xr, left_in, pxa, pya, px, py);
        }
        px += K;
        py += K;

        if (have && ++blk == nblk) {
            // every lane now holds row n; c_{n,m} sits at band offset kres
            const BandArgs &J = src.job(job);
            PairGeom g;
            pair_geometry(J, pair, g);
            const int lres = g.kres / K, tres = g.kres - lres * K;
            float r = prev[0];
#pragma unroll
            for (int t = 1; t < K; ++t)
                if (t == tres) r = prev[t];
            if (l == lres) write_result(J, pair, g, r);
            have = false;
        }
    }
}

// ------------------------------------------------------------------------
// Two pairs per group.  Each lane carries two independent DPs (pair slot A in
// the .x halves, slot B in the .y halves of float2 registers).  The
// subtraction, the fused multiply-add and the +inf/+0 mask adds of the two
// slots are single packed f32x2 instructions (IEEE per half, so every value
// is bit-identical to the one-pair kernel); the three-input minimum stays
// scalar.  Two chains per lane also double the independent work per warp.
// Each slot takes its next pair at a block boundary on its own.

template <int C>
__device__ __forceinline__ float &half(float2 &v) { return C == 0 ? v.x : v.y; }

__device__ __forceinline__ float2 f2_cell(float2 x, float2 y, float2 m)
{
    const float2 d = __ffma2_rn(make_float2(-1.f, -1.f), y, x);  // x - y, one rounding
    return __ffma2_rn(d, d, m);
}

__device__ __forceinline__ float2 f2_min3(float2 a, float2 b, float2 c)
{
    return make_float2(fmin3(a.x, b.x, c.x), fmin3(a.y, b.y, c.y));
}

__device__ __forceinline__ float2 f2_shfl_down(float2 v, int G)
{
    return make_float2(__shfl_down_sync(0xffffffffu, v.x, 1, G),
                       __shfl_down_sync(0xffffffffu, v.y, 1, G));
}

__device__ __forceinline__ float2 f2_shfl_up(float2 v, int G)
{
    return make_float2(__shfl_up_sync(0xffffffffu, v.x, 1, G),
                       __shfl_up_sync(0xffffffffu, v.y, 1, G));
}

// Per-slot bookkeeping (the DP state itself lives in the float2 arrays).
struct SlotState {
    const float *px, *py;  // px[T] = x_{T+1-l}, py[T] = y_{T+l(K-1)+K-w}; advance by K per block
    int64_t pair;
    int n, blk, nblk;
    bool have;
};

// Take the next pair of the group into slot C (and write +inf for pairs the
// strict band cannot join).  Leaves s.have false when the group has no pairs left.
template <int K, int MT, int C>
__device__ __forceinline__ void slot_setup(const BandArgs &A, int64_t &next, int64_t ngroups,
                                           int l, int G, bool first, SlotState &s,
                                           float2 (&prev)[K], float2 (&ywin)[K],
                                           float2 (&tmask)[MT], float2 &xr, float2 &left_in,
                                           float2 &pxa, float2 &pya)
{
    const float INF = finf();
    PairGeom g;
    s.have = false;
    while (next < A.n_pairs) {
        const int64_t t = next;
        next += ngroups;
        pair_geometry(A, t, g);
        if (!g.trivial) {
            s.have = true;
            s.pair = t;
            break;
        }
        if (first) write_result(A, t, g, INF);
    }
    if (!s.have) return;
    const int w = g.w, kbase = l * K;
#pragma unroll
    for (int t = 0; t < K; ++t) {
        half<C>(prev[t]) = (kbase + t == w) ? 0.f : INF;
        half<C>(ywin[t]) = __ldg(g.y + (l * (K - 1) + t - w));
    }
#pragma unroll
    for (int u = 0; u < MT; ++u) half<C>(tmask[u]) = (kbase + K - MT + u > 2 * w) ? INF : 0.f;
    s.px = g.x - l;
    s.py = g.y + (l * (K - 1) + K - 1 - w);
    half<C>(xr) = __ldg(s.px);
    half<C>(left_in) = INF;
    half<C>(pxa) = __ldg(s.px + 1);
    half<C>(pya) = __ldg(s.py + 1);
    s.n = g.n;
    s.blk = 0;
    s.nblk = (g.n + G - 1 + K - 1) / K;
}

template <int K, int C>
__device__ __forceinline__ void slot_finish(const BandArgs &A, int l, SlotState &s,
                                            float2 (&prev)[K])
{
    PairGeom g;
    pair_geometry(A, s.pair, g);
    const int lres = g.kres / K, tres = g.kres - lres * K;
    float r = half<C>(prev[0]);
#pragma unroll
    for (int t = 1; t < K; ++t)
        if (t == tres) r = half<C>(prev[t]);
    if (l == lres) write_result(A, s.pair, g, r);
    s.have = false;
}

template <int K, int MT, bool CHECK>
__device__ __forceinline__ void band2_step(const int s, const int l, const int G,
                                           const SlotState &a, const SlotState &b,
                                           float2 (&prev)[K], float2 (&ywin)[K],
                                           const float2 (&tmask)[MT], const float2 lmask,
                                           const float2 rmask, float2 &xr, float2 &left_in,
                                           float2 &pxa, float2 &pya)
{
    bool actA = true, actB = true;
    if (CHECK) {
        const int ra = a.blk * K + s + 1 - l, rb = b.blk * K + s + 1 - l;
        actA = a.have && ra >= 1 && ra <= a.n;
        actB = b.have && rb >= 1 && rb <= b.n;
    }
    float2 v0 = f2_cell(xr, ywin[s % K], f2_min3(prev[0], prev[1], left_in));
    if (MT == K) v0 = __fadd2_rn(v0, tmask[0]);
    if (CHECK) {
        v0.x = actA ? v0.x : prev[0].x;
        v0.y = actB ? v0.y : prev[0].y;
    }
    const float2 up_last = __fadd2_rn(f2_shfl_down(v0, G), rmask);
    prev[0] = v0;
    float2 c = v0;
#pragma unroll
    for (int t = 1; t < K; ++t) {
        const float2 up = (t + 1 < K) ? prev[t + 1] : up_last;
        float2 v = f2_cell(xr, ywin[(s + t) % K], f2_min3(prev[t], up, c));
        if (t >= K - MT) v = __fadd2_rn(v, tmask[t - (K - MT)]);
        if (CHECK) {
            v.x = actA ? v.x : prev[t].x;
            v.y = actB ? v.y : prev[t].y;
        }
        prev[t] = v;
        c = v;
    }
    left_in = __fadd2_rn(f2_shfl_up(prev[K - 1], G), lmask);
    ywin[s % K] = pya;
    xr = pxa;
    if (!CHECK || a.have) {
        pya.x = __ldg(a.py + s + 2);
        pxa.x = __ldg(a.px + s + 2);
    }
    if (!CHECK || b.have) {
        pya.y = __ldg(b.py + s + 2);
        pxa.y = __ldg(b.px + s + 2);
    }
}

template <int K, int MT>
constexpr int band2_min_blocks()
{
#ifdef DTWGB_BAND2_MINB
    return DTWGB_BAND2_MINB;
#else
    return 2;
#endif
}

template <int K, int MT>
__global__ void __launch_bounds__(256, band2_min_blocks<K, MT>()) dtw_band2_kernel(const BandArgs A)
{
    static_assert(K >= 2 && MT >= 1 && MT <= K, "bad band kernel shape");
    const float INF = finf();
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int G = A.G;
    const int l = lane & (G - 1);
    const int gpw = 32 >> A.log2G;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t ngroups = nwarps * gpw;
    const bool first = (l == 0), last = (l == G - 1);
    const float2 lmask = first ? make_float2(INF, INF) : make_float2(0.f, 0.f);
    const float2 rmask = last ? make_float2(INF, INF) : make_float2(0.f, 0.f);

    int64_t next = warp * gpw + (lane >> A.log2G);
    float2 prev[K], ywin[K], tmask[MT];
    float2 xr = make_float2(0.f, 0.f), left_in = make_float2(INF, INF);
    float2 pxa = xr, pya = xr;
    SlotState a, b;
    a.have = b.have = false;
    a.px = a.py = b.px = b.py = A.padded;
    a.n = b.n = a.blk = b.blk = a.nblk = b.nblk = 0;
    a.pair = b.pair = 0;
#pragma unroll
    for (int t = 0; t < K; ++t) prev[t] = ywin[t] = make_float2(INF, INF);
#pragma unroll
    for (int u = 0; u < MT; ++u) tmask[u] = make_float2(0.f, 0.f);

    while (true) {
        if (!a.have)
            slot_setup<K, MT, 0>(A, next, ngroups, l, G, first, a, prev, ywin, tmask, xr, left_in,
                                 pxa, pya);
        if (!b.have)
            slot_setup<K, MT, 1>(A, next, ngroups, l, G, first, b, prev, ywin, tmask, xr, left_in,
                                 pxa, pya);
        if (__all_sync(FULL, !a.have && !b.have)) break;

        const int T0a = a.blk * K, T0b = b.blk * K;
        const bool fast = __all_sync(FULL, a.have && b.have && T0a >= G - 1 && T0a + K <= a.n &&
                                               T0b >= G - 1 && T0b + K <= b.n);
        if (fast) {
#pragma unroll
            for (int s = 0; s < K; ++s)
                band2_step<K, MT, false>(s, l, G, a, b, prev, ywin, tmask, lmask, rmask, xr,
                                         left_in, pxa, pya);
        } else {
#pragma unroll
            for (int s = 0; s < K; ++s)
                band2_step<K, MT, true>(s, l, G, a, b, prev, ywin, tmask, lmask, rmask, xr,
                                        left_in, pxa, pya);
        }
        a.px += K;
        a.py += K;
        b.px += K;
        b.py += K;
        if (a.have && ++a.blk == a.nblk) slot_finish<K, 0>(A, l, a, prev);
        if (b.have && ++b.blk == b.nblk) slot_finish<K, 1>(A, l, b, prev);
    }
}

// Persistent grid for `items` work items at G lanes per item: SMs x resident
// blocks, fewer if there is less work.
// Persistent grid: SMs x resident blocks, each lane group striding over the
// items (the work queues of a batch, which balance by popping).  With
// `persistent` false the grid has one block per groups_per_block items, so
// each lane group takes one item and exits: the single-call launches use it,
// because a block's groups then take consecutive triangle pairs, which share
// their row series in L1 (2000 x 512, w = 51: 12.7 ms against 13.2 ms), and
// because kernels of other (higher-priority) streams get SMs as blocks retire
// instead of after the whole launch.
template <typename Kern, typename Src>
inline int launch_kernel(Kern kern, const Src &src, int64_t items, int G, cudaStream_t st,
                         int threads = kThreads, bool persistent = true)
{
    int dev = 0, sms = 0, per_sm = 0;
    DTWGB_CUDA(cudaGetDevice(&dev));
    DTWGB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    DTWGB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, 0));
    if (per_sm < 1) per_sm = 1;
    const int64_t groups_per_block = (threads / 32) * (32 / G);
    int64_t need = (items + groups_per_block - 1) / groups_per_block;
    int64_t blocks = (int64_t)sms * per_sm;
    if (need < blocks || !persistent) blocks = need;
    if (blocks > 0x7fffffffLL) blocks = 0x7fffffffLL;  // the stride loop covers the rest
    if (blocks < 1) blocks = 1;
    kern<<<(unsigned)blocks, threads, 0, st>>>(src);
    DTWGB_CUDA(cudaGetLastError());
    return DTW_OK;
}

// Launch the one-pair-per-lane (band1.cu) or two-pairs-per-lane (band2.cu)
// kernel of shape (K, MT) with A.G lanes per pair.
int launch_band1(const BandArgs &A, int K, int MT, cudaStream_t st);
int launch_band2(const BandArgs &A, int K, int MT, cudaStream_t st);
// The one-pair-per-lane kernel on a work queue (batch.cu).
int launch_band1_queue(const QueueSrc &src, int K, int MT, cudaStream_t st);

// Strip kernel (strip.cu) for bands wider than the rotated kernel holds: one
// warp per pair, `bnd` holds one column buffer of `bnd_stride` floats per warp
// of the grid (warps_total = blocks * 8).
int launch_strip(const BandArgs &A, int K, float *bnd, int64_t bnd_stride, int64_t warps_total,
                 cudaStream_t st);
int launch_strip_queue(const QueueSrc &src, int K, float *bnd, int64_t bnd_stride,
                       int64_t warps_total, cudaStream_t st);
// Warps of a persistent strip grid for n_pairs pairs (a multiple of 8).
int strip_warps(int K, int64_t n_pairs, int64_t *warps_total);
// Floats per warp of the strip kernel's column buffer for series of up to
// maxlen values: rows -32 .. maxlen + 35 (the skewed wavefront stores up to 31
// rows above a strip's first row and reads up to 33 rows below its last).
inline int64_t strip_bnd_stride(int64_t maxlen) { return (maxlen + 68 + 31) / 32 * 32; }

// Staging of a set / one series into the +inf-padded layout, and the zero
// diagonal of a full matrix (dtw_band.cu).
int launch_stage_set(const float *values, const int64_t *offsets, int32_t p, int32_t PL,
                     int32_t PR, float *padded, cudaStream_t st);
int launch_stage_one(const float *v, int64_t len, int32_t PL, int32_t PR, float *dst,
                     cudaStream_t st);
int launch_zero_diagonal(float *D, int64_t p, cudaStream_t st);

// A set staged once for many pair lists (dtw_band.cu): the kernel shape, the
// padded copy and the strip buffers are kept between list launches.
struct DtwListCtx {
    BandArgs A;
    int kind, K, G, MT;
    void *padded = nullptr, *bnd = nullptr;
    int64_t bnd_stride = 0, warps = 0, bnd_pairs = 0;
    int64_t maxlen = 0;
};
int dtw_list_prepare(const float *values, const int64_t *offsets, const int64_t *offsets_host,
                     int32_t p, int32_t window, uint32_t flags, DtwListCtx *ctx, cudaStream_t st);
int dtw_list_run(DtwListCtx *ctx, const int32_t *pa, const int32_t *pb, int64_t npairs, float *out,
                 cudaStream_t st);
void dtw_list_release(DtwListCtx *ctx, cudaStream_t st);

// Instruction-count estimates per pair used to pick shapes (dtw_band.cu).
double cost_rotated(int n, int K, int G, int MT);
double cost_strip(int n, int m, int w, int K);

// Slots per lane of the compiled rotated kernels, and the masked tail that a
// shape with G*K slots needs for a band row of `W` cells when every pair has
// that band: the G*K - W slots beyond the band sit at the top of the last lane;
// they are forced to +inf by adding +inf on the last MT slots of every lane (0
// elsewhere), so MT must be at least the masked count: 1, 4, 8, or all K slots.
// The static-stride launch (one set or query) has a slot count for every K in
// 8..24, so that some G in {8, 16} fits any band row of 65..384 cells to within
// a few slots; the work-queue launch (batch.cu) has fewer, and tunes among them.
constexpr int kRotKsQueue[] = {4, 8, 10, 12, 13, 16, 18, 20};
constexpr int kRotKsStatic[] = {4,  8,  9,  10, 11, 12, 13, 14, 15,
                                16, 17, 18, 19, 20, 21, 22, 23, 24};
inline int rot_masked_tail(int K, int G, int W)
{
    const int masked = G * K - W;
    if (masked <= 1) return 1;
    if (masked <= 4 && K > 4) return 4;
    if (masked <= 8 && K > 8) return 8;
    return K;
}
// Large K are compiled with tails of 1, 4 and 8 slots only (a full tail would spill).
inline bool rot_shape_compiled(int K, int MT, bool queue)
{
    bool listed = false;
    if (queue) {
        for (int k : kRotKsQueue) listed = listed || k == K;
        return listed && !(K >= 18 && MT == K);
    }
    for (int k : kRotKsStatic) listed = listed || k == K;
    return listed && !(K >= 17 && MT == K);
}

// (K, MT) of the rotated kernels compiled for both launches (band1.cu, band1q.cu)
#define DTWGB_BAND_SHAPES(X)                                                                    \
    X(4, 1) X(4, 4) X(8, 1) X(8, 4) X(8, 8) X(10, 1) X(10, 4) X(10, 8) X(10, 10) X(12, 1)        \
        X(12, 4) X(12, 8) X(12, 12) X(13, 1) X(13, 4) X(13, 8) X(13, 13) X(16, 1) X(16, 4)      \
            X(16, 8) X(16, 16) X(18, 1) X(18, 4) X(18, 8) X(20, 1) X(20, 4) X(20, 8)
// ... and the further ones of the static-stride launch (band1w.cu)
#define DTWGB_BAND_SHAPES_WIDE(X)                                                               \
    X(9, 1) X(9, 4) X(9, 8) X(9, 9) X(11, 1) X(11, 4) X(11, 8) X(11, 11) X(14, 1) X(14, 4)       \
        X(14, 8) X(14, 14) X(15, 1) X(15, 4) X(15, 8) X(15, 15) X(17, 1) X(17, 4) X(17, 8)      \
            X(19, 1) X(19, 4) X(19, 8) X(21, 1) X(21, 4) X(21, 8) X(22, 1) X(22, 4) X(22, 8)    \
                X(23, 1) X(23, 4) X(23, 8) X(24, 1) X(24, 4) X(24, 8)
int launch_band1_wide(const BandArgs &A, int K, int MT, cudaStream_t st);

}  // namespace dtwgb
