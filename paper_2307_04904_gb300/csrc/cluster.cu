// cluster.cu -- cluster-quality reporting and PAM over D (dtwgb_cluster.h).
//
// Every quantity here is a sum over a set of points of one row of D: the
// cluster sums of the silhouette, the two FastPAM1 terms of a swap, the BUILD
// gains.  D is symmetric, so the sum over row i's entries D[i][j], j in a set,
// is the sum down the rows j of the set in column i: contiguous, coalesced
// reads.  One kernel does all three (segred_kernel): the rows of every group (a
// cluster's members in index order, or all points) are cut into segments of at
// most L rows; block (column tile, segment) stages its rows' offsets and
// per-row scalars in shared memory and streams the rows, each thread owning VEC
// consecutive columns with a batch of loads in flight; the segment's
// Kahan-compensated float32 sums become float64 partials part[segment][column],
// which small kernels add in segment order.  One read of D per pass, spread
// over many blocks, and deterministic.
//
// Silhouette: members listed per cluster, segment sums of D, s(i) in float64;
// for very large n * (segments) one block per row gathers the members instead.
// PAM SWAP: nearest and second-nearest medoid per point, members per nearest
// medoid, the two FastPAM1 terms per (candidate, cluster) as segment sums,
// then per candidate its k deltas and a two-level argmin.  BUILD: k steps of a
// segment sum over all rows and an argmin.
#include <algorithm>
#include <vector>

#include "../../include/dtwgb_cluster.h"
#include "common.cuh"

namespace dtwgb {
namespace {

constexpr int kSilThreads = 256;
constexpr int kSilMaxK = 4096;
constexpr int kSilParts = 64;
constexpr int kSegThreads = 256;
constexpr int kSegStage = 512;  // rows staged in shared memory at a time

// Rows per segment: about eight blocks of the reduction per SM over all rows
// (a multiple of 16, from 64 to 512), so that the loads in flight cover HBM's
// latency while the partials stay a few percent of D.
int seg_rows(int64_t n)
{
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
        sms = 148;
    const int64_t tiles = (n + 4 * kSegThreads - 1) / (4 * kSegThreads);
    const int64_t L = n * tiles / (8 * (int64_t)sms) / 16 * 16;
    return (int)std::max<int64_t>(64, std::min<int64_t>(L, kSegStage));
}

// perm[cstart[c] + r] = the r-th member of cluster c in index order; one block
// of 1024 threads per cluster, 8192 labels per round: chunk u of the round is
// read by all threads (coalesced), a ballot per warp and chunk counts the
// members, warp u scans chunk u's 32 warp counts, and every member gets its
// slot.  With d1 given, the members' d1 and d2 are written in the same order
// (pd1, pd2), so that readers of a member list need no second, dependent gather.
constexpr int kMemThreads = 1024;
__global__ void __launch_bounds__(kMemThreads)
    sil_members_kernel(const int32_t *__restrict__ labels, int n, const int32_t *__restrict__ cstart,
                       int32_t *__restrict__ perm, const float *__restrict__ d1,
                       const float *__restrict__ d2, float *__restrict__ pd1, float *__restrict__ pd2)
{
    constexpr int kU = 8;
    __shared__ int wsum[kU][32], excl[kU][32], tot[kU];
    const int c = blockIdx.x, tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    int base = cstart[c];
    for (int j0 = 0; j0 < n; j0 += kU * kMemThreads) {
        unsigned bal[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int j = j0 + u * kMemThreads + tid;
            bal[u] = __ballot_sync(0xffffffffu, j < n && labels[j] == c);
            if (lane == 0) wsum[u][w] = __popc(bal[u]);
        }
        __syncthreads();
        if (w < kU) {  // warp u: exclusive scan of chunk u's warp counts
            const int v = wsum[w][lane];
            int incl = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            excl[w][lane] = incl - v;
            if (lane == 31) tot[w] = incl;
        }
        __syncthreads();
        int run = base;
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            if ((bal[u] >> lane) & 1u) {
                const int pos = run + excl[u][w] + __popc(bal[u] & ((1u << lane) - 1u));
                const int j = j0 + u * kMemThreads + tid;
                perm[pos] = j;
                if (d1) {
                    pd1[pos] = d1[j];
                    pd2[pos] = d2[j];
                }
            }
            run += tot[u];
        }
        base = run;
        __syncthreads();
    }
}

// From the cluster sizes: cstart (exclusive prefix), and the segments of at
// most L members of every cluster in cluster order; segbase[c] = the first
// segment of cluster c, segbase[k] = *nseg = their number.  One block; thread t
// takes a contiguous run of clusters, and shuffle scans give the prefixes.
__global__ void __launch_bounds__(256)
    seg_table_kernel(const int32_t *__restrict__ cnt, int k, int L, int32_t *__restrict__ cstart,
                     int32_t *__restrict__ segbase, int2 *__restrict__ segs, int32_t *__restrict__ nseg)
{
    __shared__ int wm[8], ws[8];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, per = (k + 255) / 256;
    const int c0 = min(k, tid * per), c1 = min(k, c0 + per);
    int m = 0, s = 0;
    for (int c = c0; c < c1; ++c) {
        m += cnt[c];
        s += (cnt[c] + L - 1) / L;
    }
    int im = m, is = s;  // inclusive scans within the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int a = __shfl_up_sync(0xffffffffu, im, o), b = __shfl_up_sync(0xffffffffu, is, o);
        if (lane >= o) {
            im += a;
            is += b;
        }
    }
    if (lane == 31) {
        wm[w] = im;
        ws[w] = is;
    }
    __syncthreads();
    int bm = 0, bs = 0, tm = 0, ts = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        bm += q < w ? wm[q] : 0;
        bs += q < w ? ws[q] : 0;
        tm += wm[q];
        ts += ws[q];
    }
    if (tid == 0) {
        cstart[k] = tm;
        segbase[k] = ts;
        *nseg = ts;
    }
    m = bm + im - m;  // exclusive prefix of this thread's run
    s = bs + is - s;
    for (int c = c0; c < c1; ++c) {
        cstart[c] = m;
        segbase[c] = s;
        for (int lo = m; lo < m + cnt[c]; lo += L) segs[s++] = make_int2(lo, min(lo + L, m + cnt[c]));
        m += cnt[c];
    }
}

enum SegMode { kSegSum = 0, kSegMinD1 = 1, kSegPam = 2 };

__device__ __forceinline__ void kahan_add(float &s, float &c, float x)
{
    const float y = __fsub_rn(x, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
}

// kahan_add on two columns at once with packed float32 pairs (each half rounds
// exactly as the scalar form: fma(-1, b, a) is a - b with one rounding)
__device__ __forceinline__ void kahan_add2(float2 &s, float2 &c, float2 x)
{
    const float2 m1 = make_float2(-1.f, -1.f);
    const float2 y = __ffma2_rn(m1, c, x);
    const float2 t = __fadd2_rn(s, y);
    c = __ffma2_rn(m1, y, __ffma2_rn(m1, s, t));
    s = t;
}

// the terms of one entry d = D[j][o] for row slot q
template <int MODE>
__device__ __forceinline__ void seg_take(float d, float e1, float e2, float &a, float &ca, float &b,
                                         float &cb)
{
    if (MODE == kSegSum) {
        kahan_add(a, ca, d);
    } else if (MODE == kSegMinD1) {
        kahan_add(a, ca, fminf(d, e1));
    } else {
        kahan_add(a, ca, fminf(0.f, __fsub_rn(d, e1)));
        kahan_add(b, cb, __fsub_rn(fminf(d, e2), e1));
    }
}

template <int MODE>
__device__ __forceinline__ void seg_take2(float2 d, float e1, float e2, float2 &a, float2 &ca,
                                          float2 &b, float2 &cb)
{
    if (MODE == kSegSum) {
        kahan_add2(a, ca, d);
    } else if (MODE == kSegMinD1) {
        kahan_add2(a, ca, make_float2(fminf(d.x, e1), fminf(d.y, e1)));
    } else {
        const float2 m1 = make_float2(-1.f, -1.f), ee = make_float2(e1, e1);
        const float2 u = __ffma2_rn(m1, ee, d);  // d - e1
        kahan_add2(a, ca, make_float2(fminf(0.f, u.x), fminf(0.f, u.y)));
        kahan_add2(b, cb, __ffma2_rn(m1, ee, make_float2(fminf(d.x, e2), fminf(d.y, e2))));
    }
}

// Segment sums down the rows of D.  Segment s = blockIdx.y covers the member
// positions [lo, hi) of one group: with `segs`, segs[s] (blocks with s >= *nseg
// do nothing); without, the rows [s L, min((s + 1) L, n)).  Position q in
// [lo, hi) is row j = perm[q], or q itself when perm is NULL; d1 and d2 are
// given per position (d1[q] is row j's value).  For every column o:
//   kSegSum    part1[s][o] = sum_q D[j][o]
//   kSegMinD1  part1[s][o] = sum_q min(D[j][o], d1[q])
//   kSegPam    part1[s][o] = sum_q min(0, D[j][o] - d1[q]),
//              part2[s][o] = sum_q min(D[j][o], d2[q]) - d1[q]
// as Kahan-compensated float32 over the rows in order.  VEC = 4 (four columns
// per thread, float4 loads, packed arithmetic) needs n % 4 == 0 and a 16-byte
// aligned D; both widths give the same bits.
template <int MODE, int VEC>
__global__ void __launch_bounds__(kSegThreads, 4)
    segred_kernel(const float *__restrict__ D, int n, int L, const int32_t *__restrict__ perm,
                  const int2 *__restrict__ segs, const int32_t *__restrict__ nseg,
                  const float *__restrict__ d1, const float *__restrict__ d2,
                  double *__restrict__ part1, double *__restrict__ part2)
{
    constexpr int U = VEC == 4 ? 4 : 8;  // loads in flight per thread
    constexpr int H = VEC == 4 ? 2 : 1;  // float2 pairs (VEC = 4) or scalars (VEC = 1)
    __shared__ int64_t rowoff[kSegStage];
    __shared__ float e1[MODE == kSegSum ? 1 : kSegStage];
    __shared__ float e2[MODE == kSegPam ? kSegStage : 1];
    const int s = blockIdx.y;
    int lo, hi;
    if (segs) {
        if (s >= *nseg) return;
        const int2 g = segs[s];
        lo = g.x;
        hi = g.y;
    } else {
        lo = s * L;
        hi = min(lo + L, n);
    }
    const int o = (blockIdx.x * kSegThreads + threadIdx.x) * VEC;
    const bool active = o < n;
    const float *Do = D + (active ? o : 0);
    float2 a2[H], ca2[H], b2[H], cb2[H];  // VEC = 4
    float a = 0.f, ca = 0.f, b = 0.f, cb = 0.f;  // VEC = 1
#pragma unroll
    for (int h = 0; h < H; ++h) a2[h] = ca2[h] = b2[h] = cb2[h] = make_float2(0.f, 0.f);

    for (int c0 = lo; c0 < hi; c0 += kSegStage) {
        const int m = min(kSegStage, hi - c0);
        __syncthreads();  // the previous stage is consumed
        for (int q = threadIdx.x; q < m; q += kSegThreads) {
            const int j = perm ? perm[c0 + q] : c0 + q;
            rowoff[q] = (int64_t)j * n;
            if (MODE != kSegSum) e1[q] = d1[c0 + q];
            if (MODE == kSegPam) e2[q] = d2[c0 + q];
        }
        __syncthreads();
        if (!active) continue;
        auto ev1 = [&](int q) { return MODE == kSegSum ? 0.f : e1[q]; };
        auto ev2 = [&](int q) { return MODE == kSegPam ? e2[q] : 0.f; };
        if constexpr (VEC == 4) {
            auto take = [&](const float4 &x, int q) {
                const float f1 = ev1(q), f2 = ev2(q);
                seg_take2<MODE>(make_float2(x.x, x.y), f1, f2, a2[0], ca2[0], b2[0], cb2[0]);
                seg_take2<MODE>(make_float2(x.z, x.w), f1, f2, a2[1], ca2[1], b2[1], cb2[1]);
            };
            int q = 0;
            for (; q + U <= m; q += U) {
                float4 x[U];
#pragma unroll
                for (int u = 0; u < U; ++u) x[u] = *reinterpret_cast<const float4 *>(Do + rowoff[q + u]);
#pragma unroll
                for (int u = 0; u < U; ++u) take(x[u], q + u);
            }
            for (; q < m; ++q) take(*reinterpret_cast<const float4 *>(Do + rowoff[q]), q);
        } else {
            int q = 0;
            for (; q + U <= m; q += U) {
                float x[U];
#pragma unroll
                for (int u = 0; u < U; ++u) x[u] = Do[rowoff[q + u]];
#pragma unroll
                for (int u = 0; u < U; ++u) seg_take<MODE>(x[u], ev1(q + u), ev2(q + u), a, ca, b, cb);
            }
            for (; q < m; ++q) seg_take<MODE>(Do[rowoff[q]], ev1(q), ev2(q), a, ca, b, cb);
        }
    }
    if (!active) return;
    const int64_t base = (int64_t)s * n + o;
    if constexpr (VEC == 4) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            part1[base + 2 * h] = (double)a2[h].x - (double)ca2[h].x;
            part1[base + 2 * h + 1] = (double)a2[h].y - (double)ca2[h].y;
            if (MODE == kSegPam) {
                part2[base + 2 * h] = (double)b2[h].x - (double)cb2[h].x;
                part2[base + 2 * h + 1] = (double)b2[h].y - (double)cb2[h].y;
            }
        }
    } else {
        part1[base] = (double)a - (double)ca;
        if (MODE == kSegPam) part2[base] = (double)b - (double)cb;
    }
}

__device__ __forceinline__ void cp_async16(void *dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// The same reduction with the rows staged through shared memory by per-thread
// asynchronous copies (VEC = 4 layout: n % 4 == 0, D 16-byte aligned, L <=
// kSegStage).  Each thread copies its own 16-byte chunk of kAsRows rows per
// group into its own slots of a kAsSlots-deep ring, keeps kAsAhead groups in
// flight and waits only for its own copies: no barrier, and the bytes in flight
// (kAsAhead * kAsRows * 16 per thread) hold no registers.  The slot refilled
// in step b was read in step b - 1.  Same thread-to-column map and arithmetic
// as segred_kernel, so the same bits.
constexpr int kAsRows = 4;
constexpr int kAsSlots = 4;
constexpr int kAsAhead = 3;
constexpr size_t kAsSmem = (size_t)kAsSlots * kAsRows * kSegThreads * 16;  // 64 KB, dynamic

template <int MODE>
__global__ void __launch_bounds__(kSegThreads, 3)
    segred_async_kernel(const float *__restrict__ D, int n, int L, const int32_t *__restrict__ perm,
                        const int2 *__restrict__ segs, const int32_t *__restrict__ nseg,
                        const float *__restrict__ d1, const float *__restrict__ d2,
                        double *__restrict__ part1, double *__restrict__ part2)
{
    extern __shared__ __align__(16) unsigned char as_smem[];
    float4 *ring = reinterpret_cast<float4 *>(as_smem);  // [slot][row][thread]
    __shared__ int64_t rowoff[kSegStage];
    __shared__ float e1[MODE == kSegSum ? 1 : kSegStage];
    __shared__ float e2[MODE == kSegPam ? kSegStage : 1];
    const int s = blockIdx.y, tid = threadIdx.x;
    int lo, hi;
    if (segs) {
        if (s >= *nseg) return;
        const int2 g = segs[s];
        lo = g.x;
        hi = g.y;
    } else {
        lo = s * L;
        hi = min(lo + L, n);
    }
    const int m = hi - lo;  // <= kSegStage
    for (int q = tid; q < m; q += kSegThreads) {
        const int j = perm ? perm[lo + q] : lo + q;
        rowoff[q] = (int64_t)j * n;
        if (MODE != kSegSum) e1[q] = d1[lo + q];
        if (MODE == kSegPam) e2[q] = d2[lo + q];
    }
    __syncthreads();  // the only barrier
    const int o = (blockIdx.x * kSegThreads + tid) * 4;
    if (o >= n) return;
    const float *Do = D + o;
    const int nb = (m + kAsRows - 1) / kAsRows;
    auto issue = [&](int b) {
        if (b < nb) {
#pragma unroll
            for (int r = 0; r < kAsRows; ++r) {
                const int q = b * kAsRows + r;
                if (q < m) cp_async16(&ring[((b % kAsSlots) * kAsRows + r) * kSegThreads + tid], Do + rowoff[q]);
            }
        }
        cp_async_commit();  // possibly empty, so that every step waits for the same count
    };
#pragma unroll
    for (int g = 0; g < kAsAhead; ++g) issue(g);
    float2 a2[2], ca2[2], b2[2], cb2[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) a2[h] = ca2[h] = b2[h] = cb2[h] = make_float2(0.f, 0.f);
    for (int b = 0; b < nb; ++b) {
        cp_async_wait<kAsAhead - 1>();  // this thread's copies of group b have landed
#pragma unroll
        for (int r = 0; r < kAsRows; ++r) {
            const int q = b * kAsRows + r;
            if (q < m) {
                const float4 x = ring[((b % kAsSlots) * kAsRows + r) * kSegThreads + tid];
                const float f1 = MODE == kSegSum ? 0.f : e1[q], f2 = MODE == kSegPam ? e2[q] : 0.f;
                seg_take2<MODE>(make_float2(x.x, x.y), f1, f2, a2[0], ca2[0], b2[0], cb2[0]);
                seg_take2<MODE>(make_float2(x.z, x.w), f1, f2, a2[1], ca2[1], b2[1], cb2[1]);
            }
        }
        issue(b + kAsAhead);
    }
    cp_async_wait<0>();
    const int64_t base = (int64_t)s * n + o;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        part1[base + 2 * h] = (double)a2[h].x - (double)ca2[h].x;
        part1[base + 2 * h + 1] = (double)a2[h].y - (double)ca2[h].y;
        if (MODE == kSegPam) {
            part2[base + 2 * h] = (double)b2[h].x - (double)cb2[h].x;
            part2[base + 2 * h + 1] = (double)b2[h].y - (double)cb2[h].y;
        }
    }
}

// the sum of the partials of segments [s0, s1) in column o, in segment order
__device__ __forceinline__ double seg_sum(const double *__restrict__ part, int n, int s0, int s1, int o)
{
    double t = 0.0;
#pragma unroll 4
    for (int s = s0; s < s1; ++s) t += part[(int64_t)s * n + o];
    return t;
}

// The finish kernels run 256 threads per 32 columns: lane = column, and the
// eight warps split the clusters (c = warp, warp + 8, ...) or the segments, so
// that enough partials are read at once.
constexpr int kFinCols = 32;
constexpr int kFinWarps = 8;

struct PamBest {
    double delta;
    int64_t idx;
};

__device__ __forceinline__ void keep_least(double &v, int64_t &i, double v2, int64_t i2)
{
    if (v2 < v || (v2 == v && i2 < i)) {
        v = v2;
        i = i2;
    }
}

// the least (v, i) of the block, ties to the smaller i; valid in thread 0
__device__ __forceinline__ void block_least(double &v, int64_t &i)
{
    __shared__ double sv[32];
    __shared__ int64_t si[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        keep_least(v, i, __shfl_xor_sync(0xffffffffu, v, o), __shfl_xor_sync(0xffffffffu, i, o));
    if ((threadIdx.x & 31) == 0) {
        sv[threadIdx.x >> 5] = v;
        si[threadIdx.x >> 5] = i;
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int q = 1; q < (int)(blockDim.x >> 5); ++q) keep_least(v, i, sv[q], si[q]);
}

// s(i) from the segment sums of column i: warp w takes the clusters c = w, w + 8,
// ... (each cluster's segments in order), then warp 0 combines
__global__ void __launch_bounds__(kFinWarps * 32)
    silhouette_finish_kernel(const double *__restrict__ part, int n, int k,
                             const int32_t *__restrict__ labels, const int32_t *__restrict__ cstart,
                             const int32_t *__restrict__ segbase, float *__restrict__ out_s,
                             double *__restrict__ s64)
{
    __shared__ double own_sum[kFinWarps][kFinCols], least[kFinWarps][kFinCols];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int i = blockIdx.x * kFinCols + lane;
    double a = 0.0, b = 1.0 / 0.0;
    const int own = i < n ? labels[i] : -1;
    if (i < n) {
        for (int c = w; c < k; c += kFinWarps) {
            const int mc = cstart[c + 1] - cstart[c];
            if (mc == 0) continue;
            const double t = seg_sum(part, n, segbase[c], segbase[c + 1], i);
            if (c == own)
                a = t;
            else
                b = fmin(b, t / (double)mc);
        }
    }
    own_sum[w][lane] = a;
    least[w][lane] = b;
    __syncthreads();
    if (w != 0 || i >= n) return;
    const int m = cstart[own + 1] - cstart[own];
    double s = 0.0;
    if (m > 1) {
        const double ai = own_sum[own % kFinWarps][lane] / (double)(m - 1);
        double bi = least[0][lane];
        for (int q = 1; q < kFinWarps; ++q) bi = fmin(bi, least[q][lane]);
        const double mx = ai > bi ? ai : bi;
        s = mx > 0.0 ? (bi - ai) / mx : 0.0;
    }
    s64[i] = s;
    if (out_s) out_s[i] = (float)s;
}

__device__ __forceinline__ double block_sum(double v, double *warp_part)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) warp_part[w] = v;
    __syncthreads();
    double t = 0.0;
    for (int q = 0; q < kSilThreads / 32; ++q) t += warp_part[q];
    __syncthreads();
    return t;
}

// s(i) for row i = blockIdx.x, gathering the members of every cluster from row i
__global__ void __launch_bounds__(kSilThreads)
    silhouette_kernel(const float *__restrict__ D, int n, const int32_t *__restrict__ labels,
                      int k, const int32_t *__restrict__ cstart, const int32_t *__restrict__ perm,
                      float *__restrict__ out_s, double *__restrict__ s64)
{
    extern __shared__ double csum[];  // [k]
    __shared__ double warp_part[kSilThreads / 32];
    const int i = blockIdx.x;
    const float *row = D + (int64_t)i * n;
    for (int c = 0; c < k; ++c) {
        double acc = 0.0;
        for (int q = cstart[c] + threadIdx.x; q < cstart[c + 1]; q += kSilThreads)
            acc += (double)row[perm[q]];
        const double t = block_sum(acc, warp_part);
        if (threadIdx.x == 0) csum[c] = t;
    }
    if (threadIdx.x == 0) {
        const int own = labels[i];
        const int m = cstart[own + 1] - cstart[own];
        double s = 0.0;
        if (m > 1) {
            const double a = csum[own] / (double)(m - 1);
            double b = 1.0 / 0.0;
            for (int c = 0; c < k; ++c) {
                const int mc = cstart[c + 1] - cstart[c];
                if (c == own || mc == 0) continue;
                const double v = csum[c] / (double)mc;
                if (v < b) b = v;
            }
            const double mx = a > b ? a : b;
            s = mx > 0.0 ? (b - a) / mx : 0.0;
        }
        s64[i] = s;
        if (out_s) out_s[i] = (float)s;
    }
}

__global__ void sum_parts_kernel(const double *__restrict__ v, int n, double *__restrict__ part)
{
    __shared__ double sh[256];
    double acc = 0.0;
    for (int j = blockIdx.x * 256 + threadIdx.x; j < n; j += gridDim.x * 256) acc += v[j];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// ------------------------------------------------------------------ PAM

constexpr int kPamMaxK = 64;

__device__ __forceinline__ bool is_medoid(const int32_t *M, int k, int o)
{
    for (int c = 0; c < k; ++c)
        if (M[c] == o) return true;
    return false;
}

// BUILD gain of every point from the nseg segment partials (+inf for the
// medoids M[0..slot)); warp w adds the w-th eighth of the segments, warp 0 the
// eight sums in order; per block the least (gain, o)
__global__ void __launch_bounds__(kFinWarps * 32)
    build_finish_kernel(const double *__restrict__ part, int nseg, int n,
                        const int32_t *__restrict__ M, int slot, PamBest *__restrict__ blockbest)
{
    __shared__ double sums[kFinWarps][kFinCols];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int o = blockIdx.x * kFinCols + lane;
    const int per = (nseg + kFinWarps - 1) / kFinWarps;
    sums[w][lane] = o < n ? seg_sum(part, n, min(nseg, w * per), min(nseg, (w + 1) * per), o) : 0.0;
    __syncthreads();
    double v = 1.0 / 0.0;
    int64_t i = INT64_MAX;
    if (w == 0 && o < n && !is_medoid(M, slot, o)) {
        v = sums[0][lane];
        for (int q = 1; q < kFinWarps; ++q) v += sums[q][lane];
        if (v != v) v = 1.0 / 0.0;  // a NaN in D: never the least, but still a valid point
        i = o;
    }
    block_least(v, i);
    if (threadIdx.x == 0) blockbest[blockIdx.x] = PamBest{v, i};
}

// FastPAM1 deltas of candidate o from the segment partials of the two terms:
//   t1(c) = sum over c's members j of min(0, D[j][o] - d1(j))
//   t2(c) = sum over c's members j of min(D[j][o], d2(j)) - d1(j)
//   delta(o, i) = sum_c t1(c) + t2(i) - t1(i)     (+inf for medoids)
// warp w forms the terms q = w, w + 8, ... of the 2k (t1(c) for q = 2c, t2(c)
// for q = 2c + 1); warp 0 the deltas; per block the least (delta, o k + i)
__global__ void __launch_bounds__(kFinWarps * 32)
    pam_finish_kernel(const double *__restrict__ p1, const double *__restrict__ p2, int n,
                      const int32_t *__restrict__ segbase, const int32_t *__restrict__ M, int k,
                      PamBest *__restrict__ blockbest)
{
    __shared__ double t1[kPamMaxK][kFinCols], t2[kPamMaxK][kFinCols];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int o = blockIdx.x * kFinCols + lane;
    if (o < n)
        for (int q = w; q < 2 * k; q += kFinWarps) {
            const int c = q >> 1;
            const double t = seg_sum(q & 1 ? p2 : p1, n, segbase[c], segbase[c + 1], o);
            if (q & 1)
                t2[c][lane] = t;
            else
                t1[c][lane] = t;
        }
    __syncthreads();
    double v = 1.0 / 0.0;
    int64_t idx = INT64_MAX;
    if (w == 0 && o < n && !is_medoid(M, k, o)) {
        double S = 0.0;
        for (int c = 0; c < k; ++c) S += t1[c][lane];
        for (int c = 0; c < k; ++c) {
            const double d = S + t2[c][lane] - t1[c][lane];
            if (d < v) {
                v = d;
                idx = (int64_t)o * k + c;
            }
        }
    }
    block_least(v, idx);
    if (threadIdx.x == 0) blockbest[blockIdx.x] = PamBest{v, idx};
}

// One block: the least of the per-block bests.  slot >= 0 (BUILD): M[slot] =
// its point; slot < 0 (SWAP): when its delta is negative, medoid idx % k is
// replaced by point idx / k.
__global__ void __launch_bounds__(256)
    pam_pick_kernel(const PamBest *__restrict__ blockbest, int nb, int32_t *__restrict__ M, int k,
                    int slot, PamBest *__restrict__ best)
{
    double v = 1.0 / 0.0;
    int64_t i = INT64_MAX;
    for (int q = threadIdx.x; q < nb; q += 256) keep_least(v, i, blockbest[q].delta, blockbest[q].idx);
    block_least(v, i);
    if (threadIdx.x != 0) return;
    *best = PamBest{v, i};
    if (slot >= 0)
        M[slot] = (int32_t)i;
    else if (v < 0.0)
        M[i % k] = (int32_t)(i / k);
}

// d1[j] = min(d1[j], D[M[slot]][j]) (slot 0: D[M[0]][j])
__global__ void pam_d1_update_kernel(const float *__restrict__ D, int n, const int32_t *__restrict__ M,
                                     int slot, float *__restrict__ d1)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const float v = D[(int64_t)M[slot] * n + j];
    d1[j] = slot == 0 ? v : fminf(d1[j], v);
}

// nearest (n1, ties to the smaller position) and second-nearest distances;
// counts per nearest medoid (one atomic per warp and medoid)
__global__ void pam_nearest_kernel(const float *__restrict__ D, int n, const int32_t *__restrict__ M,
                                   int k, float *__restrict__ d1, float *__restrict__ d2,
                                   int32_t *__restrict__ n1, int32_t *__restrict__ cnt)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    int c1 = -1;  // stays -1 past the end, so that whole warps reach the vote below
    if (j < n) {
        float b1 = 1.0f / 0.0f, b2 = 1.0f / 0.0f;
        c1 = 0;
        for (int c = 0; c < k; ++c) {
            const float v = D[(int64_t)M[c] * n + j];
            if (v < b1) {
                b2 = b1;
                b1 = v;
                c1 = c;
            } else if (v < b2) {
                b2 = v;
            }
        }
        d1[j] = b1;
        d2[j] = b2;
        n1[j] = c1;
    }
    const unsigned peers = __match_any_sync(0xffffffffu, c1);
    if (c1 >= 0 && (int)(threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(cnt + c1, __popc(peers));
}

// labels = nearest medoid, except that a medoid labels itself
__global__ void pam_labels_kernel(const int32_t *__restrict__ n1, int n, const int32_t *__restrict__ M,
                                  int k, int32_t *__restrict__ labels)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    int lab = n1[j];
    for (int c = 0; c < k; ++c)
        if (M[c] == j) {
            lab = c;
            break;
        }
    labels[j] = lab;
}

__global__ void sum_float_parts_kernel(const float *__restrict__ v, int n, double *__restrict__ part)
{
    __shared__ double sh[256];
    double acc = 0.0;
    for (int j = blockIdx.x * 256 + threadIdx.x; j < n; j += gridDim.x * 256) acc += (double)v[j];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// The asynchronous-copy kernels take 64 KB of dynamic shared memory, above the
// default 48 KB; set once per process (the attribute holds for every device).
int prepare_segred()
{
    static bool done = false;
    if (done) return DTW_OK;
    DTWGB_CUDA(cudaFuncSetAttribute(segred_async_kernel<kSegSum>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kAsSmem));
    DTWGB_CUDA(cudaFuncSetAttribute(segred_async_kernel<kSegMinD1>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kAsSmem));
    DTWGB_CUDA(cudaFuncSetAttribute(segred_async_kernel<kSegPam>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kAsSmem));
    done = true;
    return DTW_OK;
}

// The segment reduction over nseg_grid segments: staged by asynchronous copies
// when the rows are 16-byte aligned, else the scalar kernel.
template <int MODE>
void launch_segred(const float *D, int n, int L, const int32_t *perm, const int2 *segs,
                   const int32_t *nseg, int nseg_grid, const float *d1, const float *d2, double *p1,
                   double *p2, cudaStream_t st)
{
    if ((n % 4 == 0) && ((uintptr_t)D % 16 == 0) && L <= kSegStage) {
        const dim3 grid((unsigned)((n / 4 + kSegThreads - 1) / kSegThreads), (unsigned)nseg_grid);
        segred_async_kernel<MODE><<<grid, kSegThreads, kAsSmem, st>>>(D, n, L, perm, segs, nseg, d1, d2,
                                                                      p1, p2);
    } else {
        const dim3 grid((unsigned)((n + kSegThreads - 1) / kSegThreads), (unsigned)nseg_grid);
        segred_kernel<MODE, 1><<<grid, kSegThreads, 0, st>>>(D, n, L, perm, segs, nseg, d1, d2, p1, p2);
    }
}

// a scratch region's bytes, rounded up to 256 so that every region stays aligned
size_t al(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace
}  // namespace dtwgb

using namespace dtwgb;

extern "C" int kmedoids_silhouette(const float *D, int32_t n, const int32_t *labels, int32_t k,
                                   float *out_s, double *out_mean, void *stream)
{
    clear_error();
    cudaStream_t st = (cudaStream_t)stream;
    if (!D || !labels || !out_mean) { set_error("NULL pointer argument"); return DTW_EINVAL; }
    if (n < 2 || k < 2 || k > kSilMaxK) {
        set_error("need n >= 2 and 2 <= k <= %d (n = %d, k = %d)", kSilMaxK, n, k);
        return DTW_EINVAL;
    }
    std::vector<int32_t> hl((size_t)n);
    DTWGB_CUDA(cudaMemcpyAsync(hl.data(), labels, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, st));
    DTWGB_CUDA(cudaStreamSynchronize(st));
    std::vector<int32_t> cnt((size_t)k, 0);
    for (int j = 0; j < n; ++j) {
        if (hl[j] < 0 || hl[j] >= k) {
            set_error("labels[%d] = %d is outside [0, %d)", j, hl[j], k);
            return DTW_EINVAL;
        }
        ++cnt[hl[j]];
    }
    int nonempty = 0;
    for (int c = 0; c < k; ++c) nonempty += cnt[c] > 0;
    if (nonempty < 2) {
        set_error("the silhouette needs at least two non-empty clusters (%d)", nonempty);
        return DTW_EINVAL;
    }
    int rc = prepare_segred();
    if (rc) return rc;
    const int L = seg_rows(n);
    const int nseg_grid = (n + L - 1) / L + k;
    // segment partials of at most 2^27 doubles; beyond, one block per row gathers
    const bool by_columns = (int64_t)n * nseg_grid <= (128ll << 20);
    const size_t bytes = al(sizeof(double) * n) + al(sizeof(double) * kSilParts) +
                         (by_columns ? al(sizeof(double) * (size_t)n * nseg_grid) : 0) +
                         al(sizeof(int32_t) * (3 * (size_t)k + 3 + n)) + al(sizeof(int2) * nseg_grid);
    void *buf = nullptr;
    rc = scratch_alloc(&buf, bytes, st);
    if (rc) return rc;
    char *p = (char *)buf;
    double *s64 = (double *)p;
    p += al(sizeof(double) * n);
    double *part = (double *)p;
    p += al(sizeof(double) * kSilParts);
    double *seg = (double *)p;
    if (by_columns) p += al(sizeof(double) * (size_t)n * nseg_grid);
    int32_t *dcnt = (int32_t *)p;
    int32_t *cstart = dcnt + k;
    int32_t *segbase = cstart + k + 1;
    int32_t *nseg = segbase + k + 1;
    int32_t *perm = nseg + 1;
    p += al(sizeof(int32_t) * (3 * (size_t)k + 3 + n));
    int2 *segs = (int2 *)p;
    cudaError_t e = cudaMemcpyAsync(dcnt, cnt.data(), sizeof(int32_t) * k, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        seg_table_kernel<<<1, 256, 0, st>>>(dcnt, k, L, cstart, segbase, segs, nseg);
        sil_members_kernel<<<k, kMemThreads, 0, st>>>(labels, n, cstart, perm, nullptr, nullptr,
                                                      nullptr, nullptr);
        if (by_columns) {
            launch_segred<kSegSum>(D, n, L, perm, segs, nseg, nseg_grid, nullptr, nullptr, seg,
                                   nullptr, st);
            silhouette_finish_kernel<<<(n + kFinCols - 1) / kFinCols, kFinWarps * 32, 0, st>>>(
                seg, n, k, labels, cstart, segbase, out_s, s64);
        } else {
            silhouette_kernel<<<n, kSilThreads, sizeof(double) * k, st>>>(D, n, labels, k, cstart,
                                                                          perm, out_s, s64);
        }
        sum_parts_kernel<<<kSilParts, 256, 0, st>>>(s64, n, part);
        e = cudaGetLastError();
    }
    std::vector<double> hp(kSilParts);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(hp.data(), part, sizeof(double) * kSilParts, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    scratch_free(buf, st);
    if (e != cudaSuccess) return cuda_fail(e, "silhouette kernels");
    double tot = 0.0;
    for (double v : hp) tot += v;
    *out_mean = tot / (double)n;
    return DTW_OK;
}

extern "C" int kmedoids_pam(const float *D, int32_t n, int32_t k, const int32_t *init_medoids,
                            int32_t max_swaps, int32_t *out_medoids, int32_t *out_labels,
                            double *out_cost, int32_t *out_swaps, void *stream)
{
    clear_error();
    cudaStream_t st = (cudaStream_t)stream;
    if (!D || !out_medoids || !out_labels) { set_error("NULL pointer argument"); return DTW_EINVAL; }
    if (n < 1 || k < 1 || k > n || k > kPamMaxK || max_swaps < 0) {
        set_error("need n >= 1, 1 <= k <= min(n, %d), max_swaps >= 0 (n = %d, k = %d, max_swaps = %d)",
                  kPamMaxK, n, k, max_swaps);
        return DTW_EINVAL;
    }
    if (init_medoids) {
        std::vector<int32_t> h((size_t)k);
        DTWGB_CUDA(cudaMemcpyAsync(h.data(), init_medoids, sizeof(int32_t) * k, cudaMemcpyDeviceToHost, st));
        DTWGB_CUDA(cudaStreamSynchronize(st));
        for (int c = 0; c < k; ++c) {
            if (h[c] < 0 || h[c] >= n) { set_error("init_medoids[%d] = %d is outside [0, %d)", c, h[c], n); return DTW_EINVAL; }
            for (int d = 0; d < c; ++d)
                if (h[d] == h[c]) { set_error("init_medoids[%d] and [%d] are both %d", d, c, h[c]); return DTW_EINVAL; }
        }
    }
    int rc = prepare_segred();
    if (rc) return rc;
    const int L = seg_rows(n);
    const int nrow_seg = (n + L - 1) / L;  // segments of all rows (BUILD)
    const int nseg_grid = nrow_seg + k;    // bound on the segments of the clusters (SWAP)
    const unsigned nb = (unsigned)((n + 255) / 256);
    const unsigned nfb = (unsigned)((n + kFinCols - 1) / kFinCols);  // finish blocks
    const size_t pbytes = al(sizeof(double) * (size_t)n * nseg_grid);
    const size_t bytes = 2 * pbytes + al(sizeof(double) * kSilParts) + al(sizeof(PamBest) * (nfb + 1)) +
                         al(sizeof(float) * 4 * (size_t)n) +
                         al(sizeof(int32_t) * (2 * (size_t)n + 3 * (size_t)k + 3)) +
                         al(sizeof(int2) * nseg_grid);
    void *buf = nullptr;
    rc = scratch_alloc(&buf, bytes, st);
    if (rc) return rc;
    char *p = (char *)buf;
    double *p1 = (double *)p;
    double *p2 = (double *)(p + pbytes);
    p += 2 * pbytes;
    double *part = (double *)p;
    p += al(sizeof(double) * kSilParts);
    PamBest *blockbest = (PamBest *)p;
    PamBest *best = blockbest + nfb;
    p += al(sizeof(PamBest) * (nfb + 1));
    float *d1 = (float *)p;
    float *d2 = d1 + n;
    float *pd1 = d2 + n;  // d1, d2 in member-list order
    float *pd2 = pd1 + n;
    p += al(sizeof(float) * 4 * (size_t)n);
    int32_t *n1 = (int32_t *)p;
    int32_t *perm = n1 + n;
    int32_t *cnt = perm + n;
    int32_t *cstart = cnt + k;
    int32_t *segbase = cstart + k + 1;
    int32_t *nseg = segbase + k + 1;
    p += al(sizeof(int32_t) * (2 * (size_t)n + 3 * (size_t)k + 3));
    int2 *segs = (int2 *)p;
    int32_t *M = out_medoids;
    cudaError_t e = cudaSuccess;
    auto fail = [&](cudaError_t ce, const char *what) {
        scratch_free(buf, st);
        return cuda_fail(ce, what);
    };
    if (init_medoids) {
        e = cudaMemcpyAsync(M, init_medoids, sizeof(int32_t) * k, cudaMemcpyDeviceToDevice, st);
    } else {
        for (int s = 0; s < k; ++s) {  // BUILD: the gains as segment sums down all rows
            if (s == 0)
                launch_segred<kSegSum>(D, n, L, nullptr, nullptr, nullptr, nrow_seg, nullptr, nullptr,
                                       p1, nullptr, st);
            else
                launch_segred<kSegMinD1>(D, n, L, nullptr, nullptr, nullptr, nrow_seg, d1, nullptr, p1,
                                         nullptr, st);
            build_finish_kernel<<<nfb, kFinWarps * 32, 0, st>>>(p1, nrow_seg, n, M, s, blockbest);
            pam_pick_kernel<<<1, 256, 0, st>>>(blockbest, (int)nfb, M, k, s, best);
            pam_d1_update_kernel<<<nb, 256, 0, st>>>(D, n, M, s, d1);
        }
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return fail(e, "PAM build");
    int32_t swaps = 0;
    for (;;) {
        e = cudaMemsetAsync(cnt, 0, sizeof(int32_t) * k, st);
        if (e != cudaSuccess) break;
        pam_nearest_kernel<<<nb, 256, 0, st>>>(D, n, M, k, d1, d2, n1, cnt);
        if (swaps >= max_swaps) break;
        seg_table_kernel<<<1, 256, 0, st>>>(cnt, k, L, cstart, segbase, segs, nseg);
        sil_members_kernel<<<k, kMemThreads, 0, st>>>(n1, n, cstart, perm, d1, d2, pd1, pd2);
        launch_segred<kSegPam>(D, n, L, perm, segs, nseg, nseg_grid, pd1, pd2, p1, p2, st);
        pam_finish_kernel<<<nfb, kFinWarps * 32, 0, st>>>(p1, p2, n, segbase, M, k, blockbest);
        pam_pick_kernel<<<1, 256, 0, st>>>(blockbest, (int)nfb, M, k, -1, best);
        PamBest h;
        e = cudaMemcpyAsync(&h, best, sizeof(PamBest), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) break;
        if (!(h.delta < 0.0)) break;
        ++swaps;
    }
    if (e == cudaSuccess) {
        pam_labels_kernel<<<nb, 256, 0, st>>>(n1, n, M, k, out_labels);
        sum_float_parts_kernel<<<kSilParts, 256, 0, st>>>(d1, n, part);
        e = cudaGetLastError();
    }
    std::vector<double> hp(kSilParts);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hp.data(), part, sizeof(double) * kSilParts, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(e, "PAM swap passes");
    scratch_free(buf, st);
    double tot = 0.0;
    for (double v : hp) tot += v;
    if (out_cost) *out_cost = tot;
    if (out_swaps) *out_swaps = swaps;
    return DTW_OK;
}
