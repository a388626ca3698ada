// dtw_band.cu -- all-pairs and 1-vs-N windowed DTW on sm_103a.
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
//   * x_i enters at lane 0 and moves one lane per step (shuffle up); the band
//     slides one column per row, so each lane's window of y values shifts by
//     one slot per step, the new value coming from lane l+1 and, at the last
//     lane, from memory.
// Cells with j outside [1, m] see y = +inf and therefore stay +inf, which
// also realises c_{i,0} = +inf.  Slots beyond 2w (when G*K > 2w+1) are forced
// to +inf by a max with a per-lane mask on the last MT slots.
//
// Only the previous row is kept (the paper's previous-row vector), here in
// registers; no shared memory, no per-cell band test.  One float is written
// per pair; the full matrix gets d_ij and d_ji (the DP is exactly symmetric).
#include "common.cuh"

namespace dtwgb {

enum : int { SRC_TRIANGLE = 0, SRC_QUERY = 1 };
enum : int { OUT_FULL = 0, OUT_PACKED = 1, OUT_ROW = 2 };

struct BandArgs {
    const float *padded;     // series staged with PL leading and PR trailing +inf (see stage_kernel)
    const int64_t *offsets;  // offsets of the unpadded set
    int64_t qbase;           // SRC_QUERY: index of the query's x_1 in `padded`
    int64_t qlen;
    int64_t p;        // series in the set
    int64_t n_pairs;  // p(p-1)/2 for the triangle, p for a query
    int32_t window;   // < 0: no band
    int32_t strict;
    int32_t src;
    int32_t out_mode;
    float *out;
    int32_t G, log2G;
    int32_t PL, PR;   // padding of every staged series
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
    if (A.src == SRC_TRIANGLE) {
        int64_t a, b;
        tri_index(t, A.p, a, b);
        g.a = a;
        g.b = b;
        const int64_t oa = A.offsets[a], ob = A.offsets[b];
        s0 = A.padded + (oa - o0) + a * pad + A.PL;
        n0 = A.offsets[a + 1] - oa;
        s1 = A.padded + (ob - o0) + b * pad + A.PL;
        n1 = A.offsets[b + 1] - ob;
    } else {
        g.a = -1;
        g.b = t;
        const int64_t ob = A.offsets[t];
        s0 = A.padded + A.qbase;
        n0 = A.qlen;
        s1 = A.padded + (ob - o0) + t * pad + A.PL;
        n1 = A.offsets[t + 1] - ob;
    }
    if (n0 <= n1) {
        g.x = s0; g.n = (int32_t)n0; g.y = s1; g.m = (int32_t)n1;
    } else {
        g.x = s1; g.n = (int32_t)n1; g.y = s0; g.m = (int32_t)n0;
    }
    const int32_t diff = g.m - g.n;
    int32_t w;
    if (A.window < 0) w = g.m - 1;
    else if (A.strict) w = A.window;
    else w = A.window > diff ? A.window : diff;
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
    } else if (A.out_mode == OUT_PACKED) {
        A.out[t] = r;
    } else {
        A.out[g.b] = r;
    }
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
// Each lane fetches its own next x and y values from the padded series,
// two steps ahead: px[T'] = x_{T'+1-l} and py[T'] = the y value that enters
// its last slot after step T' (pb* are those pointers advanced to the block).
template <int K, int MT, bool CHECK>
__device__ __forceinline__ void band_step(const int s, const int T, const int l, const int G,
                                          const bool have, const int n, float (&prev)[K],
                                          float (&ywin)[K], const float (&tmask)[MT],
                                          const float lmask, const float rmask, float &xr,
                                          float &left_in, float &pxa, float &pxb, float &pya,
                                          float &pyb, const float *pbx, const float *pby)
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
    pya = pyb;
    pxa = pxb;
    if (!CHECK || have) {
        pyb = __ldg(pby + s + 3);
        pxb = __ldg(pbx + s + 3);
    }
}

// Resident blocks per SM the register allocation aims for: 4 (64 registers)
// for the narrow shapes, 3 where 64 registers would spill.
template <int K, int MT>
constexpr int band_min_blocks()
{
#ifdef DTWGB_BAND_MINB
    return DTWGB_BAND_MINB;
#else
    return (K <= 13 && MT == 1) || K <= 8 ? 4 : 3;
#endif
}

template <int K, int MT>
__global__ void __launch_bounds__(256, band_min_blocks<K, MT>()) dtw_band_kernel(const BandArgs A)
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
    const int kbase = l * K;
    const float lmask = first ? INF : 0.f;
    const float rmask = last ? INF : 0.f;

    int64_t pair = warp * gpw + (lane >> A.log2G) - ngroups;
    float prev[K], ywin[K], tmask[MT];
    float xr = 0.f, left_in = INF, pxa = 0.f, pxb = 0.f, pya = 0.f, pyb = 0.f;
    // px[T] = x_{T+1-l}, py[T] = y_{T+l(K-1)+K-w}; both advance by K per block
    const float *px = A.padded, *py = A.padded;
    bool have = false;
    int n = 0, blk = 0, nblk = 0;

    while (true) {
        if (!have) {
            // next pair of this group; pairs the strict band cannot join are +inf
            PairGeom g;
            while (true) {
                pair += ngroups;
                if (pair >= A.n_pairs) break;
                pair_geometry(A, pair, g);
                if (!g.trivial) { have = true; break; }
                if (first) write_result(A, pair, g, INF);
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
                pxb = __ldg(px + 2);
                pya = __ldg(py + 1);
                pyb = __ldg(py + 2);
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
                                        rmask, xr, left_in, pxa, pxb, pya, pyb, px, py);
        } else {
#pragma unroll
            for (int s = 0; s < K; ++s)
                band_step<K, MT, true>(s, T0 + s + 1, l, G, have, n, prev, ywin, tmask, lmask,
                                       rmask, xr, left_in, pxa, pxb, pya, pyb, px, py);
        }
        px += K;
        py += K;

        if (have && ++blk == nblk) {
            // every lane now holds row n; c_{n,m} sits at band offset kres
            PairGeom g;
            pair_geometry(A, pair, g);
            const int lres = g.kres / K, tres = g.kres - lres * K;
            float r = prev[0];
#pragma unroll
            for (int t = 1; t < K; ++t)
                if (t == tres) r = prev[t];
            if (l == lres) write_result(A, pair, g, r);
            have = false;
        }
    }
}

// Copy series i of a set into the padded layout: PL values of +inf, the
// series, PR values of +inf.  One block per series.
__global__ void stage_kernel(const float *__restrict__ values, const int64_t *__restrict__ offsets,
                             int32_t PL, int32_t PR, float *__restrict__ padded)
{
    const int64_t i = blockIdx.x;
    const int64_t o0 = offsets[0], a = offsets[i], len = offsets[i + 1] - a;
    float *dst = padded + (a - o0) + i * (int64_t)(PL + PR);
    const int64_t total = len + PL + PR;
    for (int64_t q = threadIdx.x; q < total; q += blockDim.x)
        dst[q] = (q >= PL && q < PL + len) ? values[a + q - PL] : finf();
}

__global__ void stage_one_kernel(const float *__restrict__ v, int64_t len, int32_t PL, int32_t PR,
                                 float *__restrict__ dst)
{
    const int64_t total = len + PL + PR;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x)
        dst[q] = (q >= PL && q < PL + len) ? v[q - PL] : finf();
}

__global__ void zero_diagonal_kernel(float *D, int64_t p)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < p) D[i * p + i] = 0.f;
}

__global__ void finite_scan_kernel(const float *v, int64_t n, int *bad)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        if (!isfinite(v[i])) *bad = 1;
}

// ---------------------------------------------------------------- host side

namespace {

constexpr int kMaxG = 32;
constexpr int kMaxK = 16;
constexpr int kThreads = 256;

struct Shape {
    int K, G, MT;  // MT is 1 or K
};

// Band shape for rows of `wneed` cells: smallest estimated instruction count
// per pair over the compiled K values.
bool pick_shape(int wneed, int rows, Shape &out)
{
    static const int Ks[] = {4, 8, 13, 16};
    double best = 1e300;
    bool ok = false;
    for (int K : Ks) {
        int G = 2;
        while (G * K < wneed && G < kMaxG) G *= 2;
        if (G * K < wneed) continue;
        const int waste = G * K - wneed;
        const int MT = waste <= 1 ? 1 : K;
        const double steps = rows + G - 1 + 0.5 * (K - 1);
        const double per_step = 3.0 * K + MT + 14.0;  // cells + masks + shuffles/loads
        const double cost = G * steps * per_step;
        if (cost < best) {
            best = cost;
            out = Shape{K, G, MT};
            ok = true;
        }
    }
    return ok;
}

template <int K, int MT>
int launch_shape(BandArgs A, cudaStream_t st)
{
    auto kern = dtw_band_kernel<K, MT>;
    int dev = 0, sms = 0, per_sm = 0;
    DTWGB_CUDA(cudaGetDevice(&dev));
    DTWGB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    DTWGB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, 0));
    if (per_sm < 1) per_sm = 1;
    const int64_t groups_per_block = (kThreads / 32) * (32 / A.G);
    int64_t need = (A.n_pairs + groups_per_block - 1) / groups_per_block;
    int64_t blocks = (int64_t)sms * per_sm;
    if (need < blocks) blocks = need;
    if (blocks < 1) blocks = 1;
    kern<<<(unsigned)blocks, kThreads, 0, st>>>(A);
    DTWGB_CUDA(cudaGetLastError());
    return DTW_OK;
}

int launch_band(BandArgs A, const Shape &s, cudaStream_t st)
{
    A.G = s.G;
    A.log2G = 0;
    while ((1 << A.log2G) < s.G) ++A.log2G;
    const bool full = s.MT != 1;
    switch (s.K) {
    case 4: return full ? launch_shape<4, 4>(A, st) : launch_shape<4, 1>(A, st);
    case 8: return full ? launch_shape<8, 8>(A, st) : launch_shape<8, 1>(A, st);
    case 13: return full ? launch_shape<13, 13>(A, st) : launch_shape<13, 1>(A, st);
    case 16: return full ? launch_shape<16, 16>(A, st) : launch_shape<16, 1>(A, st);
    default: set_error("internal: no kernel for K=%d", s.K); return DTW_EUNSUPPORTED;
    }
}

// Band half-width bound over every pair of lengths in [minlen, maxlen], and
// the same bound for a query of length qlen.
int64_t band_bound(int64_t minlen, int64_t maxlen, int32_t window, bool strict)
{
    int64_t w;
    if (window < 0) w = maxlen - 1;
    else if (strict) w = window;
    else w = window > (maxlen - minlen) ? window : (maxlen - minlen);
    if (w > maxlen - 1) w = maxlen - 1;
    return w;
}

struct SetInfo {
    int64_t total = 0, minlen = 0, maxlen = 0;
};

int check_offsets(const int64_t *h, int32_t p, SetInfo &info)
{
    if (h[0] < 0) {
        set_error("offsets[0] = %lld is negative", (long long)h[0]);
        return DTW_EINVAL;
    }
    info.minlen = INT64_MAX;
    info.maxlen = 0;
    for (int32_t i = 0; i < p; ++i) {
        const int64_t len = h[i + 1] - h[i];
        if (len <= 0) {
            set_error("series %d is empty or offsets decrease (offsets[%d]=%lld, offsets[%d]=%lld)",
                      i, i, (long long)h[i], i + 1, (long long)h[i + 1]);
            return DTW_EINVAL;
        }
        if (len > INT32_MAX / 4) {
            set_error("series %d is too long (%lld)", i, (long long)len);
            return DTW_EINVAL;
        }
        if (len < info.minlen) info.minlen = len;
        if (len > info.maxlen) info.maxlen = len;
    }
    info.total = h[p];
    return DTW_OK;
}

// RAII for stream-ordered scratch
struct DevBuf {
    void *p = nullptr;
    cudaStream_t st = nullptr;
    ~DevBuf() { scratch_free(p, st); }
};

int alloc(DevBuf &b, size_t bytes, cudaStream_t st)
{
    b.st = st;
    return scratch_alloc(&b.p, bytes, st);
}

int scan_finite(const float *v, int64_t n, cudaStream_t st, const char *what)
{
    DevBuf flag;
    int rc = alloc(flag, sizeof(int), st);
    if (rc) return rc;
    DTWGB_CUDA(cudaMemsetAsync(flag.p, 0, sizeof(int), st));
    if (n > 0) {
        finite_scan_kernel<<<1024, 256, 0, st>>>(v, n, (int *)flag.p);
        DTWGB_CUDA(cudaGetLastError());
    }
    int h = 0;
    DTWGB_CUDA(cudaMemcpyAsync(&h, flag.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    DTWGB_CUDA(cudaStreamSynchronize(st));
    if (h) {
        set_error("%s contain a NaN or Inf", what);
        return DTW_EINVAL;
    }
    return DTW_OK;
}

// Stage the set (and the query, if any) into a padded buffer and launch the
// band kernel.  Pads: PL > max(widest band half-width, G) (the first y window
// reaches y_{1-w}, ramp lanes read x_{3-G}), PR >= G*K + K + G + 1 (the last
// prefetches run that far past the end of a series).  The buffer is released stream-ordered.
int stage_and_launch(BandArgs A, const Shape &shape, int64_t wb, const float *vals,
                     const int64_t *offs, int64_t span, int32_t p, const float *q, int64_t qlen,
                     cudaStream_t st)
{
    A.PL = (int32_t)((wb > shape.G ? wb : shape.G) + 2);
    A.PR = shape.G * shape.K + shape.K + shape.G + 2;
    const int64_t pad = A.PL + A.PR;
    const int64_t nser = (int64_t)p + (q ? 1 : 0);
    const size_t elems = (size_t)(span + (q ? qlen : 0) + nser * pad);
    DevBuf buf;
    int rc = alloc(buf, sizeof(float) * elems, st);
    if (rc) return rc;
    float *padded = (float *)buf.p;
    stage_kernel<<<(unsigned)p, 256, 0, st>>>(vals, offs, A.PL, A.PR, padded);
    DTWGB_CUDA(cudaGetLastError());
    if (q) {
        const int64_t qoff = span + (int64_t)p * pad;
        A.qbase = qoff + A.PL;
        stage_one_kernel<<<(unsigned)((qlen + pad + 255) / 256), 256, 0, st>>>(q, qlen, A.PL, A.PR,
                                                                              padded + qoff);
        DTWGB_CUDA(cudaGetLastError());
    }
    A.padded = padded;
    return launch_band(A, shape, st);
}

}  // namespace

}  // namespace dtwgb

using namespace dtwgb;

extern "C" int32_t dtw_max_band_cells(void) { return kMaxG * kMaxK; }

extern "C" int dtw_pairwise(const float *values, const int64_t *offsets, int32_t p,
                            int32_t window, uint32_t flags, float *out_D, void *stream)
{
    clear_error();
    cudaStream_t st = (cudaStream_t)stream;
    if (p < 1) { set_error("p = %d must be >= 1", p); return DTW_EINVAL; }
    if (!values || !offsets || !out_D) { set_error("NULL pointer argument"); return DTW_EINVAL; }
    const bool host_io = flags & DTW_HOST_IO;
    const bool strict = flags & DTW_BAND_STRICT;
    const bool packed = flags & DTW_OUT_PACKED_UPPER;

    // offsets on the host for validation and shape selection
    int64_t *hoff = nullptr;
    int64_t *hbuf = nullptr;
    if (host_io) {
        hoff = const_cast<int64_t *>(offsets);
    } else {
        hbuf = (int64_t *)malloc(sizeof(int64_t) * ((size_t)p + 1));
        if (!hbuf) { set_error("host malloc failed"); return DTW_ENOMEM; }
        cudaError_t e = cudaMemcpyAsync(hbuf, offsets, sizeof(int64_t) * ((size_t)p + 1),
                                        cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) { free(hbuf); return cuda_fail(e, "reading offsets"); }
        hoff = hbuf;
    }
    SetInfo info;
    int rc = check_offsets(hoff, p, info);
    if (rc) { free(hbuf); return rc; }
    const int64_t hspan = hoff[p] - hoff[0];
    const int64_t wb = band_bound(info.minlen, info.maxlen, window, strict);
    const int64_t wneed = 2 * wb + 1;
    if (wneed > dtw_max_band_cells()) {
        free(hbuf);
        set_error("band of %lld cells per row exceeds this build's maximum of %d", (long long)wneed,
                  dtw_max_band_cells());
        return DTW_EUNSUPPORTED;
    }
    Shape shape;
    if (!pick_shape((int)wneed, (int)info.minlen, shape)) {
        free(hbuf);
        set_error("no kernel shape for a band of %lld cells", (long long)wneed);
        return DTW_EUNSUPPORTED;
    }
    const int64_t n_pairs = (int64_t)p * (p - 1) / 2;
    const size_t out_elems = packed ? (size_t)n_pairs : (size_t)p * (size_t)p;

    // device views of the inputs and the output
    DevBuf dv, doff, dout;
    const float *vals = values;
    const int64_t *offs = offsets;
    float *out = out_D;
    if (host_io) {
        if ((rc = alloc(dv, sizeof(float) * (size_t)info.total, st)) ||
            (rc = alloc(doff, sizeof(int64_t) * ((size_t)p + 1), st)) ||
            (rc = alloc(dout, sizeof(float) * out_elems, st))) {
            free(hbuf);
            return rc;
        }
        DTWGB_CUDA(cudaMemcpyAsync(dv.p, values, sizeof(float) * (size_t)info.total,
                                   cudaMemcpyHostToDevice, st));
        DTWGB_CUDA(cudaMemcpyAsync(doff.p, offsets, sizeof(int64_t) * ((size_t)p + 1),
                                   cudaMemcpyHostToDevice, st));
        vals = (const float *)dv.p;
        offs = (const int64_t *)doff.p;
        out = (float *)dout.p;
    }
    free(hbuf);
    if (flags & DTW_CHECK_FINITE) {
        if ((rc = scan_finite(vals, info.total, st, "values"))) return rc;
    }

    if (n_pairs > 0) {
        BandArgs A{};
        A.offsets = offs;
        A.p = p;
        A.n_pairs = n_pairs;
        A.window = window;
        A.strict = strict ? 1 : 0;
        A.src = SRC_TRIANGLE;
        A.out_mode = packed ? OUT_PACKED : OUT_FULL;
        A.out = out;
        if ((rc = stage_and_launch(A, shape, wb, vals, offs, hspan, p, nullptr, 0, st))) return rc;
    }
    if (!packed) {
        zero_diagonal_kernel<<<(unsigned)((p + 255) / 256), 256, 0, st>>>(out, p);
        DTWGB_CUDA(cudaGetLastError());
    }
    if (host_io) {
        DTWGB_CUDA(cudaMemcpyAsync(out_D, out, sizeof(float) * out_elems, cudaMemcpyDeviceToHost,
                                   st));
        DTWGB_CUDA(cudaStreamSynchronize(st));
    }
    return DTW_OK;
}

extern "C" int dtw_query(const float *query, int32_t qlen, const float *values,
                         const int64_t *offsets, int32_t p, int32_t window, uint32_t flags,
                         float *out, void *stream)
{
    clear_error();
    cudaStream_t st = (cudaStream_t)stream;
    if (p < 1) { set_error("p = %d must be >= 1", p); return DTW_EINVAL; }
    if (qlen < 1) { set_error("qlen = %d must be >= 1", qlen); return DTW_EINVAL; }
    if (!query || !values || !offsets || !out) { set_error("NULL pointer argument"); return DTW_EINVAL; }
    const bool host_io = flags & DTW_HOST_IO;
    const bool strict = flags & DTW_BAND_STRICT;

    int64_t *hoff = nullptr, *hbuf = nullptr;
    if (host_io) {
        hoff = const_cast<int64_t *>(offsets);
    } else {
        hbuf = (int64_t *)malloc(sizeof(int64_t) * ((size_t)p + 1));
        if (!hbuf) { set_error("host malloc failed"); return DTW_ENOMEM; }
        cudaError_t e = cudaMemcpyAsync(hbuf, offsets, sizeof(int64_t) * ((size_t)p + 1),
                                        cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) { free(hbuf); return cuda_fail(e, "reading offsets"); }
        hoff = hbuf;
    }
    SetInfo info;
    int rc = check_offsets(hoff, p, info);
    if (rc) { free(hbuf); return rc; }
    const int64_t hspan = hoff[p] - hoff[0];
    const int64_t lo = info.minlen < qlen ? info.minlen : qlen;
    const int64_t hi = info.maxlen > qlen ? info.maxlen : qlen;
    const int64_t wb = band_bound(lo, hi, window, strict);
    const int64_t wneed = 2 * wb + 1;
    Shape shape;
    if (wneed > dtw_max_band_cells() || !pick_shape((int)wneed, (int)lo, shape)) {
        free(hbuf);
        set_error("band of %lld cells per row exceeds this build's maximum of %d", (long long)wneed,
                  dtw_max_band_cells());
        return DTW_EUNSUPPORTED;
    }
    DevBuf dq, dv, doff, dout;
    const float *q = query, *vals = values;
    const int64_t *offs = offsets;
    float *o = out;
    if (host_io) {
        if ((rc = alloc(dq, sizeof(float) * (size_t)qlen, st)) ||
            (rc = alloc(dv, sizeof(float) * (size_t)info.total, st)) ||
            (rc = alloc(doff, sizeof(int64_t) * ((size_t)p + 1), st)) ||
            (rc = alloc(dout, sizeof(float) * (size_t)p, st))) {
            free(hbuf);
            return rc;
        }
        DTWGB_CUDA(cudaMemcpyAsync(dq.p, query, sizeof(float) * (size_t)qlen,
                                   cudaMemcpyHostToDevice, st));
        DTWGB_CUDA(cudaMemcpyAsync(dv.p, values, sizeof(float) * (size_t)info.total,
                                   cudaMemcpyHostToDevice, st));
        DTWGB_CUDA(cudaMemcpyAsync(doff.p, offsets, sizeof(int64_t) * ((size_t)p + 1),
                                   cudaMemcpyHostToDevice, st));
        q = (const float *)dq.p;
        vals = (const float *)dv.p;
        offs = (const int64_t *)doff.p;
        o = (float *)dout.p;
    }
    free(hbuf);
    if (flags & DTW_CHECK_FINITE) {
        if ((rc = scan_finite(q, qlen, st, "query values"))) return rc;
        if ((rc = scan_finite(vals, info.total, st, "values"))) return rc;
    }
    BandArgs A{};
    A.offsets = offs;
    A.qlen = qlen;
    A.p = p;
    A.n_pairs = p;
    A.window = window;
    A.strict = strict ? 1 : 0;
    A.src = SRC_QUERY;
    A.out_mode = OUT_ROW;
    A.out = o;
    if ((rc = stage_and_launch(A, shape, wb, vals, offs, hspan, p, q, qlen, st))) return rc;
    if (host_io) {
        DTWGB_CUDA(cudaMemcpyAsync(out, o, sizeof(float) * (size_t)p, cudaMemcpyDeviceToHost, st));
        DTWGB_CUDA(cudaStreamSynchronize(st));
    }
    return DTW_OK;
}
