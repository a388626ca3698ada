// dtw_band.cu -- all-pairs and 1-vs-N windowed DTW on sm_103a: entry points,
// staging and shape selection (the kernels are in band_kernels.cuh).
//
// Design of the kernels:
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
#include <algorithm>
#include <vector>

#include "band_kernels.cuh"
#include "band_multirow.cuh"
#include "band_tworow.cuh"

namespace dtwgb {

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

// Estimated warp-instructions per pair (n rows, m columns, band half-width w)
// for a rotated shape: G lanes x steps x (3 per cell + masks + exchange).
double cost_rotated(int n, int K, int G, int MT)
{
    const double steps = n + G - 1 + 0.5 * (K - 1);
    return G * steps * (3.0 * K + MT + 10.0) / 32.0;
}

// The same for a two-row shape (2H slots per lane, two rows per step): per
// step H packed subtractions, 2H three-input minimums and 2H fused
// multiply-adds, the masks and the exchange; the ramp is 2G - 1 steps.  The
// factor 1.1 is its lower issue rate at half the resident warps (measured on
// 2000 x 512, w = 51: 13.15 ms against 15.75 ms for the one-row K = 13).
// A fully masked tail (MT = 2H: every slot adds a mask) costs a further 1.15,
// measured on 1000 x 768, w = 76: H = 10, G = 8 with every slot masked 5632
// GCUPS against 6511 for the one-row K = 20, G = 8 with an 8-slot tail.
double cost_tworow(int n, int H, int G, int MT)
{
    const double steps = n + 2 * G - 1 + 0.5 * (H - 1);
    const double masks = MT == 2 * H ? H : MT;
    const double full = MT == 2 * H ? 1.15 : 1.0;
    return 1.1 * full * G * steps * (5.0 * H + masks + 10.0) / 32.0;
}

// The same for a three-row shape (3H slots per lane, three rows per step): per
// step 3H subtractions, minimums and fma each, the masks and the exchange; the
// ramp is 3G - 1 steps.  The factor 1.09 is calibrated like the two-row one
// (1500 x 600, w = 65: H = 11, G = 4 in 10.97 ms against 12.61 ms for the
// one-row K = 17, G = 8).
double cost_threerow(int n, int H, int G, int MT)
{
    const double steps = n + 3 * G - 1 + 0.5 * (H - 1);
    return 1.09 * G * steps * (9.0 * H + MT + 10.0) / 32.0;
}

// Same estimate for a strip shape: every strip visits its band rows with a
// 31-step skew; rows that an edge of the band crosses pay a mask addition
// per cell.
double cost_strip(int n, int m, int w, int K)
{
    const int WS = 32 * K;
    double c = 0.0;
    for (int j0 = 1; j0 <= m; j0 += WS) {
        const int rs = j0 - w > 1 ? j0 - w : 1;
        const int re = j0 + WS - 1 + w < n ? j0 + WS - 1 + w : n;
        const int rows = re - rs + 1;
        if (rows <= 0) continue;
        const int jmax = j0 + WS - 1 < m ? j0 + WS - 1 : m;
        // rows cut by the upper edge (columns beyond r + w) and by the lower edge (j0 < r - w)
        const int top_hi = (jmax - w - 1 < re ? jmax - w - 1 : re);
        const int top = top_hi >= rs ? top_hi - rs + 1 : 0;
        const int bot_lo = (j0 + w + 1 > rs ? j0 + w + 1 : rs);
        const int bot = re >= bot_lo ? re - bot_lo + 1 : 0;
        const int edge = (top ? top + 32 : 0) + (bot ? bot + 32 : 0);
        // masked steps: one mask addition per cell and the block's K + 7 masks
        c += (rows + 31) * (3.0 * K + 6.0) + (edge < rows ? edge : rows) * (K + 3.0 * (K + 7) / 8.0);
    }
    return c;
}

// Kernel shape for pairs of `n` rows and `m` columns with band half-width
// `w`: the cheapest estimate over the compiled rotated shapes (if the band
// row fits, 2w+1 <= 512) and the strip shapes.
namespace {

constexpr int kMaxG = 32;
constexpr int kMaxK = 16;

struct Shape {
    int kind;      // 0: rotated band kernel, 1: strip kernel, 2: two-row rotated kernel,
                   // 3: three-row rotated kernel (K = 3H)
    int K, G, MT;  // rotated: slots per lane, lanes per pair, masked tail (1, 4 or K); strip: K;
                   // two-row: K = 2H slots per lane, G lanes, masked tail (1, 4 or K)
    int ppl;       // rotated: pairs per lane, 1 (dtw_band_kernel) or 2 (dtw_band2_kernel)
};

// Pairs per lane: 1 unless DTWGB_PAIRS_PER_LANE=2 is set in the environment
// (the two layouts run the 2000 x 512, w = 51 set at the same speed; one pair
// per lane is faster on small sets).
int pairs_per_lane_default()
{
    const char *e = getenv("DTWGB_PAIRS_PER_LANE");
    return (e && e[0] == '2') ? 2 : 1;
}

// DTWGB_SHAPE forces a shape ("strip:K" or "rot:K:G[:ppl]"), for measurement
// and tests; an override that cannot run this band is ignored.
bool forced_shape(int wneed, bool uniform, Shape &out)
{
    const char *e = getenv("DTWGB_SHAPE");
    if (!e || !*e) return false;
    int K = 0, G = 0, ppl = 1;
    if (sscanf(e, "strip:%d", &K) == 1) {
        if (K != 4 && K != 8 && K != 16) return false;
        out = Shape{1, K, 32, 0, 1};
        return true;
    }
    int H = 0;
    if (sscanf(e, "three:%d:%d", &H, &G) == 2) {
        const int MT = uniform ? threerow_masked_tail(H, G, wneed) : 3 * H;
        if (G >= 2 && G <= 32 && (G & (G - 1)) == 0 && G * 3 * H >= wneed &&
            threerow_shape_compiled(H, MT)) {
            out = Shape{3, 3 * H, G, MT, 1};
            return true;
        }
        return false;
    }
    if (sscanf(e, "two:%d:%d", &H, &G) == 2) {
        const int MT = uniform ? tworow_masked_tail(H, G, wneed) : 2 * H;
        if (G >= 2 && G <= 32 && (G & (G - 1)) == 0 && G * 2 * H >= wneed &&
            tworow_shape_compiled(H, MT)) {
            out = Shape{2, 2 * H, G, MT, 1};
            return true;
        }
        return false;
    }
    const int got = sscanf(e, "rot:%d:%d:%d", &K, &G, &ppl);
    const int MT = uniform ? rot_masked_tail(K, G, wneed) : K;
    if (got >= 2 && G >= 2 && G <= 32 && (G & (G - 1)) == 0 && G * K >= wneed &&
        rot_shape_compiled(K, MT, false)) {
        out = Shape{0, K, G, MT, (got == 3 && ppl == 2) ? 2 : 1};
        return true;
    }
    return false;
}

// `uniform`: every pair of the call has the band half-width w (series of one
// length).  Otherwise a pair may have a narrower band than w, so its slots
// beyond its own band can lie anywhere in the lanes, and only a full masked
// tail (MT = K) covers them.
bool pick_shape(int n, int m, int w, bool uniform, Shape &out)
{
    const int wneed = 2 * w + 1;
    if (forced_shape(wneed, uniform, out)) return true;
    double best = 1e300;
    bool ok = false;
    for (int K : kRotKsStatic) {
        for (int G = 2; G <= kMaxG; G *= 2) {  // every G whose slots hold the band
            if (G * K < wneed) continue;
            const int MT = uniform ? rot_masked_tail(K, G, wneed) : K;
            if (!rot_shape_compiled(K, MT, false)) continue;
            const double c = cost_rotated(n, K, G, MT);
            if (c < best) {
                best = c;
                out = Shape{0, K, G, MT, pairs_per_lane_default()};
                ok = true;
            }
            break;  // a larger G only adds lanes beyond the band
        }
    }
    for (int H : kTwoRowHs) {
        for (int G = 2; G <= kMaxG; G *= 2) {  // the two-row shapes, likewise
            if (G * 2 * H < wneed) continue;
            const int MT = uniform ? tworow_masked_tail(H, G, wneed) : 2 * H;
            if (!tworow_shape_compiled(H, MT)) break;
            const double c = cost_tworow(n, H, G, MT);
            if (c < best) {
                best = c;
                out = Shape{2, 2 * H, G, MT, 1};
                ok = true;
            }
            break;
        }
    }
    for (int H : kThreeRowHs) {
        if (!uniform) break;  // compiled with the tails of one-length sets only
        for (int G = 2; G <= kMaxG; G *= 2) {
            if (G * 3 * H < wneed) continue;
            const int MT = threerow_masked_tail(H, G, wneed);
            if (!threerow_shape_compiled(H, MT)) break;
            const double c = cost_threerow(n, H, G, MT);
            if (c < best) {
                best = c;
                out = Shape{3, 3 * H, G, MT, 1};
                ok = true;
            }
            break;
        }
    }
    static const int Ks_strip[] = {4, 8, 16};
    for (int K : Ks_strip) {
        const double c = cost_strip(n, m, w, K);
        if (c < best) {
            best = c;
            out = Shape{1, K, 32, 0, 1};
            ok = true;
        }
    }
    // For a set of several lengths the model only sees the extreme pair (the
    // shortest series against the longest, the widest band), for which 512-column
    // strips look best; most pairs are closer in length and narrower, where they
    // waste more.  Measured on 700 series of lengths U[64, 2048] (5 % band widened
    // to |n - m|): K = 8 4142 against K = 16 3546 GCUPS (on one-length sets the two
    // are within 2 %).
    if (!uniform && out.kind == 1 && out.K == 16) out.K = 8;
    return ok;
}

int launch_band(BandArgs A, const Shape &s, cudaStream_t st)
{
    A.G = s.G;
    A.log2G = 0;
    while ((1 << A.log2G) < s.G) ++A.log2G;
    if (s.kind == 2) return launch_tworow(A, s.K / 2, s.MT, st);
    if (s.kind == 3) return launch_threerow(A, s.K / 3, s.MT, st);
    return s.ppl == 2 ? launch_band2(A, s.K, s.MT, st) : launch_band1(A, s.K, s.MT, st);
}

// Pads of the staged copy for a band-kernel shape (see stage_and_launch).
void shape_pads(const Shape &s, int64_t wb, int32_t &PL, int32_t &PR)
{
    if (s.kind == 0) {
        PL = (int32_t)((wb > s.G ? wb : s.G) + 2);
        PR = s.G * s.K + s.K + s.G + 2;
    } else if (s.kind == 2) {
        PL = tworow_pad_left(wb, s.G);
        PR = tworow_pad_right(s.G, s.K / 2);
    } else if (s.kind == 3) {
        PL = multirow_pad_left(wb, 3, s.G);
        PR = multirow_pad_right(3, s.G, s.K / 3);
    } else {
        // strip: x rows down to 1-31 and up to n+41, y columns up to m+32K-1
        PL = 34;
        PR = (32 * s.K > 48 ? 32 * s.K : 48) + 8;
    }
}

// Band half-width bound over every pair of lengths in [minlen, maxlen], and
// the same bound for a query of length qlen.
int64_t band_bound(int64_t minlen, int64_t maxlen, int32_t window, bool strict,
                   bool permille = false)
{
    if (permille && window >= 0) window = (int32_t)((int64_t)window * maxlen / 1000);
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
int stage_and_launch(BandArgs A, const Shape &shape, int64_t wb, int64_t maxlen,
                     const float *vals, const int64_t *offs, int64_t span, int32_t p,
                     const float *q, int64_t qlen, cudaStream_t st)
{
    shape_pads(shape, wb, A.PL, A.PR);
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
    if (shape.kind != 1) return launch_band(A, shape, st);
    int64_t warps = 0;
    if ((rc = strip_warps(shape.K, A.n_pairs, &warps))) return rc;
    const int64_t stride = strip_bnd_stride(maxlen);
    DevBuf bnd;
    if ((rc = alloc(bnd, sizeof(float) * (size_t)(stride * warps), st))) return rc;
    return launch_strip(A, shape.K, (float *)bnd.p, stride, warps, st);
}

// Series of a set of several lengths in order of length (stable), as int32: the
// kernels visit the set in that order, so that the lane groups of a warp get
// pairs of similar lengths (outputs keep the original indices).  Empty for a
// one-length set or fewer than three series.
std::vector<int32_t> length_order(const int64_t *hoff, int32_t p, const SetInfo &info)
{
    std::vector<int32_t> order;
    if (p < 3 || info.minlen == info.maxlen) return order;
    order.resize((size_t)p);
    for (int32_t i = 0; i < p; ++i) order[(size_t)i] = i;
    std::stable_sort(order.begin(), order.end(), [hoff](int32_t x, int32_t y) {
        return hoff[x + 1] - hoff[x] < hoff[y + 1] - hoff[y];
    });
    return order;
}

// Upload a visiting order into a stream-ordered buffer and point A at it.
int set_order(BandArgs &A, const std::vector<int32_t> &order, DevBuf &buf, cudaStream_t st)
{
    if (order.empty()) return DTW_OK;
    int rc = alloc(buf, sizeof(int32_t) * order.size(), st);
    if (rc) return rc;
    DTWGB_CUDA(cudaMemcpyAsync(buf.p, order.data(), sizeof(int32_t) * order.size(),
                               cudaMemcpyHostToDevice, st));
    A.perm = (const int32_t *)buf.p;
    return DTW_OK;
}

}  // namespace

// Host launchers shared with the batch planner (batch.cu).
int launch_stage_set(const float *values, const int64_t *offsets, int32_t p, int32_t PL,
                     int32_t PR, float *padded, cudaStream_t st)
{
    if (p > 0) stage_kernel<<<(unsigned)p, 256, 0, st>>>(values, offsets, PL, PR, padded);
    DTWGB_CUDA(cudaGetLastError());
    return DTW_OK;
}

int launch_stage_one(const float *v, int64_t len, int32_t PL, int32_t PR, float *dst,
                     cudaStream_t st)
{
    const int64_t total = len + PL + PR;
    stage_one_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(v, len, PL, PR, dst);
    DTWGB_CUDA(cudaGetLastError());
    return DTW_OK;
}

int launch_zero_diagonal(float *D, int64_t p, cudaStream_t st)
{
    zero_diagonal_kernel<<<(unsigned)((p + 255) / 256), 256, 0, st>>>(D, p);
    DTWGB_CUDA(cudaGetLastError());
    return DTW_OK;
}

}  // namespace dtwgb

using namespace dtwgb;

namespace dtwgb {

int dtw_list_prepare(const float *values, const int64_t *offsets, const int64_t *offsets_host,
                     int32_t p, int32_t window, uint32_t flags, DtwListCtx *ctx, cudaStream_t st)
{
    SetInfo info;
    int rc = check_offsets(offsets_host, p, info);
    if (rc) return rc;
    const bool strict = flags & DTW_BAND_STRICT, permille = flags & DTW_WINDOW_PERMILLE;
    const int64_t wb = band_bound(info.minlen, info.maxlen, window, strict, permille);
    Shape shape;
    if (!pick_shape((int)info.minlen, (int)info.maxlen, (int)wb, info.minlen == info.maxlen, shape)) {
        set_error("no kernel shape for a band of %lld cells", (long long)(2 * wb + 1));
        return DTW_EUNSUPPORTED;
    }
    BandArgs A{};
    A.offsets = offsets;
    A.p = p;
    A.window = (permille && window > 0) ? -1 : window;
    A.wpermille = (permille && window > 0) ? window : 0;
    A.strict = strict ? 1 : 0;
    A.src = SRC_LIST;
    A.out_mode = OUT_LIST;
    shape_pads(shape, wb, A.PL, A.PR);
    A.G = shape.G;
    A.log2G = 0;
    while ((1 << A.log2G) < shape.G) ++A.log2G;
    const int64_t span = offsets_host[p] - offsets_host[0];
    const size_t elems = (size_t)(span + (int64_t)p * (A.PL + A.PR));
    if ((rc = scratch_alloc(&ctx->padded, sizeof(float) * elems, st))) return rc;
    stage_kernel<<<(unsigned)p, 256, 0, st>>>(values, offsets, A.PL, A.PR, (float *)ctx->padded);
    DTWGB_CUDA(cudaGetLastError());
    A.padded = (const float *)ctx->padded;
    ctx->A = A;
    ctx->kind = shape.kind;
    ctx->K = shape.K;
    ctx->G = shape.G;
    ctx->MT = shape.MT;
    ctx->maxlen = info.maxlen;
    ctx->bnd = nullptr;
    ctx->bnd_pairs = 0;
    return DTW_OK;
}

int dtw_list_run(DtwListCtx *ctx, const int32_t *pa, const int32_t *pb, int64_t npairs, float *out,
                 cudaStream_t st)
{
    if (npairs <= 0) return DTW_OK;
    BandArgs A = ctx->A;
    A.pa = pa;
    A.pb = pb;
    A.n_pairs = npairs;
    A.out = out;
    if (ctx->kind == 0) return ctx->G > 0 ? launch_band1(A, ctx->K, ctx->MT, st) : DTW_EUNSUPPORTED;
    if (ctx->kind == 2) return launch_tworow(A, ctx->K / 2, ctx->MT, st);
    if (ctx->kind == 3) return launch_threerow(A, ctx->K / 3, ctx->MT, st);
    int64_t warps = 0;
    int rc = strip_warps(ctx->K, npairs, &warps);
    if (rc) return rc;
    const int64_t stride = strip_bnd_stride(ctx->maxlen);
    if (!ctx->bnd || warps > ctx->warps) {  // grow the strip buffers
        if (ctx->bnd) scratch_free(ctx->bnd, st);
        ctx->bnd = nullptr;
        if ((rc = scratch_alloc(&ctx->bnd, sizeof(float) * (size_t)(stride * warps), st))) return rc;
        ctx->warps = warps;
    }
    return launch_strip(A, ctx->K, (float *)ctx->bnd, stride, warps, st);
}

void dtw_list_release(DtwListCtx *ctx, cudaStream_t st)
{
    if (ctx->padded) scratch_free(ctx->padded, st);
    if (ctx->bnd) scratch_free(ctx->bnd, st);
    ctx->padded = ctx->bnd = nullptr;
}

}  // namespace dtwgb

extern "C" int dtw_pairs(const float *values, const int64_t *offsets, int32_t p,
                         const int32_t *pair_a, const int32_t *pair_b, int64_t npairs,
                         int32_t window, uint32_t flags, float *out, void *stream)
{
    clear_error();
    cudaStream_t st = (cudaStream_t)stream;
    if (p < 1) { set_error("p = %d must be >= 1", p); return DTW_EINVAL; }
    if (npairs < 0) { set_error("npairs = %lld must be >= 0", (long long)npairs); return DTW_EINVAL; }
    if (!values || !offsets || (npairs > 0 && (!pair_a || !pair_b || !out))) {
        set_error("NULL pointer argument");
        return DTW_EINVAL;
    }
    // offsets and pair indices to the host for validation
    std::vector<int64_t> hoff((size_t)p + 1);
    std::vector<int32_t> ha((size_t)npairs), hb((size_t)npairs);
    cudaError_t e = cudaMemcpyAsync(hoff.data(), offsets, sizeof(int64_t) * ((size_t)p + 1),
                                    cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && npairs > 0)
        e = cudaMemcpyAsync(ha.data(), pair_a, sizeof(int32_t) * (size_t)npairs,
                            cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && npairs > 0)
        e = cudaMemcpyAsync(hb.data(), pair_b, sizeof(int32_t) * (size_t)npairs,
                            cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "reading offsets and pairs");
    for (int64_t t = 0; t < npairs; ++t)
        if (ha[t] < 0 || ha[t] >= p || hb[t] < 0 || hb[t] >= p) {
            set_error("pair %lld = (%d, %d) has an index outside [0, %d)", (long long)t, ha[t], hb[t], p);
            return DTW_EINVAL;
        }
    if (npairs == 0) return DTW_OK;
    DtwListCtx ctx;
    int rc = dtw_list_prepare(values, offsets, hoff.data(), p, window, flags, &ctx, st);
    if (!rc) rc = dtw_list_run(&ctx, pair_a, pair_b, npairs, out, st);
    dtw_list_release(&ctx, st);
    return rc;
}

extern "C" int32_t dtw_max_band_cells(void) { return kMaxG * kMaxK; }

extern "C" int dtw_describe_shape(int32_t minlen, int32_t maxlen, int32_t window, uint32_t flags,
                                  char *buf, int32_t buflen)
{
    clear_error();
    if (minlen < 1 || maxlen < minlen) {
        set_error("lengths %d..%d are not a valid range", minlen, maxlen);
        return DTW_EINVAL;
    }
    if (!buf || buflen < 1) { set_error("NULL or empty buffer"); return DTW_EINVAL; }
    const int64_t wb = band_bound(minlen, maxlen, window, flags & DTW_BAND_STRICT,
                                  flags & DTW_WINDOW_PERMILLE);
    Shape s;
    if (!pick_shape(minlen, maxlen, (int)wb, minlen == maxlen, s)) {
        set_error("no kernel shape for a band of %lld cells", (long long)(2 * wb + 1));
        return DTW_EUNSUPPORTED;
    }
    if (s.kind == 0)
        snprintf(buf, (size_t)buflen, "dtw_band_kernel<K=%d,MT=%d> G=%d pairs_per_lane=%d", s.K,
                 s.MT, s.G, s.ppl);
    else if (s.kind == 2)
        snprintf(buf, (size_t)buflen, "dtw_tworow_kernel<H=%d,MT=%d> G=%d", s.K / 2, s.MT, s.G);
    else if (s.kind == 3)
        snprintf(buf, (size_t)buflen, "dtw_multirow_kernel<R=3,H=%d,MT=%d> G=%d", s.K / 3, s.MT,
                 s.G);
    else
        snprintf(buf, (size_t)buflen, "dtw_strip_kernel<K=%d>", s.K);
    return DTW_OK;
}

extern "C" int dtw_pairwise(const float *values, const int64_t *offsets, int32_t p,
                            int32_t window, uint32_t flags, float *out_D, void *stream)
{
    clear_error();
    cudaStream_t st = (cudaStream_t)stream;
    if (p < 1) { set_error("p = %d must be >= 1", p); return DTW_EINVAL; }
    if (!values || !offsets || !out_D) { set_error("NULL pointer argument"); return DTW_EINVAL; }
    const bool host_io = flags & DTW_HOST_IO;
    const bool offs_host = (flags & DTW_OFFSETS_HOST) && !host_io;
    const bool strict = flags & DTW_BAND_STRICT;
    const bool packed = flags & DTW_OUT_PACKED_UPPER;

    // offsets on the host for validation and shape selection
    int64_t *hoff = nullptr;
    int64_t *hbuf = nullptr;
    if (host_io || offs_host) {
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
    const std::vector<int32_t> order =
        (flags & DTW_OUT_PACKED_UPPER) ? std::vector<int32_t>() : length_order(hoff, p, info);
    const bool permille = flags & DTW_WINDOW_PERMILLE;
    const int64_t wb = band_bound(info.minlen, info.maxlen, window, strict, permille);
    Shape shape;
    if (!pick_shape((int)info.minlen, (int)info.maxlen, (int)wb, info.minlen == info.maxlen, shape)) {
        free(hbuf);
        set_error("no kernel shape for a band of %lld cells", (long long)(2 * wb + 1));
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
    } else if (offs_host) {  // the kernels read offsets on the device
        if ((rc = alloc(doff, sizeof(int64_t) * ((size_t)p + 1), st))) return rc;
        DTWGB_CUDA(cudaMemcpyAsync(doff.p, offsets, sizeof(int64_t) * ((size_t)p + 1),
                                   cudaMemcpyHostToDevice, st));
        offs = (const int64_t *)doff.p;
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
        A.window = (permille && window > 0) ? -1 : window;
        A.wpermille = (permille && window > 0) ? window : 0;
        A.strict = strict ? 1 : 0;
        A.src = SRC_TRIANGLE;
        A.out_mode = packed ? OUT_PACKED : OUT_FULL;
        A.out = out;
        DevBuf dorder;
        if ((rc = set_order(A, order, dorder, st))) return rc;
        if ((rc = stage_and_launch(A, shape, wb, info.maxlen, vals, offs, hspan, p, nullptr, 0, st)))
            return rc;
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
    const bool offs_host = (flags & DTW_OFFSETS_HOST) && !host_io;
    const bool strict = flags & DTW_BAND_STRICT;

    int64_t *hoff = nullptr, *hbuf = nullptr;
    if (host_io || offs_host) {
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
    const std::vector<int32_t> order = length_order(hoff, p, info);
    const int64_t lo = info.minlen < qlen ? info.minlen : qlen;
    const int64_t hi = info.maxlen > qlen ? info.maxlen : qlen;
    const bool permille = flags & DTW_WINDOW_PERMILLE;
    const int64_t wb = band_bound(lo, hi, window, strict, permille);
    Shape shape;
    if (!pick_shape((int)lo, (int)hi, (int)wb, lo == hi, shape)) {
        free(hbuf);
        set_error("no kernel shape for a band of %lld cells", (long long)(2 * wb + 1));
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
    } else if (offs_host) {  // the kernels read offsets on the device
        if ((rc = alloc(doff, sizeof(int64_t) * ((size_t)p + 1), st))) { free(hbuf); return rc; }
        DTWGB_CUDA(cudaMemcpyAsync(doff.p, offsets, sizeof(int64_t) * ((size_t)p + 1),
                                   cudaMemcpyHostToDevice, st));
        offs = (const int64_t *)doff.p;
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
    A.window = (permille && window > 0) ? -1 : window;
    A.wpermille = (permille && window > 0) ? window : 0;
    A.strict = strict ? 1 : 0;
    A.src = SRC_QUERY;
    A.out_mode = OUT_ROW;
    A.out = o;
    DevBuf dorder;
    if ((rc = set_order(A, order, dorder, st))) return rc;
    if ((rc = stage_and_launch(A, shape, wb, hi, vals, offs, hspan, p, q, qlen, st))) return rc;
    if (host_io) {
        DTWGB_CUDA(cudaMemcpyAsync(out, o, sizeof(float) * (size_t)p, cudaMemcpyDeviceToHost, st));
        DTWGB_CUDA(cudaStreamSynchronize(st));
    }
    return DTW_OK;
}
