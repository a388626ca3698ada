// kmedoids.cu -- alternate (Voronoi-iteration) k-medoids over a DTW distance
// matrix on sm_103a.
//
// The paper offers k-medoids as the faster, locally optimal alternative to
// its MIP clustering (Mathematical background, last paragraph) and reports
// the clustering cost, the sum of distances of every series to its cluster
// centroid (Overview of method, item 5).  It does not give the algorithm;
// this is the alternate k-medoids of Park & Jun (2009):
//   assign  label_j = argmin_c D[M_c, j], ties to the smallest c, and a medoid
//           always labels itself, so no cluster is empty;
//   update  M_c = argmin over members i of S_i = sum_{j in C_c} D[i, j], with
//           sums as accurate as plain float64 ones (relative error about
//           n 2^-53: TwoSum pairs of float32 per lane, float64 across lanes);
//           a tie keeps the current medoid when it attains the minimum,
//           otherwise the smallest index wins;
// repeated while a medoid changes.  D is the symmetric matrix written by
// dtw_pairwise, so D[M_c, j] = D[j, M_c] bit for bit and the assignment reads
// medoid rows, which keeps its loads coalesced.
#include <mutex>

#include "common.cuh"

namespace dtwgb {

__global__ void kmed_assign_kernel(const float *__restrict__ D, int32_t n, int32_t k,
                                   const int32_t *__restrict__ M, int32_t *__restrict__ labels)
{
    const int32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    int32_t best = 0, own = -1;
    int32_t m0 = __ldg(M);
    float bd = __ldg(D + (int64_t)m0 * n + j);
    if (m0 == j) own = 0;
    for (int32_t c = 1; c < k; ++c) {
        const int32_t mc = __ldg(M + c);
        if (mc == j) own = c;
        const float d = __ldg(D + (int64_t)mc * n + j);
        if (d < bd) {
            bd = d;
            best = c;
        }
    }
    labels[j] = own >= 0 ? own : best;
}

// (hi, lo) += x by Knuth's TwoSum: after m additions hi + lo is within about
// m 2^-48 of the sum (relative), at float32 speed -- GB300's float64 rate is
// far below its float32 one
__device__ __forceinline__ void two_sum_add(float &hi, float &lo, float x)
{
    const float s = __fadd_rn(hi, x);
    const float bp = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(x, bp));
    hi = s;
    lo = __fadd_rn(lo, err);
}

// S_i = sum over j with label_j == label_i of D[i, j], one warp per row i.  Each
// lane sums its entries j = lane, lane + 32, ... in order as a TwoSum pair of
// float32 (non-members add an exact 0); the lanes' pairs are added in float64.
// An infinite entry makes S_i infinite.
__global__ void kmed_rowsum_kernel(const float *__restrict__ D, int32_t n,
                                   const int32_t *__restrict__ labels, double *__restrict__ S,
                                   int vec4)
{
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= n) return;
    const int32_t i = (int32_t)warp;
    const int32_t c = __ldg(labels + i);
    const float *row = D + (int64_t)i * n;
    float hi = 0.f, lo = 0.f;
    if (vec4) {  // n % 4 == 0 and D, labels 16-byte aligned (checked on the host)
        const float4 *r4 = reinterpret_cast<const float4 *>(row);
        const int4 *l4 = reinterpret_cast<const int4 *>(labels);
        auto take = [&](const float4 &v, const int4 &lb) {
            two_sum_add(hi, lo, lb.x == c ? v.x : 0.f);
            two_sum_add(hi, lo, lb.y == c ? v.y : 0.f);
            two_sum_add(hi, lo, lb.z == c ? v.z : 0.f);
            two_sum_add(hi, lo, lb.w == c ? v.w : 0.f);
        };
        const int32_t nq = n >> 2;
        int32_t q = lane;
        // four row loads in flight per lane; the additions keep the order q, q + 32, ...
        for (; q + 96 < nq; q += 128) {
            float4 v[4];
            int4 lb[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                v[u] = __ldg(r4 + q + 32 * u);
                lb[u] = __ldg(l4 + q + 32 * u);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) take(v[u], lb[u]);
        }
        for (; q < nq; q += 32) take(__ldg(r4 + q), __ldg(l4 + q));
    } else {
        for (int32_t j = lane; j < n; j += 32)
            two_sum_add(hi, lo, __ldg(labels + j) == c ? __ldg(row + j) : 0.f);
    }
    // once hi is infinite, lo may hold inf - inf
    double acc = isinf(hi) ? (double)hi : (double)hi + (double)lo;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) S[i] = acc;
}

// One block per cluster: argmin of S over the cluster's members with the
// tie rules above; writes the new medoid and raises *changed if it moved.
__global__ void kmed_update_kernel(int32_t n, const int32_t *__restrict__ labels,
                                   const double *__restrict__ S, const int32_t *__restrict__ M,
                                   int32_t *__restrict__ Mnew, int32_t *__restrict__ changed)
{
    const int32_t c = blockIdx.x;
    double bs = __longlong_as_double(0x7ff0000000000000LL);  // +inf
    int32_t bi = INT32_MAX;
    // four labels and sums in flight per thread (the scan is latency-bound otherwise)
    const int32_t step = (int32_t)blockDim.x;
    for (int32_t i0 = threadIdx.x; i0 < n; i0 += 4 * step) {
        int32_t lb[4];
        double sv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int32_t i = i0 + u * step;
            lb[u] = i < n ? __ldg(labels + i) : -1;
            sv[u] = i < n ? __ldg(S + i) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int32_t i = i0 + u * step;
            if (lb[u] == c && (sv[u] < bs || (sv[u] == bs && i < bi))) {
                bs = sv[u];
                bi = i;
            }
        }
    }
    __shared__ double ss[32];
    __shared__ int32_t si[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double s2 = __shfl_down_sync(0xffffffffu, bs, o);
        const int32_t i2 = __shfl_down_sync(0xffffffffu, bi, o);
        if (s2 < bs || (s2 == bs && i2 < bi)) {
            bs = s2;
            bi = i2;
        }
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        ss[w] = bs;
        si[w] = bi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 1; q < (int)(blockDim.x >> 5); ++q)
            if (ss[q] < bs || (ss[q] == bs && si[q] < bi)) {
                bs = ss[q];
                bi = si[q];
            }
        const int32_t cur = M[c];
        const int32_t chosen = (S[cur] == bs) ? cur : bi;
        Mnew[c] = chosen;
        if (chosen != cur) atomicOr(changed, 1);
    }
}

// Clustering cost: per-block float64 partial sums of D[M_{label_j}, j], then
// one block adds the partials in a fixed order (deterministic).
__global__ void kmed_cost_partial_kernel(const float *__restrict__ D, int32_t n,
                                         const int32_t *__restrict__ M,
                                         const int32_t *__restrict__ labels,
                                         double *__restrict__ partial)
{
    double acc = 0.0;
    for (int32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
        acc += (double)__ldg(D + (int64_t)__ldg(M + __ldg(labels + j)) * n + j);
    __shared__ double sh[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += sh[q];
        partial[blockIdx.x] = t;
    }
}

__global__ void kmed_cost_final_kernel(const double *__restrict__ partial, int32_t nb,
                                       double *__restrict__ out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double t = 0.0;
        for (int32_t q = 0; q < nb; ++q) t += partial[q];
        *out = t;
    }
}

namespace {

constexpr int kCostBlocks = 120;

struct Scratch {
    double *S;
    double *partial;
    double *cost;
    int32_t *Ma, *Mb, *flag;
};

size_t scratch_bytes(int32_t n, int32_t k)
{
    size_t b = 0;
    b += sizeof(double) * (size_t)n;        // S
    b += sizeof(double) * kCostBlocks;      // partial
    b += sizeof(double);                    // cost
    b += sizeof(int32_t) * (2 * (size_t)k + 2);  // Ma, Mb, flag (+pad)
    return b + 256;
}

Scratch carve(void *base, int32_t n, int32_t k)
{
    char *p = (char *)base;
    Scratch s;
    s.S = (double *)p;
    p += sizeof(double) * (size_t)n;
    s.partial = (double *)p;
    p += sizeof(double) * kCostBlocks;
    s.cost = (double *)p;
    p += sizeof(double);
    s.Ma = (int32_t *)p;
    p += sizeof(int32_t) * (size_t)k;
    s.Mb = (int32_t *)p;
    p += sizeof(int32_t) * (size_t)k;
    s.flag = (int32_t *)p;
    return s;
}

}  // namespace

// The sweeps themselves on caller-provided scratch; shared by the allocating
// entry point.  `hM` holds the validated initial medoids on the host.
int kmedoids_run(const float *D, int32_t n, int32_t k, const int32_t *init, int32_t max_iter,
                 int32_t *out_medoids, int32_t *out_labels, double *out_cost, int32_t *out_iters,
                 const Scratch &s, cudaStream_t st)
{
    DTWGB_CUDA(cudaMemcpyAsync(s.Ma, init, sizeof(int32_t) * (size_t)k, cudaMemcpyDeviceToDevice,
                               st));
    int32_t *M = s.Ma, *Mn = s.Mb;
    const unsigned ab = (unsigned)((n + 255) / 256);
    const unsigned rb = (unsigned)(((int64_t)n * 32 + 255) / 256);
    const int vec4 = (n % 4 == 0) && ((uintptr_t)D % 16 == 0) && ((uintptr_t)out_labels % 16 == 0);
    int32_t iters = 0;
    for (int32_t it = 1; it <= max_iter; ++it) {
        DTWGB_CUDA(cudaMemsetAsync(s.flag, 0, sizeof(int32_t), st));
        kmed_assign_kernel<<<ab, 256, 0, st>>>(D, n, k, M, out_labels);
        kmed_rowsum_kernel<<<rb, 256, 0, st>>>(D, n, out_labels, s.S, vec4);
        kmed_update_kernel<<<(unsigned)k, 1024, 0, st>>>(n, out_labels, s.S, M, Mn, s.flag);
        DTWGB_CUDA(cudaGetLastError());
        int32_t h = 0;
        DTWGB_CUDA(cudaMemcpyAsync(&h, s.flag, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        DTWGB_CUDA(cudaStreamSynchronize(st));
        iters = it;
        if (!h) break;
        int32_t *t = M;
        M = Mn;
        Mn = t;
    }
    kmed_assign_kernel<<<ab, 256, 0, st>>>(D, n, k, M, out_labels);
    kmed_cost_partial_kernel<<<kCostBlocks, 256, 0, st>>>(D, n, M, out_labels, s.partial);
    kmed_cost_final_kernel<<<1, 32, 0, st>>>(s.partial, kCostBlocks, s.cost);
    DTWGB_CUDA(cudaGetLastError());
    DTWGB_CUDA(cudaMemcpyAsync(out_medoids, M, sizeof(int32_t) * (size_t)k,
                               cudaMemcpyDeviceToDevice, st));
    double hc = 0.0;
    DTWGB_CUDA(cudaMemcpyAsync(&hc, s.cost, sizeof(double), cudaMemcpyDeviceToHost, st));
    DTWGB_CUDA(cudaStreamSynchronize(st));
    if (out_cost) *out_cost = hc;
    if (out_iters) *out_iters = iters;
    return DTW_OK;
}

// Validates sizes and the initial medoids (read to the host).
int kmedoids_check(const float *D, int32_t n, int32_t k, const int32_t *init, int32_t max_iter,
                   const int32_t *out_medoids, const int32_t *out_labels, cudaStream_t st)
{
    if (n < 1) { set_error("n = %d must be >= 1", n); return DTW_EINVAL; }
    if (k < 1 || k > n) { set_error("k = %d must be in [1, n = %d]", k, n); return DTW_EINVAL; }
    if (max_iter < 1) { set_error("max_iter = %d must be >= 1", max_iter); return DTW_EINVAL; }
    if (!D || !init || !out_medoids || !out_labels) {
        set_error("NULL pointer argument");
        return DTW_EINVAL;
    }
    int32_t *h = (int32_t *)malloc(sizeof(int32_t) * (size_t)k);
    if (!h) { set_error("host malloc failed"); return DTW_ENOMEM; }
    cudaError_t e = cudaMemcpyAsync(h, init, sizeof(int32_t) * (size_t)k, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { free(h); return cuda_fail(e, "reading init_medoids"); }
    int rc = DTW_OK;
    for (int32_t c = 0; c < k && rc == DTW_OK; ++c) {
        if (h[c] < 0 || h[c] >= n) {
            set_error("init_medoids[%d] = %d is outside [0, %d)", c, h[c], n);
            rc = DTW_EINVAL;
        }
        for (int32_t d = 0; d < c && rc == DTW_OK; ++d)
            if (h[d] == h[c]) {
                set_error("init_medoids[%d] and [%d] are both %d", d, c, h[c]);
                rc = DTW_EINVAL;
            }
    }
    free(h);
    return rc;
}

// ------------------------------------------------------------------------
// Allocation-free variant.  Its scratch (the float64 sums, the cost partials,
// the two medoid sets and the convergence flag) lives in the file-scope
// device array below instead of the scratch pool, so kmedoids_fit_noalloc
// never allocates device memory.  Every GPU that loads the library holds the
// array (about 0.5 MB) until the process exits.

constexpr int32_t kNoallocMaxN = 65536;  // largest n the static scratch serves
constexpr int32_t kNoallocMaxK = 1024;   // largest k the static scratch serves
constexpr size_t kNoallocBytes = sizeof(double) * (size_t)kNoallocMaxN +
                                 sizeof(double) * kCostBlocks + sizeof(double) +
                                 sizeof(int32_t) * (2 * (size_t)kNoallocMaxK + 2) + 256;

static __device__ __align__(256) unsigned char g_kmed_noalloc_scratch[kNoallocBytes];

namespace {

constexpr int kMaxDevicesNoalloc = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[kMaxDevicesNoalloc] = {};

// Device address of the static scratch on the current device.  The first call
// on a device looks it up with cudaGetSymbolAddress (host code cannot use the
// array's name as a device pointer) and caches it.
int noalloc_scratch(void **out)
{
    int dev = 0;
    DTWGB_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevicesNoalloc) {
        set_error("device %d out of range", dev);
        return DTW_EUNSUPPORTED;
    }
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_kmed_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(static k-medoids scratch)");
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return DTW_OK;
}

// Same checks as kmedoids_check, reading the initial medoids into a stack
// buffer instead of a heap one.
int kmedoids_check_noalloc(const float *D, int32_t n, int32_t k, const int32_t *init,
                           int32_t max_iter, const int32_t *out_medoids,
                           const int32_t *out_labels, cudaStream_t st)
{
    if (n < 1) { set_error("n = %d must be >= 1", n); return DTW_EINVAL; }
    if (k < 1 || k > n) { set_error("k = %d must be in [1, n = %d]", k, n); return DTW_EINVAL; }
    if (n > kNoallocMaxN || k > kNoallocMaxK) {
        set_error("n = %d, k = %d exceed the static scratch of kmedoids_fit_noalloc "
                  "(n <= %d, k <= %d); use kmedoids_fit",
                  n, k, kNoallocMaxN, kNoallocMaxK);
        return DTW_EINVAL;
    }
    if (max_iter < 1) { set_error("max_iter = %d must be >= 1", max_iter); return DTW_EINVAL; }
    if (!D || !init || !out_medoids || !out_labels) {
        set_error("NULL pointer argument");
        return DTW_EINVAL;
    }
    int32_t h[kNoallocMaxK];
    cudaError_t e = cudaMemcpyAsync(h, init, sizeof(int32_t) * (size_t)k, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "reading init_medoids");
    for (int32_t c = 0; c < k; ++c) {
        if (h[c] < 0 || h[c] >= n) {
            set_error("init_medoids[%d] = %d is outside [0, %d)", c, h[c], n);
            return DTW_EINVAL;
        }
        for (int32_t d = 0; d < c; ++d)
            if (h[d] == h[c]) {
                set_error("init_medoids[%d] and [%d] are both %d", d, c, h[c]);
                return DTW_EINVAL;
            }
    }
    return DTW_OK;
}

}  // namespace

}  // namespace dtwgb

using namespace dtwgb;

extern "C" int kmedoids_fit(const float *D, int32_t n, int32_t k, const int32_t *init_medoids,
                            int32_t max_iter, int32_t *out_medoids, int32_t *out_labels,
                            double *out_cost, int32_t *out_iters, void *stream)
{
    clear_error();
    cudaStream_t st = (cudaStream_t)stream;
    int rc = kmedoids_check(D, n, k, init_medoids, max_iter, out_medoids, out_labels, st);
    if (rc) return rc;
    void *base = nullptr;
    if ((rc = scratch_alloc(&base, scratch_bytes(n, k), st))) return rc;
    rc = kmedoids_run(D, n, k, init_medoids, max_iter, out_medoids, out_labels, out_cost,
                      out_iters, carve(base, n, k), st);
    const int frc = scratch_free(base, st);
    return rc ? rc : frc;
}

// Every call shares the static scratch and overwrites what it needs (the
// convergence flag is cleared before each sweep, the sums and partials are
// written in full); calls that overlap on the GPU, from several streams or
// threads, race on it.
extern "C" int kmedoids_fit_noalloc(const float *D, int32_t n, int32_t k,
                                    const int32_t *init_medoids, int32_t max_iter,
                                    int32_t *out_medoids, int32_t *out_labels, double *out_cost,
                                    int32_t *out_iters, void *stream)
{
    clear_error();
    cudaStream_t st = (cudaStream_t)stream;
    int rc = kmedoids_check_noalloc(D, n, k, init_medoids, max_iter, out_medoids, out_labels, st);
    if (rc) return rc;
    void *base = nullptr;
    if ((rc = noalloc_scratch(&base))) return rc;
    return kmedoids_run(D, n, k, init_medoids, max_iter, out_medoids, out_labels, out_cost,
                        out_iters, carve(base, n, k), st);
}
