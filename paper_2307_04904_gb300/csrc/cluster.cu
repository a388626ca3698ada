// cluster.cu -- cluster-quality reporting over D (dtwgb_cluster.h).
//
// Silhouette: the members of every cluster are listed in index order once;
// one block per row i then sums D[i][j] over each cluster's member segment
// (float64 partials per thread, warp shuffles, then the 8 warp sums in order)
// and turns the k sums into s(i).  The mean of s(i) is a fixed-order
// reduction, so the score is deterministic.
//
// PAM: per SWAP pass one thread per point finds the nearest and second-nearest
// medoid distances, the points are listed per nearest medoid, and one block
// per candidate o sums, cluster segment by cluster segment, the two FastPAM1
// terms in float64 -- every delta(o, i) from one read of row o; a single-block
// reduction picks the least delta (ties to the smaller o, then i).  BUILD uses
// the same row reduction with min(D[o][j], d1(j)).
#include <vector>

#include "../../include/dtwgb_cluster.h"
#include "common.cuh"

namespace dtwgb {
namespace {

constexpr int kSilThreads = 256;
constexpr int kSilMaxK = 4096;
constexpr int kSilParts = 64;

// perm[cstart[c] + r] = the r-th member of cluster c in index order; one block per cluster
__global__ void sil_members_kernel(const int32_t *__restrict__ labels, int n,
                                   const int32_t *__restrict__ cstart, int32_t *__restrict__ perm)
{
    __shared__ int scan[256];
    const int c = blockIdx.x, tid = threadIdx.x;
    int base = cstart[c];
    for (int j0 = 0; j0 < n; j0 += 256) {
        const int j = j0 + tid;
        const int f = (j < n && labels[j] == c) ? 1 : 0;
        scan[tid] = f;
        __syncthreads();
        for (int o = 1; o < 256; o <<= 1) {
            const int v = tid >= o ? scan[tid - o] : 0;
            __syncthreads();
            scan[tid] += v;
            __syncthreads();
        }
        if (f) perm[base + scan[tid] - 1] = j;
        const int total = scan[255];
        __syncthreads();
        base += total;
    }
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

// s(i) for row i = blockIdx.x
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

// val[o] = sum_j min(D[o][j], d1[j]) (d1 == NULL: the row sum); +inf for the
// first `k` medoids M
__global__ void __launch_bounds__(kSilThreads)
    pam_build_kernel(const float *__restrict__ D, int n, const float *__restrict__ d1,
                     const int32_t *__restrict__ M, int k, double *__restrict__ val)
{
    __shared__ double warp_part[kSilThreads / 32];
    const int o = blockIdx.x;
    if (is_medoid(M, k, o)) {
        if (threadIdx.x == 0) val[o] = 1.0 / 0.0;
        return;
    }
    const float *row = D + (int64_t)o * n;
    double acc = 0.0;
    for (int j = threadIdx.x; j < n; j += kSilThreads)
        acc += d1 ? (double)fminf(row[j], d1[j]) : (double)row[j];
    const double t = block_sum(acc, warp_part);
    if (threadIdx.x == 0) val[o] = t;
}

// one block: the least val (ties to the smaller index) -> M[slot]
__global__ void pam_argmin_row_kernel(const double *__restrict__ val, int n, int32_t *__restrict__ M,
                                      int slot)
{
    __shared__ double bv[1024];
    __shared__ int bi[1024];
    double v = 1.0 / 0.0;
    int idx = 0x7fffffff;
    for (int o = threadIdx.x; o < n; o += blockDim.x)
        if (val[o] < v) {
            v = val[o];
            idx = o;
        }
    bv[threadIdx.x] = v;
    bi[threadIdx.x] = idx;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            const double w = bv[threadIdx.x + s];
            const int wi = bi[threadIdx.x + s];
            if (w < bv[threadIdx.x] || (w == bv[threadIdx.x] && wi < bi[threadIdx.x])) {
                bv[threadIdx.x] = w;
                bi[threadIdx.x] = wi;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) M[slot] = bi[0];
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
// counts per nearest medoid
__global__ void pam_nearest_kernel(const float *__restrict__ D, int n, const int32_t *__restrict__ M,
                                   int k, float *__restrict__ d1, float *__restrict__ d2,
                                   int32_t *__restrict__ n1, int32_t *__restrict__ cnt)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    float b1 = 1.0f / 0.0f, b2 = 1.0f / 0.0f;
    int c1 = 0;
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
    atomicAdd(cnt + c1, 1);
}

__global__ void pam_prefix_kernel(const int32_t *__restrict__ cnt, int k, int32_t *__restrict__ cstart)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int run = 0;
    for (int c = 0; c < k; ++c) {
        cstart[c] = run;
        run += cnt[c];
    }
    cstart[k] = run;
}

__device__ __forceinline__ void block_sum2(double &a, double &b, double *wa, double *wb)
{
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        wa[w] = a;
        wb[w] = b;
    }
    __syncthreads();
    double ta = 0.0, tb = 0.0;
    for (int q = 0; q < kSilThreads / 32; ++q) {
        ta += wa[q];
        tb += wb[q];
    }
    __syncthreads();
    a = ta;
    b = tb;
}

// delta[o][i] for candidate o = blockIdx.x (+inf for medoids)
__global__ void __launch_bounds__(kSilThreads)
    pam_delta_kernel(const float *__restrict__ D, int n, const int32_t *__restrict__ M, int k,
                     const float *__restrict__ d1, const float *__restrict__ d2,
                     const int32_t *__restrict__ cstart, const int32_t *__restrict__ perm,
                     double *__restrict__ delta)
{
    __shared__ double wa[kSilThreads / 32], wb[kSilThreads / 32];
    __shared__ double t1[kPamMaxK], t2[kPamMaxK];
    const int o = blockIdx.x;
    if (is_medoid(M, k, o)) {
        for (int c = threadIdx.x; c < k; c += kSilThreads) delta[(int64_t)o * k + c] = 1.0 / 0.0;
        return;
    }
    const float *row = D + (int64_t)o * n;
    for (int c = 0; c < k; ++c) {
        double a = 0.0, b = 0.0;
        for (int q = cstart[c] + threadIdx.x; q < cstart[c + 1]; q += kSilThreads) {
            const int j = perm[q];
            const double d = (double)row[j], e1 = (double)d1[j], e2 = (double)d2[j];
            a += fmin(0.0, d - e1);
            b += fmin(d, e2) - e1;
        }
        block_sum2(a, b, wa, wb);
        if (threadIdx.x == 0) {
            t1[c] = a;
            t2[c] = b;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double S = 0.0;
        for (int c = 0; c < k; ++c) S += t1[c];
        for (int c = 0; c < k; ++c) delta[(int64_t)o * k + c] = S + t2[c] - t1[c];
    }
}

struct PamBest {
    double delta;
    int64_t idx;  // o * k + i
};

// one block: the least delta, ties to the smaller flat index o * k + i
__global__ void pam_argmin_delta_kernel(const double *__restrict__ delta, int64_t total,
                                        PamBest *__restrict__ out)
{
    __shared__ double bv[1024];
    __shared__ int64_t bi[1024];
    double v = 1.0 / 0.0;
    int64_t idx = INT64_MAX;
    for (int64_t t = threadIdx.x; t < total; t += blockDim.x)
        if (delta[t] < v) {
            v = delta[t];
            idx = t;
        }
    bv[threadIdx.x] = v;
    bi[threadIdx.x] = idx;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            const double w = bv[threadIdx.x + s];
            const int64_t wi = bi[threadIdx.x + s];
            if (w < bv[threadIdx.x] || (w == bv[threadIdx.x] && wi < bi[threadIdx.x])) {
                bv[threadIdx.x] = w;
                bi[threadIdx.x] = wi;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out->delta = bv[0];
        out->idx = bi[0];
    }
}

__global__ void pam_apply_kernel(int32_t *__restrict__ M, const PamBest *__restrict__ best, int k)
{
    if (threadIdx.x == 0 && blockIdx.x == 0 && best->delta < 0.0)
        M[best->idx % k] = (int32_t)(best->idx / k);
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
    std::vector<int32_t> cnt((size_t)k, 0), start((size_t)k + 1, 0);
    for (int j = 0; j < n; ++j) {
        if (hl[j] < 0 || hl[j] >= k) {
            set_error("labels[%d] = %d is outside [0, %d)", j, hl[j], k);
            return DTW_EINVAL;
        }
        ++cnt[hl[j]];
    }
    int nonempty = 0;
    for (int c = 0; c < k; ++c) {
        start[c + 1] = start[c] + cnt[c];
        nonempty += cnt[c] > 0;
    }
    if (nonempty < 2) {
        set_error("the silhouette needs at least two non-empty clusters (%d)", nonempty);
        return DTW_EINVAL;
    }
    void *buf = nullptr;
    const size_t bytes = sizeof(int32_t) * ((size_t)k + 1 + n) + sizeof(double) * ((size_t)n + kSilParts) + 64;
    int rc = scratch_alloc(&buf, bytes, st);
    if (rc) return rc;
    double *s64 = (double *)buf;
    double *part = s64 + n;
    int32_t *cstart = (int32_t *)(part + kSilParts);
    int32_t *perm = cstart + k + 1;
    cudaError_t e = cudaMemcpyAsync(cstart, start.data(), sizeof(int32_t) * (k + 1),
                                    cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        sil_members_kernel<<<k, 256, 0, st>>>(labels, n, cstart, perm);
        silhouette_kernel<<<n, kSilThreads, sizeof(double) * k, st>>>(D, n, labels, k, cstart, perm,
                                                                      out_s, s64);
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
    const size_t bytes = sizeof(double) * ((size_t)n * k + n + kSilParts) + sizeof(PamBest) +
                         sizeof(float) * 2 * (size_t)n + sizeof(int32_t) * (3 * (size_t)n + 2 * k + 2) + 256;
    void *buf = nullptr;
    int rc = scratch_alloc(&buf, bytes, st);
    if (rc) return rc;
    double *delta = (double *)buf;
    double *val = delta + (size_t)n * k;
    double *part = val + n;
    PamBest *best = (PamBest *)(part + kSilParts);
    float *d1 = (float *)(best + 1);
    float *d2 = d1 + n;
    int32_t *n1 = (int32_t *)(d2 + n);
    int32_t *perm = n1 + n;
    int32_t *cnt = perm + n;
    int32_t *cstart = cnt + k;
    int32_t *M = out_medoids;
    const unsigned nb = (unsigned)((n + 255) / 256);
    cudaError_t e = cudaSuccess;
    auto fail = [&](cudaError_t err, const char *what) {
        scratch_free(buf, st);
        return cuda_fail(err, what);
    };
    if (init_medoids) {
        e = cudaMemcpyAsync(M, init_medoids, sizeof(int32_t) * k, cudaMemcpyDeviceToDevice, st);
    } else {
        for (int s = 0; s < k; ++s) {  // BUILD
            pam_build_kernel<<<n, kSilThreads, 0, st>>>(D, n, s ? d1 : nullptr, M, s, val);
            pam_argmin_row_kernel<<<1, 1024, 0, st>>>(val, n, M, s);
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
        pam_prefix_kernel<<<1, 32, 0, st>>>(cnt, k, cstart);
        sil_members_kernel<<<k, 256, 0, st>>>(n1, n, cstart, perm);
        pam_delta_kernel<<<n, kSilThreads, 0, st>>>(D, n, M, k, d1, d2, cstart, perm, delta);
        pam_argmin_delta_kernel<<<1, 1024, 0, st>>>(delta, (int64_t)n * k, best);
        pam_apply_kernel<<<1, 32, 0, st>>>(M, best, k);
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
