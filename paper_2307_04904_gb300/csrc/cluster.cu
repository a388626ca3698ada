// cluster.cu -- cluster-quality reporting over D (dtwgb_cluster.h).
//
// Silhouette: the members of every cluster are listed in index order once;
// one block per row i then sums D[i][j] over each cluster's member segment
// (float64 partials per thread, warp shuffles, then the 8 warp sums in order)
// and turns the k sums into s(i).  The mean of s(i) is a fixed-order
// reduction, so the score is deterministic.
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
