// cluster.cu -- cluster-quality reporting over D (dtwgb_cluster.h).
//
// Silhouette: the members of every cluster are listed in index order once;
// the k cluster sums of every point are compensated float32 column reductions
// down the members' rows (coalesced reads of D, one thread per column, members
// in index order), then s(i) per point in float64; for very large n * k one block per row
// sums the gathered segments instead.  The mean of s(i) is a fixed-order
// reduction, so the score is deterministic.
//
// PAM: per SWAP pass one thread per point finds the nearest and second-nearest
// medoid distances, the points are listed per nearest medoid, and the two
// FastPAM1 terms of every (candidate o, cluster c) are Kahan-compensated
// float32 column reductions down the rows of c's members (D is symmetric) --
// one coalesced read of D per pass; a single-block reduction picks the least
// delta (ties to the smaller o, then i).  BUILD uses fixed-order float64 row
// reductions.
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

// Column reductions over cluster segments (D is symmetric, so the sums over a
// row's members are sums down the members' rows): block (column tile, cluster
// c) walks the members j of c in index order, each thread owning one column o
// and reading D[j][o0 + tid] -- contiguous rows, no gathers.
//   csum[o][c] = sum_{j in C_c} D[j][o]        (Kahan-compensated float32)
__global__ void __launch_bounds__(kSilThreads)
    colsum_segments_kernel(const float *__restrict__ D, int n, int k,
                           const int32_t *__restrict__ cstart, const int32_t *__restrict__ perm,
                           double *__restrict__ csum)
{
    const int o = blockIdx.x * kSilThreads + threadIdx.x, c = blockIdx.y;
    if (o >= n) return;
    float acc = 0.f, comp = 0.f;  // Kahan-compensated float32 (float64 rate is low on GB300)
#pragma unroll 8
    for (int q = cstart[c]; q < cstart[c + 1]; ++q) {
        const float y = __fsub_rn(D[(int64_t)perm[q] * n + o], comp);
        const float t = __fadd_rn(acc, y);
        comp = __fsub_rn(__fsub_rn(t, acc), y);
        acc = t;
    }
    csum[(int64_t)o * k + c] = (double)acc - (double)comp;
}

// s(i) from the cluster sums of row i
__global__ void silhouette_finish_kernel(const double *__restrict__ csum, int n, int k,
                                         const int32_t *__restrict__ labels,
                                         const int32_t *__restrict__ cstart, float *__restrict__ out_s,
                                         double *__restrict__ s64)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double *cs = csum + (int64_t)i * k;
    const int own = labels[i];
    const int m = cstart[own + 1] - cstart[own];
    double s = 0.0;
    if (m > 1) {
        const double a = cs[own] / (double)(m - 1);
        double b = 1.0 / 0.0;
        for (int c = 0; c < k; ++c) {
            const int mc = cstart[c + 1] - cstart[c];
            if (c == own || mc == 0) continue;
            const double v = cs[c] / (double)mc;
            if (v < b) b = v;
        }
        const double mx = a > b ? a : b;
        s = mx > 0.0 ? (b - a) / mx : 0.0;
    }
    s64[i] = s;
    if (out_s) out_s[i] = (float)s;
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

// FastPAM1 terms as column reductions over the members j of cluster c = blockIdx.y
// (in index order):
//   t1[o][c] = sum_j min(0, D[j][o] - d1(j)),  t2[o][c] = sum_j min(D[j][o], d2(j)) - d1(j)
__global__ void __launch_bounds__(kSilThreads)
    pam_colred_kernel(const float *__restrict__ D, int n, int k, const float *__restrict__ d1,
                      const float *__restrict__ d2, const int32_t *__restrict__ cstart,
                      const int32_t *__restrict__ perm, double *__restrict__ t1,
                      double *__restrict__ t2)
{
    const int o = blockIdx.x * kSilThreads + threadIdx.x, c = blockIdx.y;
    if (o >= n) return;
    // float32 terms summed with Kahan compensation (error about 2 eps sum |term|,
    // independent of the cluster size): GB300's float64 rate would bound the pass
    float a = 0.f, ca = 0.f, b = 0.f, cb = 0.f;
#pragma unroll 4
    for (int q = cstart[c]; q < cstart[c + 1]; ++q) {
        const int j = perm[q];
        const float d = D[(int64_t)j * n + o], e1 = d1[j], e2 = d2[j];
        const float ya = fminf(0.f, __fsub_rn(d, e1)) - ca;
        const float ta = __fadd_rn(a, ya);
        ca = __fsub_rn(__fsub_rn(ta, a), ya);
        a = ta;
        const float yb = __fsub_rn(__fsub_rn(fminf(d, e2), e1), cb);
        const float tb = __fadd_rn(b, yb);
        cb = __fsub_rn(__fsub_rn(tb, b), yb);
        b = tb;
    }
    t1[(int64_t)o * k + c] = (double)a - (double)ca;
    t2[(int64_t)o * k + c] = (double)b - (double)cb;
}

// delta[o][i] = sum_c t1[o][c] + t2[o][i] - t1[o][i]; +inf for medoids
__global__ void pam_delta_finish_kernel(const double *__restrict__ t1, const double *__restrict__ t2,
                                        int n, const int32_t *__restrict__ M, int k,
                                        double *__restrict__ delta)
{
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= n) return;
    const int64_t base = (int64_t)o * k;
    if (is_medoid(M, k, o)) {
        for (int c = 0; c < k; ++c) delta[base + c] = 1.0 / 0.0;
        return;
    }
    double S = 0.0;
    for (int c = 0; c < k; ++c) S += t1[base + c];
    for (int c = 0; c < k; ++c) delta[base + c] = S + t2[base + c] - t1[base + c];
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
    const bool by_columns = (int64_t)n * k <= (64ll << 20);  // cluster sums as column reductions
    const size_t bytes = sizeof(int32_t) * ((size_t)k + 1 + n) +
                         sizeof(double) * ((size_t)n + kSilParts + (by_columns ? (size_t)n * k : 0)) + 64;
    int rc = scratch_alloc(&buf, bytes, st);
    if (rc) return rc;
    double *s64 = (double *)buf;
    double *part = s64 + n;
    double *csum = part + kSilParts;
    int32_t *cstart = (int32_t *)(csum + (by_columns ? (size_t)n * k : 0));
    int32_t *perm = cstart + k + 1;
    cudaError_t e = cudaMemcpyAsync(cstart, start.data(), sizeof(int32_t) * (k + 1),
                                    cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        sil_members_kernel<<<k, 256, 0, st>>>(labels, n, cstart, perm);
        if (by_columns) {
            colsum_segments_kernel<<<dim3((n + kSilThreads - 1) / kSilThreads, k), kSilThreads, 0, st>>>(
                D, n, k, cstart, perm, csum);
            silhouette_finish_kernel<<<(n + 255) / 256, 256, 0, st>>>(csum, n, k, labels, cstart,
                                                                     out_s, s64);
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
    const size_t bytes = sizeof(double) * (3 * (size_t)n * k + n + kSilParts) + sizeof(PamBest) +
                         sizeof(float) * 2 * (size_t)n + sizeof(int32_t) * (3 * (size_t)n + 2 * k + 2) + 256;
    void *buf = nullptr;
    int rc = scratch_alloc(&buf, bytes, st);
    if (rc) return rc;
    double *delta = (double *)buf;
    double *t1 = delta + (size_t)n * k;
    double *t2 = t1 + (size_t)n * k;
    double *val = t2 + (size_t)n * k;
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
        pam_colred_kernel<<<dim3((n + kSilThreads - 1) / kSilThreads, k), kSilThreads, 0, st>>>(
            D, n, k, d1, d2, cstart, perm, t1, t2);
        pam_delta_finish_kernel<<<nb, 256, 0, st>>>(t1, t2, n, M, k, delta);
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
