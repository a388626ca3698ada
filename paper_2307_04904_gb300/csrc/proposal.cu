// proposal.cu -- k-means++ seeding in embedding space and lazy k-medoids
// over exact DTW (dtwgb_proposal.h).
//
// kmedoids_lazy_fit runs the alternate k-medoids of kmedoids_fit, but instead
// of the full matrix D it asks the DTW kernels for exactly the pairs a sweep
// needs, as explicit pair lists over one staged copy of the set:
//   assign  (M_c, j) for every medoid c and point j        -> k*n pairs
//   update  (candidate, member) within every cluster       -> sum ncand_c*|C_c|
// Candidates of a cluster are its current medoid and the members nearest to
// the cluster's embedding centroid (or every member).  Cluster member lists
// are built in index order, every sum is taken in a fixed order, so a fit is
// deterministic.
#include <algorithm>
#include <vector>

#include "../../include/dtwgb_proposal.h"
#include "band_kernels.cuh"

namespace dtwgb {
namespace {

// splitmix64 (Steele, Lea & Flood 2014): state += golden gamma, then mix.
uint64_t splitmix64_next(uint64_t &state)
{
    state += 0x9E3779B97F4A7C15ull;
    uint64_t z = state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// ------------------------------------------------------------ k-means++

// D2[j] = min(D2[j], ||e_j - e_c||^2) for the newest centre c = centers[i]
// (the squared differences added in dimension order; rows read as float4 when
// they are 16-byte aligned, which changes no operation)
__global__ void kpp_update_kernel(const float *__restrict__ emb, int n, int dim,
                                  const int32_t *__restrict__ centers, int i, double *__restrict__ D2,
                                  bool vec4)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int c = centers[i];
    float s = 0.f;
    if (vec4) {
        const float4 *ej = reinterpret_cast<const float4 *>(emb + (int64_t)j * dim);
        const float4 *ec = reinterpret_cast<const float4 *>(emb + (int64_t)c * dim);
        for (int d = 0; d < dim / 4; ++d) {
            const float4 a = __ldg(ej + d), b = __ldg(ec + d);
            float df = a.x - b.x;
            s = fmaf(df, df, s);
            df = a.y - b.y;
            s = fmaf(df, df, s);
            df = a.z - b.z;
            s = fmaf(df, df, s);
            df = a.w - b.w;
            s = fmaf(df, df, s);
        }
    } else {
        for (int d = 0; d < dim; ++d) {
            const float df = emb[(int64_t)j * dim + d] - emb[(int64_t)c * dim + d];
            s = fmaf(df, df, s);
        }
    }
    D2[j] = (i == 0) ? (double)s : fmin(D2[j], (double)s);
}

// One block of kPickThreads threads picks the smallest j whose running sum of
// D2 exceeds u * total, with D2[j] > 0 (k-means++ draws j with probability
// D2[j] / total).  Thread t sums chunk t (ceil(n / kPickThreads) values, in
// index order); an inclusive scan of the chunk sums (warp shuffles, then over
// the warp totals) gives every chunk its prefix; the first chunk with values
// whose prefix passes u * total walks its own values from the prefix before
// it.  Where rounding leaves the threshold unreached, the last positive value
// of the last chunk with values is taken.  If every D2 is zero, the smallest
// index not chosen yet.
constexpr int kPickThreads = 1024;

__global__ void __launch_bounds__(kPickThreads) kpp_pick_kernel(const double *__restrict__ D2, int n,
                                                                double u,
                                                                int32_t *__restrict__ centers, int i)
{
    __shared__ double wsum[kPickThreads / 32];
    __shared__ double total_sh;
    __shared__ int qsel, qlast;
    const unsigned FULL = 0xffffffffu;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int chunk = (n + kPickThreads - 1) / kPickThreads;
    const int lo = min(n, tid * chunk), hi = min(n, lo + chunk);
    double s = 0.0;
    for (int j = lo; j < hi; ++j) s += __ldg(D2 + j);
    if (tid == 0) {
        qsel = kPickThreads;
        qlast = -1;
    }
    double x = s;  // inclusive scan within the warp
    for (int d = 1; d < 32; d <<= 1) {
        const double y = __shfl_up_sync(FULL, x, d);
        if (lane >= d) x += y;
    }
    double xprev = __shfl_up_sync(FULL, x, 1);
    if (lane == 0) xprev = 0.0;
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    if (wid == 0) {  // inclusive scan of the warp totals
        double w = wsum[lane];
        for (int d = 1; d < 32; d <<= 1) {
            const double y = __shfl_up_sync(FULL, w, d);
            if (lane >= d) w += y;
        }
        __syncwarp();
        wsum[lane] = w;
    }
    __syncthreads();
    const double base = wid ? wsum[wid - 1] : 0.0;
    const double incl = base + x, excl = base + xprev;
    if (tid == kPickThreads - 1) total_sh = incl;
    __syncthreads();
    const double total = total_sh;
    const double thr = u * total;
    if (total > 0.0 && s > 0.0) {
        if (incl > thr) atomicMin(&qsel, tid);
        atomicMax(&qlast, tid);
    }
    __syncthreads();
    if (total > 0.0) {
        if (tid == qsel) {
            double run = excl;
            int pick = -1;
            for (int j = lo; j < hi; ++j) {
                run += D2[j];
                if (run > thr && D2[j] > 0.0) {
                    pick = j;
                    break;
                }
            }
            if (pick < 0)  // rounding left the threshold unreached in this chunk
                for (int j = hi - 1; j >= lo; --j)
                    if (D2[j] > 0.0) { pick = j; break; }
            centers[i] = pick;
        } else if (qsel == kPickThreads && tid == qlast) {
            int pick = lo;
            for (int j = hi - 1; j >= lo; --j)
                if (D2[j] > 0.0) { pick = j; break; }
            centers[i] = pick;
        }
    } else if (tid == 0) {
        int pick = -1;
        for (int j = 0; j < n && pick < 0; ++j) {
            bool used = false;
            for (int q = 0; q < i; ++q) used |= (centers[q] == j);
            if (!used) pick = j;
        }
        centers[i] = pick;
    }
}

// ------------------------------------------------- k-means in embedding space

__global__ void set_first_kernel(int32_t *centers, int32_t first) { centers[0] = first; }

__global__ void gather_rows_kernel(const float *__restrict__ emb, int dim,
                                   const int32_t *__restrict__ idx, int k, float *__restrict__ C)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < k * dim) C[t] = emb[(int64_t)idx[t / dim] * dim + t % dim];
}

// label_j = argmin_c ||e_j - C_c||^2 (ties to the smallest c), dist_j that minimum;
// sets *changed when a label differs from the one it replaces.  Does nothing
// once *stop is set (Lloyd's iterations converged).  With dynamic shared
// memory of k * dim floats the centroids are read from there.
__global__ void km_assign_kernel(const float *__restrict__ emb, int n, int dim,
                                 const float *__restrict__ Cg, int k, int32_t *__restrict__ lab,
                                 float *__restrict__ dist, int32_t *__restrict__ changed,
                                 const int32_t *__restrict__ stop, int smem_c, bool vec4)
{
    extern __shared__ float4 Cs4[];  // k x dim centroids when smem_c (16-byte aligned)
    float *Cs = reinterpret_cast<float *>(Cs4);
    if (stop && *stop) return;
    if (smem_c) {
        for (int i = threadIdx.x; i < k * dim; i += blockDim.x) Cs[i] = Cg[i];
        __syncthreads();
    }
    const float *C = smem_c ? Cs : Cg;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const float *e = emb + (int64_t)j * dim;
    float bd = 0.f;
    int best = 0;
    if (k <= 16 && vec4) {
        // as below, four dimensions per load (each distance still summed in dimension order)
        const float4 *e4 = reinterpret_cast<const float4 *>(e);
        const float4 *C4 = reinterpret_cast<const float4 *>(C);
        const int dim4 = dim / 4;
        float acc[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) acc[c] = 0.f;
        for (int d = 0; d < dim4; ++d) {
            const float4 ed = __ldg(e4 + d);
#pragma unroll
            for (int c = 0; c < 16; ++c)
                if (c < k) {
                    const float4 cd = C4[c * dim4 + d];
                    float df = ed.x - cd.x;
                    acc[c] = fmaf(df, df, acc[c]);
                    df = ed.y - cd.y;
                    acc[c] = fmaf(df, df, acc[c]);
                    df = ed.z - cd.z;
                    acc[c] = fmaf(df, df, acc[c]);
                    df = ed.w - cd.w;
                    acc[c] = fmaf(df, df, acc[c]);
                }
        }
#pragma unroll
        for (int c = 0; c < 16; ++c)
            if (c < k && (c == 0 || acc[c] < bd)) {
                bd = acc[c];
                best = c;
            }
    } else if (k <= 16) {  // each e[d] read once, the k distances accumulated side by side
        float acc[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) acc[c] = 0.f;
        for (int d = 0; d < dim; ++d) {
            const float ed = e[d];
#pragma unroll
            for (int c = 0; c < 16; ++c)
                if (c < k) {
                    const float df = ed - C[c * dim + d];
                    acc[c] = fmaf(df, df, acc[c]);
                }
        }
#pragma unroll
        for (int c = 0; c < 16; ++c)
            if (c < k && (c == 0 || acc[c] < bd)) {
                bd = acc[c];
                best = c;
            }
    } else {
        for (int c = 0; c < k; ++c) {
            float s = 0.f;
            for (int d = 0; d < dim; ++d) {
                const float df = e[d] - C[c * dim + d];
                s = fmaf(df, df, s);
            }
            if (c == 0 || s < bd) {
                bd = s;
                best = c;
            }
        }
    }
    if (lab[j] != best) atomicOr(changed, 1);
    lab[j] = best;
    dist[j] = bd;
}

// Centroid sums without member lists: block q sums the points of chunk q
// into per-cluster accumulators in shared memory (thread d owns dimension d and
// walks the chunk's points in order), partials [q][c][d] and counts [q][c].
constexpr int kKmChunk = 64;
constexpr int kKmSmemFloats = 12288;  // k * dim bound of the shared accumulators (48 KB)
constexpr int kAssignThreads = 128;   // threads per block of km_assign_kernel
// Chunk partials of the centroid sums.  Returns at once when the assignment of
// this iteration changed no label (*changed == 0: converged, or skipped after
// convergence).
__global__ void km_partial_kernel(const float *__restrict__ emb, int n, int dim,
                                  const int32_t *__restrict__ lab, int k, float *__restrict__ psum,
                                  int32_t *__restrict__ pcnt, const int32_t *__restrict__ changed)
{
    extern __shared__ float acc[];  // [k][dim], then int counts [k]
    if (*changed == 0) return;  // the same for every thread of the launch
    int *cnt = (int *)(acc + k * dim);
    for (int i = threadIdx.x; i < k * dim; i += blockDim.x) acc[i] = 0.f;
    for (int i = threadIdx.x; i < k; i += blockDim.x) cnt[i] = 0;
    __syncthreads();
    const int j0 = blockIdx.x * kKmChunk, j1 = min(n, j0 + kKmChunk);
    for (int d = threadIdx.x; d < dim; d += blockDim.x) {
        int j = j0;
        for (; j + 8 <= j1; j += 8) {  // 8 rows' loads in flight, then the sums in row order
            float v[8];
            int L[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                L[u] = lab[j + u];
                v[u] = emb[(int64_t)(j + u) * dim + d];
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) acc[L[u] * dim + d] += v[u];
        }
        for (; j < j1; ++j) acc[lab[j] * dim + d] += emb[(int64_t)j * dim + d];
    }
    if (threadIdx.x == 0)
        for (int j = j0; j < j1; ++j) cnt[lab[j]] += 1;
    __syncthreads();
    for (int i = threadIdx.x; i < k * dim; i += blockDim.x) psum[(int64_t)blockIdx.x * k * dim + i] = acc[i];
    for (int i = threadIdx.x; i < k; i += blockDim.x) pcnt[(int64_t)blockIdx.x * k + i] = cnt[i];
}

// C[c][d] = (sum over chunks, in order) / count; an empty cluster keeps its centroid
// C = per-cluster mean from the chunk partials: 32 outputs per block, warp w
// adds chunks w, w + kRedWarps, ... in order (four loads in flight), then the
// warp sums are added in warp order -- a fixed order, so C is deterministic.
// The iteration's flags: `changed` (set by this iteration's assignment, only
// read here), `next` (the next iteration's, cleared here by block 0) and
// `stop` (raised by block 0 when no label changed; the next assignments then
// return at once).  No block writes a word another block of the launch reads.
constexpr int kRedWarps = 16;

__global__ void __launch_bounds__(32 * kRedWarps) km_reduce_kernel(
    const float *__restrict__ psum, const int32_t *__restrict__ pcnt, int nchunks, int k, int dim,
    float *__restrict__ C, const int32_t *__restrict__ changed, int32_t *__restrict__ next,
    int32_t *__restrict__ stop)
{
    __shared__ float sh[kRedWarps][33];
    __shared__ int shm[kRedWarps][33];
    const bool first = blockIdx.x == 0 && threadIdx.x == 0;
    if (first) *next = 0;
    if (*changed == 0) {  // the same for every thread of the launch
        if (first) *stop = 1;
        return;
    }
    const int o = threadIdx.x & 31, w = threadIdx.x >> 5, i = blockIdx.x * 32 + o;
    const int KD = k * dim;
    float s = 0.f;
    int m = 0;
    if (i < KD) {
        const int c = i / dim;
        int q = w;
        for (; q + 3 * kRedWarps < nchunks; q += 4 * kRedWarps) {
            const float a0 = psum[(int64_t)q * KD + i];
            const float a1 = psum[(int64_t)(q + kRedWarps) * KD + i];
            const float a2 = psum[(int64_t)(q + 2 * kRedWarps) * KD + i];
            const float a3 = psum[(int64_t)(q + 3 * kRedWarps) * KD + i];
            const int b0 = pcnt[(int64_t)q * k + c], b1 = pcnt[(int64_t)(q + kRedWarps) * k + c];
            const int b2 = pcnt[(int64_t)(q + 2 * kRedWarps) * k + c];
            const int b3 = pcnt[(int64_t)(q + 3 * kRedWarps) * k + c];
            s = (((s + a0) + a1) + a2) + a3;
            m += b0 + b1 + b2 + b3;
        }
        for (; q < nchunks; q += kRedWarps) {
            s += psum[(int64_t)q * KD + i];
            m += pcnt[(int64_t)q * k + c];
        }
    }
    sh[w][o] = s;
    shm[w][o] = m;
    __syncthreads();
    if (w == 0 && i < KD) {
        float t = 0.f;
        int mm = 0;
        for (int p = 0; p < kRedWarps; ++p) {
            t += sh[p][o];
            mm += shm[p][o];
        }
        if (mm > 0) C[i] = t / (float)mm;
    }
}

// Lloyd's iterations stop at the first assignment that changes no label
__global__ void prefix_kernel(const int32_t *__restrict__ cnt, int k, int32_t *__restrict__ cstart)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int run = 0;
    for (int c = 0; c < k; ++c) {
        cstart[c] = run;
        run += cnt[c];
    }
    cstart[k] = run;
}

// one block: inertia = sum of the partials in order; a restart whose inertia is
// strictly below the best so far replaces it (its centroids are copied)
__global__ void keep_best_kernel(const double *__restrict__ part, int nparts,
                                 const float *__restrict__ C, int kd, double *__restrict__ best,
                                 float *__restrict__ bestC, int first)
{
    __shared__ int take;
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int q = 0; q < nparts; ++q) tot += part[q];
        take = first || tot < *best;
        if (take) *best = tot;
    }
    __syncthreads();
    if (take)
        for (int t = threadIdx.x; t < kd; t += blockDim.x) bestC[t] = C[t];
}

// proposal of cluster c: its member nearest to the centroid (dist, ties to the
// smaller index); one block per cluster; empty clusters are filled afterwards
__global__ void nearest_member_kernel(const float *__restrict__ dist, const int32_t *__restrict__ members,
                                      const int32_t *__restrict__ cstart, const int32_t *__restrict__ cnt,
                                      int32_t *__restrict__ out)
{
    __shared__ float sd[256];
    __shared__ int si[256];
    const int c = blockIdx.x, tid = threadIdx.x, m = cnt[c];
    float bd = 3.4e38f;
    int bi = 0x7fffffff;
    for (int q = tid; q < m; q += 256) {
        const int j = members[cstart[c] + q];
        if (dist[j] < bd || (dist[j] == bd && j < bi)) {
            bd = dist[j];
            bi = j;
        }
    }
    sd[tid] = bd;
    si[tid] = bi;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (tid < o && (sd[tid + o] < sd[tid] || (sd[tid + o] == sd[tid] && si[tid + o] < si[tid]))) {
            sd[tid] = sd[tid + o];
            si[tid] = si[tid + o];
        }
        __syncthreads();
    }
    if (tid == 0) out[c] = m > 0 ? si[0] : -1;
}

// an empty cluster takes the point nearest to its centroid that no cluster
// has taken (ties to the smaller index); clusters in order, one thread
__global__ void fill_empty_kernel(const float *__restrict__ emb, int n, int dim,
                                  const float *__restrict__ C, int k, int32_t *__restrict__ out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int c = 0; c < k; ++c) {
        if (out[c] >= 0) continue;
        float bd = 3.4e38f;
        int bi = -1;
        for (int j = 0; j < n; ++j) {
            bool used = false;
            for (int q = 0; q < k; ++q) used |= (out[q] == j);
            if (used) continue;
            float s = 0.f;
            for (int d = 0; d < dim; ++d) {
                const float df = emb[(int64_t)j * dim + d] - C[c * dim + d];
                s = fmaf(df, df, s);
            }
            if (bi < 0 || s < bd) {
                bd = s;
                bi = j;
            }
        }
        out[c] = bi;
    }
}

// ---------------------------------------------------------- lazy k-medoids

__global__ void gen_assign_pairs_kernel(const int32_t *__restrict__ M, int k, int n,
                                        int32_t *__restrict__ pa, int32_t *__restrict__ pb)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)k * n) return;
    pa[t] = M[t / n];
    pb[t] = (int32_t)(t % n);
}

// label_j = argmin_c R[c][j], ties to the smallest c; a medoid labels itself
__global__ void lazy_assign_kernel(const float *__restrict__ R, int k, int n,
                                   const int32_t *__restrict__ M, int32_t *__restrict__ labels,
                                   float *__restrict__ dmin)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    int best = 0, own = -1;
    float bd = R[j];
    if (M[0] == j) own = 0;
    for (int c = 1; c < k; ++c) {
        if (M[c] == j) own = c;
        const float d = R[(int64_t)c * n + j];
        if (d < bd) {
            bd = d;
            best = c;
        }
    }
    const int lab = own >= 0 ? own : best;
    labels[j] = lab;
    dmin[j] = R[(int64_t)lab * n + j];
}

__global__ void count_kernel(const int32_t *__restrict__ labels, int n, int32_t *__restrict__ cnt)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) atomicAdd(cnt + labels[j], 1);
}

// members of cluster c in index order at members[cstart[c] ...]; one block per cluster
__global__ void members_kernel(const int32_t *__restrict__ labels, int n,
                               const int32_t *__restrict__ cstart, int32_t *__restrict__ members)
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
        if (f) members[base + scan[tid] - 1] = j;
        const int total = scan[255];
        __syncthreads();
        base += total;
    }
}

// centroid of the cluster's embeddings: one block of 256 threads per cluster;
// warp w sums members w, w+8, ... per dimension, the 8 warp sums are added in
// warp order.  An empty cluster keeps its centroid.
constexpr int kCentWarps = 8;
__global__ void centroid_kernel(const float *__restrict__ emb, int dim,
                                const int32_t *__restrict__ members, const int32_t *__restrict__ cstart,
                                const int32_t *__restrict__ cnt, float *__restrict__ cent)
{
    extern __shared__ float wsum[];  // [kCentWarps][dim]
    const int c = blockIdx.x, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int m = cnt[c];
    const int32_t *mem = members + cstart[c];
    for (int d = lane; d < dim; d += 32) {
        float s = 0.f;
        for (int q = w; q < m; q += kCentWarps) s += emb[(int64_t)mem[q] * dim + d];
        wsum[w * dim + d] = s;
    }
    __syncthreads();
    for (int d = threadIdx.x; d < dim; d += blockDim.x) {
        if (m == 0) continue;
        float s = 0.f;
        for (int q = 0; q < kCentWarps; ++q) s += wsum[q * dim + d];
        cent[c * dim + d] = s / (float)m;
    }
}

// cdist[q] = squared embedding distance of member q of the lists (point members[q])
// to its cluster's centroid; one thread per member, dimensions in order
__global__ void member_dist_kernel(const float *__restrict__ emb, int dim,
                                   const int32_t *__restrict__ members,
                                   const int32_t *__restrict__ labels, int n,
                                   const float *__restrict__ cent, float *__restrict__ cdist)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const int j = members[q], c = labels[j];
    float s = 0.f;
    for (int d = 0; d < dim; ++d) {
        const float df = emb[(int64_t)j * dim + d] - cent[c * dim + d];
        s = fmaf(df, df, s);
    }
    cdist[q] = s;
}

// base candidates of cluster c at cand[cbase[c] ...]: the current medoid, then
// the nbase-1 other members nearest to the centroid (ties to the smaller
// index), picked in increasing (distance, index) order from the distances of
// member_dist_kernel.  One block per cluster.
__global__ void candidates_kernel(const float *__restrict__ cdist, const int32_t *__restrict__ members,
                                  const int32_t *__restrict__ cstart, const int32_t *__restrict__ cnt,
                                  const int32_t *__restrict__ M, const int32_t *__restrict__ cbase,
                                  const int32_t *__restrict__ nbase, int32_t *__restrict__ cand)
{
    __shared__ float sd[256];
    __shared__ int si[256];
    const int c = blockIdx.x, tid = threadIdx.x;
    const int m = cnt[c], medoid = M[c];
    if (tid == 0) cand[cbase[c]] = medoid;
    float last_d = -1.f;
    int last_i = -1;
    for (int q = 1; q < nbase[c]; ++q) {
        float bd = 3.4e38f;
        int bi = 0x7fffffff;
        for (int r = tid; r < m; r += 256) {
            const int j = members[cstart[c] + r];
            if (j == medoid) continue;
            const float s = cdist[cstart[c] + r];
            const bool after = s > last_d || (s == last_d && j > last_i);
            if (after && (s < bd || (s == bd && j < bi))) {
                bd = s;
                bi = j;
            }
        }
        sd[tid] = bd;
        si[tid] = bi;
        __syncthreads();
        for (int o = 128; o > 0; o >>= 1) {
            if (tid < o && (sd[tid + o] < sd[tid] || (sd[tid + o] == sd[tid] && si[tid + o] < si[tid]))) {
                sd[tid] = sd[tid + o];
                si[tid] = si[tid + o];
            }
            __syncthreads();
        }
        last_d = sd[0];
        last_i = si[0];
        if (tid == 0) cand[cbase[c] + q] = last_i;
        __syncthreads();
    }
}

// Screening: member i of cluster c is paired with the s_c sampled members
// mem[floor(q * m_c / s_c)], q < s_c; pair t of cluster c (t - sbase[c] =
// i * s_c + q) is (mem[i], sample q).  Pairs [t_lo, t_lo + np) of one chunk.
__global__ void gen_screen_pairs_kernel(const int32_t *__restrict__ members,
                                        const int32_t *__restrict__ cstart, const int32_t *__restrict__ cnt,
                                        const int32_t *__restrict__ ssz, const int64_t *__restrict__ sbase,
                                        int k, int64_t t_lo, int64_t np, int32_t *__restrict__ pa,
                                        int32_t *__restrict__ pb)
{
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= np) return;
    const int64_t t = t_lo + u;
    int lo = 0, hi = k - 1;  // last cluster with sbase <= t
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (sbase[mid] <= t) lo = mid;
        else hi = mid - 1;
    }
    const int c = lo, sc = ssz[c], m = cnt[c];
    const int64_t r = t - sbase[c];
    const int i = (int)(r / sc), q = (int)(r % sc);
    const int32_t *mem = members + cstart[c];
    pa[u] = mem[i];
    pb[u] = mem[(int)((int64_t)q * m / sc)];
}

// score[p] = sum over the sample of DTW(member p, sample q), q in order, float64;
// p indexes the member lists (cluster-major)
__global__ void screen_score_kernel(const float *__restrict__ R, int64_t r_lo, int64_t r_hi, int n, int k,
                                    const int32_t *__restrict__ cstart, const int32_t *__restrict__ ssz,
                                    const int64_t *__restrict__ sbase, double *__restrict__ score)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    int lo = 0, hi = k - 1;  // last cluster with cstart <= p
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (cstart[mid] <= p) lo = mid;
        else hi = mid - 1;
    }
    const int c = lo, sc = ssz[c];
    const int64_t t0 = sbase[c] + (int64_t)(p - cstart[c]) * sc;
    if (t0 < r_lo || t0 >= r_hi) return;  // this member's pairs belong to another chunk
    double acc = 0.0;
    for (int q = 0; q < sc; ++q) acc += (double)R[t0 - r_lo + q];
    score[p] = acc;
}

// the keep_c members of least score (ties to the smaller index), in that order,
// at cand[cbase[c] + nbase[c] ...]; one block per cluster
__global__ void screen_select_kernel(const double *__restrict__ score, const int32_t *__restrict__ members,
                                     const int32_t *__restrict__ cstart, const int32_t *__restrict__ cnt,
                                     const int32_t *__restrict__ cbase, const int32_t *__restrict__ nbase,
                                     const int32_t *__restrict__ keep, int32_t *__restrict__ cand)
{
    __shared__ double sd[256];
    __shared__ int si[256];
    const int c = blockIdx.x, tid = threadIdx.x, m = cnt[c];
    const int32_t *mem = members + cstart[c];
    const double *sc = score + cstart[c];
    double last_d = -1.0;
    int last_i = -1;
    for (int q = 0; q < keep[c]; ++q) {
        double bd = 1.0 / 0.0;
        int bi = 0x7fffffff;
        for (int r = tid; r < m; r += 256) {
            const double s = sc[r];
            const int j = mem[r];
            const bool after = s > last_d || (s == last_d && j > last_i);
            if (after && (s < bd || (s == bd && j < bi))) {
                bd = s;
                bi = j;
            }
        }
        sd[tid] = bd;
        si[tid] = bi;
        __syncthreads();
        for (int o = 128; o > 0; o >>= 1) {
            if (tid < o && (sd[tid + o] < sd[tid] || (sd[tid + o] == sd[tid] && si[tid + o] < si[tid]))) {
                sd[tid] = sd[tid + o];
                si[tid] = si[tid + o];
            }
            __syncthreads();
        }
        last_d = sd[0];
        last_i = si[0];
        if (tid == 0) cand[cbase[c] + nbase[c] + q] = last_i;
        __syncthreads();
    }
}

// pairs of candidate slots [s_lo, s_lo + nslots): slot s pairs with every member of
// its cluster; spoff[s - s_lo] is its first pair in the chunk
__global__ void gen_update_pairs_kernel(const int32_t *__restrict__ cand,
                                        const int32_t *__restrict__ slot_cl,
                                        const int64_t *__restrict__ spoff, int s_lo, int nslots,
                                        int64_t npairs, const int32_t *__restrict__ members,
                                        const int32_t *__restrict__ cstart,
                                        int32_t *__restrict__ pa, int32_t *__restrict__ pb)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= npairs) return;
    int lo = 0, hi = nslots - 1;  // last slot with spoff <= t
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (spoff[mid] <= t) lo = mid;
        else hi = mid - 1;
    }
    const int s = s_lo + lo, c = slot_cl[s];
    pa[t] = cand[s];
    pb[t] = members[cstart[c] + (int)(t - spoff[lo])];
}

// S[s] = sum of the slot's pair distances (f64, fixed-order block reduction)
__global__ void cand_sum_kernel(const float *__restrict__ out, const int64_t *__restrict__ spoff,
                                const int32_t *__restrict__ slot_cl, const int32_t *__restrict__ cnt,
                                int s_lo, double *__restrict__ S)
{
    __shared__ double sh[256];
    const int r = blockIdx.x, s = s_lo + r, tid = threadIdx.x;
    const int m = cnt[slot_cl[s]];
    const float *seg = out + spoff[r];
    double acc = 0.0;
    for (int q = tid; q < m; q += 256) acc += (double)seg[q];
    sh[tid] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (tid < o) sh[tid] += sh[tid + o];
        __syncthreads();
    }
    if (tid == 0) S[s] = sh[0];
}

// new medoid per cluster: smallest S; a tie keeps the current medoid, else the smallest index
__global__ void lazy_update_kernel(const double *__restrict__ S, const int32_t *__restrict__ cand,
                                   const int32_t *__restrict__ cbase, const int32_t *__restrict__ ncand,
                                   int k, const int32_t *__restrict__ M, int32_t *__restrict__ Mnew,
                                   int32_t *__restrict__ changed)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= k) return;
    double bs = 1.0 / 0.0;
    int bi = 0x7fffffff;
    double cur = 1.0 / 0.0;
    for (int q = 0; q < ncand[c]; ++q) {
        const double v = S[cbase[c] + q];
        const int j = cand[cbase[c] + q];
        if (j == M[c]) cur = v;
        if (v < bs || (v == bs && j < bi)) {
            bs = v;
            bi = j;
        }
    }
    const int chosen = (cur == bs) ? M[c] : bi;
    Mnew[c] = chosen;
    if (chosen != M[c]) atomicOr(changed, 1);
}

__global__ void cost_partial_kernel(const float *__restrict__ dmin, int n, double *__restrict__ part)
{
    __shared__ double sh[256];
    double acc = 0.0;
    for (int j = blockIdx.x * 256 + threadIdx.x; j < n; j += gridDim.x * 256) acc += (double)dmin[j];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

struct Pool {  // stream-ordered scratch owned by one call
    std::vector<void *> ptrs;
    cudaStream_t st;
    explicit Pool(cudaStream_t s) : st(s) {}
    ~Pool()
    {
        for (void *p : ptrs) scratch_free(p, st);
    }
    template <typename T>
    int get(T **p, size_t n)
    {
        void *q = nullptr;
        int rc = scratch_alloc(&q, sizeof(T) * (n ? n : 1), st);
        if (rc) return rc;
        ptrs.push_back(q);
        *p = (T *)q;
        return DTW_OK;
    }
};

constexpr int64_t kPairCap = 16ll << 20;  // pairs per update launch
constexpr int kCostBlocks = 64;
constexpr int kMaxScreen = 4096;  // sampled members per cluster

}  // namespace
}  // namespace dtwgb

using namespace dtwgb;

namespace dtwgb {
namespace {

// k-means++ centres into `centers` (device), asynchronous; D2 holds n doubles
void kpp_seed(const float *emb, int n, int dim, int k, uint64_t seed, int32_t *centers, double *D2,
              cudaStream_t st)
{
    uint64_t state = seed;
    set_first_kernel<<<1, 1, 0, st>>>(centers, (int32_t)(splitmix64_next(state) % (uint64_t)n));
    const bool vec4 = (dim % 4 == 0) && ((uintptr_t)emb % 16 == 0);
    for (int i = 1; i < k; ++i) {
        kpp_update_kernel<<<(n + 255) / 256, 256, 0, st>>>(emb, n, dim, centers, i - 1, D2, vec4);
        const double u = (double)(splitmix64_next(state) >> 11) * (1.0 / 9007199254740992.0);
        kpp_pick_kernel<<<1, kPickThreads, 0, st>>>(D2, n, u, centers, i);
    }
}

}  // namespace
}  // namespace dtwgb

extern "C" int proposal_kmeanspp(const float *emb, int32_t n, int32_t dim, int32_t k, uint64_t seed,
                                 int32_t *out_medoids, void *stream)
{
    clear_error();
    if (!emb || !out_medoids) { set_error("NULL pointer argument"); return DTW_EINVAL; }
    if (n < 1 || dim < 1 || k < 1 || k > n) {
        set_error("need n >= 1, dim >= 1, 1 <= k <= n (n = %d, dim = %d, k = %d)", n, dim, k);
        return DTW_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    Pool pool(st);
    double *D2 = nullptr;
    int rc = pool.get(&D2, (size_t)n);
    if (rc) return rc;
    kpp_seed(emb, n, dim, k, seed, out_medoids, D2, st);
    DTWGB_CUDA(cudaGetLastError());
    return DTW_OK;
}

extern "C" int proposal_kmeans(const float *emb, int32_t n, int32_t dim, int32_t k,
                               int32_t restarts, int32_t iters, uint64_t seed,
                               int32_t *out_medoids, double *out_inertia, void *stream)
{
    clear_error();
    if (!emb || !out_medoids) { set_error("NULL pointer argument"); return DTW_EINVAL; }
    if (n < 1 || dim < 1 || dim > 1024 || k < 1 || k > n || restarts < 1 || iters < 0) {
        set_error("need n >= 1, 1 <= dim <= 1024, 1 <= k <= n, restarts >= 1, iters >= 0 "
                  "(n = %d, dim = %d, k = %d, restarts = %d, iters = %d)", n, dim, k, restarts, iters);
        return DTW_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    Pool pool(st);
    double *D2, *part, *best;
    int32_t *seeds, *lab, *cnt, *cstart, *members, *changed, *stop, *pcnt = nullptr;
    float *C, *bestC, *dist, *psum = nullptr;
    int rc;
    const bool chunked = (int64_t)k * dim <= kKmSmemFloats;  // shared accumulators fit
    const int nchunks = (n + kKmChunk - 1) / kKmChunk;
    if ((rc = pool.get(&D2, n)) || (rc = pool.get(&part, kCostBlocks)) || (rc = pool.get(&best, 1)) ||
        (rc = pool.get(&seeds, k)) || (rc = pool.get(&lab, n)) || (rc = pool.get(&cnt, k)) ||
        (rc = pool.get(&cstart, k + 1)) || (rc = pool.get(&members, n)) ||
        (rc = pool.get(&changed, 2)) || (rc = pool.get(&stop, 1)) ||
        (rc = pool.get(&C, (size_t)k * dim)) ||
        (rc = pool.get(&bestC, (size_t)k * dim)) || (rc = pool.get(&dist, n)))
        return rc;
    if (chunked && ((rc = pool.get(&psum, (size_t)nchunks * k * dim)) ||
                    (rc = pool.get(&pcnt, (size_t)nchunks * k))))
        return rc;
    const int pthreads = std::min(1024, (dim + 31) / 32 * 32);
    const size_t psh = sizeof(float) * (size_t)k * dim + sizeof(int) * (size_t)k;
    if (chunked)
        DTWGB_CUDA(cudaFuncSetAttribute(km_partial_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)psh));  // <= 96 KB: k * dim <= 12288 and k <= 12288
    const unsigned nb = (unsigned)((n + 255) / 256), kb = (unsigned)((k * dim + 255) / 256);
    // assignment: smaller blocks so that a 20000-point set covers every SM; float4 rows and
    // shared centroids where the layout allows (the centroids are in shared memory when chunked)
    const unsigned nba = (unsigned)((n + kAssignThreads - 1) / kAssignThreads);
    const bool avec4 = chunked && dim % 4 == 0 && (uintptr_t)emb % 16 == 0;
    const size_t csh = sizeof(float) * kCentWarps * dim;
    const size_t ash = chunked ? sizeof(float) * (size_t)k * dim : 0;  // <= 48 KB
    auto assign_members = [&](const float *Cc) -> int {
        DTWGB_CUDA(cudaMemsetAsync(changed, 0, sizeof(int32_t), st));
        km_assign_kernel<<<nba, kAssignThreads, ash, st>>>(emb, n, dim, Cc, k, lab, dist, changed,
                                                           nullptr, chunked, avec4);
        DTWGB_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * k, st));
        count_kernel<<<nb, 256, 0, st>>>(lab, n, cnt);
        prefix_kernel<<<1, 1, 0, st>>>(cnt, k, cstart);
        members_kernel<<<k, 256, 0, st>>>(lab, n, cstart, members);
        DTWGB_CUDA(cudaGetLastError());
        return DTW_OK;
    };
    for (int r = 0; r < restarts; ++r) {
        kpp_seed(emb, n, dim, k, seed + (uint64_t)r, seeds, D2, st);
        gather_rows_kernel<<<kb, 256, 0, st>>>(emb, dim, seeds, k, C);
        DTWGB_CUDA(cudaMemsetAsync(lab, 0xff, sizeof(int32_t) * n, st));  // labels -1
        if (chunked) {
            // all iterations enqueued at once, three launches each; after the first
            // assignment that changes no label (C is then their centroid already) every
            // kernel returns at once.  Iteration `it` sets changed[it & 1]; its reduction
            // clears the other word for the next one.
            DTWGB_CUDA(cudaMemsetAsync(stop, 0, sizeof(int32_t), st));
            DTWGB_CUDA(cudaMemsetAsync(changed, 0, 2 * sizeof(int32_t), st));
            for (int it = 0; it < iters; ++it) {
                int32_t *cur = changed + (it & 1), *nxt = changed + ((it + 1) & 1);
                km_assign_kernel<<<nba, kAssignThreads, ash, st>>>(emb, n, dim, C, k, lab, dist,
                                                                   cur, stop, 1, avec4);
                km_partial_kernel<<<nchunks, pthreads, psh, st>>>(emb, n, dim, lab, k, psum, pcnt,
                                                                  cur);
                km_reduce_kernel<<<(unsigned)((k * dim + 31) / 32), 32 * kRedWarps, 0, st>>>(
                    psum, pcnt, nchunks, k, dim, C, cur, nxt, stop);
            }
            DTWGB_CUDA(cudaGetLastError());
        } else {
            for (int it = 0; it < iters; ++it) {
                if ((rc = assign_members(C))) return rc;
                int32_t h = 0;
                DTWGB_CUDA(cudaMemcpyAsync(&h, changed, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
                DTWGB_CUDA(cudaStreamSynchronize(st));
                if (!h) break;  // labels stable: C is their centroid already
                centroid_kernel<<<k, 32 * kCentWarps, csh, st>>>(emb, dim, members, cstart, cnt, C);
                DTWGB_CUDA(cudaGetLastError());
            }
        }
        // inertia of the final centroids
        DTWGB_CUDA(cudaMemsetAsync(changed, 0, sizeof(int32_t), st));
        km_assign_kernel<<<nba, kAssignThreads, ash, st>>>(emb, n, dim, C, k, lab, dist, changed,
                                                           nullptr, chunked, avec4);
        cost_partial_kernel<<<kCostBlocks, 256, 0, st>>>(dist, n, part);
        keep_best_kernel<<<1, 256, 0, st>>>(part, kCostBlocks, C, k * dim, best, bestC, r == 0);
        DTWGB_CUDA(cudaGetLastError());
    }
    if ((rc = assign_members(bestC))) return rc;
    nearest_member_kernel<<<k, 256, 0, st>>>(dist, members, cstart, cnt, out_medoids);
    fill_empty_kernel<<<1, 1, 0, st>>>(emb, n, dim, bestC, k, out_medoids);
    DTWGB_CUDA(cudaGetLastError());
    double hb = 0.0;
    DTWGB_CUDA(cudaMemcpyAsync(&hb, best, sizeof(double), cudaMemcpyDeviceToHost, st));
    DTWGB_CUDA(cudaStreamSynchronize(st));
    if (out_inertia) *out_inertia = hb;
    return DTW_OK;
}

extern "C" int kmedoids_lazy_fit(const float *values, const int64_t *offsets, int32_t n,
                                 int32_t window, uint32_t flags, const float *emb, int32_t dim,
                                 int32_t k, const int32_t *init_medoids, int32_t candidates,
                                 int32_t screen_sample, int32_t screen_keep, int32_t max_iter,
                                 int32_t *out_medoids, int32_t *out_labels, double *out_cost,
                                 int32_t *out_iters, int64_t *out_pairs, void *stream)
{
    clear_error();
    cudaStream_t st = (cudaStream_t)stream;
    if (n < 1) { set_error("n = %d must be >= 1", n); return DTW_EINVAL; }
    if (k < 1 || k > n) { set_error("k = %d must be in [1, n = %d]", k, n); return DTW_EINVAL; }
    if (max_iter < 1) { set_error("max_iter = %d must be >= 1", max_iter); return DTW_EINVAL; }
    if (!values || !offsets || !init_medoids || !out_medoids || !out_labels) {
        set_error("NULL pointer argument");
        return DTW_EINVAL;
    }
    if (emb && (dim < 1 || dim > 1024)) { set_error("dim = %d must be in [1, 1024]", dim); return DTW_EINVAL; }
    if (screen_sample < 0 || screen_sample > kMaxScreen || screen_keep < 0 ||
        (screen_sample > 0 && screen_keep < 1)) {
        set_error("screen_sample = %d must be in [0, %d] and screen_keep = %d >= 1 when sampling",
                  screen_sample, kMaxScreen, screen_keep);
        return DTW_EINVAL;
    }
    const bool propose = emb && candidates > 0;
    const bool screen = screen_sample > 0;
    const bool every = !propose && !screen;  // every member a candidate: the plain update

    std::vector<int64_t> hoff((size_t)n + 1);
    std::vector<int32_t> hM((size_t)k);
    cudaError_t e = cudaMemcpyAsync(hoff.data(), offsets, sizeof(int64_t) * ((size_t)n + 1),
                                    cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(hM.data(), init_medoids, sizeof(int32_t) * (size_t)k,
                            cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "reading offsets and initial medoids");
    for (int c = 0; c < k; ++c) {
        if (hM[c] < 0 || hM[c] >= n) { set_error("init_medoids[%d] = %d is outside [0, %d)", c, hM[c], n); return DTW_EINVAL; }
        for (int d = 0; d < c; ++d)
            if (hM[d] == hM[c]) { set_error("init_medoids[%d] and [%d] are both %d", d, c, hM[c]); return DTW_EINVAL; }
    }

    DtwListCtx ctx;
    int rc = dtw_list_prepare(values, offsets, hoff.data(), n, window, flags, &ctx, st);
    if (rc) return rc;
    struct Release {
        DtwListCtx *c;
        cudaStream_t s;
        ~Release() { dtw_list_release(c, s); }
    } release{&ctx, st};

    Pool pool(st);
    const int64_t kn = (int64_t)k * n;
    const int64_t cap = std::max<int64_t>(std::max<int64_t>(kPairCap, kn), (int64_t)n * screen_sample);
    const int64_t slots = 2 * (int64_t)n + k;  // base (<= |C_c|) plus screened (<= |C_c|) per cluster
    int32_t *pa, *pb, *M, *Mn, *flag, *cnt, *cstart, *members, *cand, *cbase, *ncand, *nbase, *keep,
        *slot_cl, *ssz = nullptr;
    int64_t *spoff, *sbase = nullptr;
    float *R, *dmin, *cent = nullptr, *cdist = nullptr;
    double *S, *cpart, *score = nullptr;
    if ((rc = pool.get(&pa, cap)) || (rc = pool.get(&pb, cap)) || (rc = pool.get(&R, cap)) ||
        (rc = pool.get(&M, k)) || (rc = pool.get(&Mn, k)) || (rc = pool.get(&flag, 1)) ||
        (rc = pool.get(&cnt, k)) || (rc = pool.get(&cstart, k + 1)) || (rc = pool.get(&members, n)) ||
        (rc = pool.get(&cand, slots)) || (rc = pool.get(&cbase, k + 1)) || (rc = pool.get(&ncand, k)) ||
        (rc = pool.get(&nbase, k)) || (rc = pool.get(&keep, k)) ||
        (rc = pool.get(&slot_cl, slots)) || (rc = pool.get(&spoff, slots + 1)) ||
        (rc = pool.get(&dmin, n)) || (rc = pool.get(&S, slots)) || (rc = pool.get(&cpart, kCostBlocks)))
        return rc;
    if (propose && ((rc = pool.get(&cent, (size_t)k * dim)) || (rc = pool.get(&cdist, n)))) return rc;
    if (screen && ((rc = pool.get(&ssz, k)) || (rc = pool.get(&sbase, k + 1)) ||
                   (rc = pool.get(&score, n))))
        return rc;
    DTWGB_CUDA(cudaMemcpyAsync(M, init_medoids, sizeof(int32_t) * k, cudaMemcpyDeviceToDevice, st));

    int64_t pairs = 0;
    auto assign = [&]() -> int {
        gen_assign_pairs_kernel<<<(unsigned)((kn + 255) / 256), 256, 0, st>>>(M, k, n, pa, pb);
        int r2 = dtw_list_run(&ctx, pa, pb, kn, R, st);
        if (r2) return r2;
        lazy_assign_kernel<<<(n + 255) / 256, 256, 0, st>>>(R, k, n, M, out_labels, dmin);
        pairs += kn;
        DTWGB_CUDA(cudaGetLastError());
        return DTW_OK;
    };

    std::vector<int32_t> hcnt(k), hstart(k + 1), hncand(k), hnbase(k), hkeep(k), hcbase(k + 1),
        hssz(k), hslot;
    std::vector<int64_t> hspoff, hsbase(k + 1);
    int32_t iters = 0;
    bool converged = false;
    for (int32_t it = 1; it <= max_iter; ++it) {
        if ((rc = assign())) return rc;
        // cluster sizes and member lists
        DTWGB_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * k, st));
        count_kernel<<<(n + 255) / 256, 256, 0, st>>>(out_labels, n, cnt);
        DTWGB_CUDA(cudaMemcpyAsync(hcnt.data(), cnt, sizeof(int32_t) * k, cudaMemcpyDeviceToHost, st));
        DTWGB_CUDA(cudaStreamSynchronize(st));
        hstart[0] = 0;
        for (int c = 0; c < k; ++c) hstart[c + 1] = hstart[c] + hcnt[c];
        hcbase[0] = 0;
        hsbase[0] = 0;
        for (int c = 0; c < k; ++c) {
            hnbase[c] = every ? hcnt[c] : propose ? std::min(candidates, hcnt[c]) : 1;
            hkeep[c] = screen ? std::min(screen_keep, hcnt[c]) : 0;
            hncand[c] = hnbase[c] + hkeep[c];
            hcbase[c + 1] = hcbase[c] + hncand[c];
            hssz[c] = std::min(screen_sample, hcnt[c]);
            hsbase[c + 1] = hsbase[c] + (int64_t)hcnt[c] * hssz[c];
        }
        DTWGB_CUDA(cudaMemcpyAsync(cstart, hstart.data(), sizeof(int32_t) * (k + 1), cudaMemcpyHostToDevice, st));
        DTWGB_CUDA(cudaMemcpyAsync(cbase, hcbase.data(), sizeof(int32_t) * (k + 1), cudaMemcpyHostToDevice, st));
        DTWGB_CUDA(cudaMemcpyAsync(ncand, hncand.data(), sizeof(int32_t) * k, cudaMemcpyHostToDevice, st));
        DTWGB_CUDA(cudaMemcpyAsync(nbase, hnbase.data(), sizeof(int32_t) * k, cudaMemcpyHostToDevice, st));
        DTWGB_CUDA(cudaMemcpyAsync(keep, hkeep.data(), sizeof(int32_t) * k, cudaMemcpyHostToDevice, st));
        members_kernel<<<k, 256, 0, st>>>(out_labels, n, cstart, members);
        if (every) {
            DTWGB_CUDA(cudaMemcpyAsync(cand, members, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, st));
        } else {
            if (propose)
                centroid_kernel<<<k, 32 * kCentWarps, sizeof(float) * kCentWarps * dim, st>>>(
                    emb, dim, members, cstart, cnt, cent);
            // with nbase 1 only the medoid is written; the distances are not read
            if (propose)
                member_dist_kernel<<<(n + 255) / 256, 256, 0, st>>>(emb, dim, members, out_labels, n,
                                                                    cent, cdist);
            candidates_kernel<<<k, 256, 0, st>>>(cdist, members, cstart, cnt, M, cbase, nbase, cand);
        }
        if (screen) {  // one chunk: cap >= n * screen_sample >= every screening pair
            const int64_t ns = hsbase[k];
            DTWGB_CUDA(cudaMemcpyAsync(ssz, hssz.data(), sizeof(int32_t) * k, cudaMemcpyHostToDevice, st));
            DTWGB_CUDA(cudaMemcpyAsync(sbase, hsbase.data(), sizeof(int64_t) * (k + 1), cudaMemcpyHostToDevice, st));
            gen_screen_pairs_kernel<<<(unsigned)((ns + 255) / 256), 256, 0, st>>>(
                members, cstart, cnt, ssz, sbase, k, 0, ns, pa, pb);
            if ((rc = dtw_list_run(&ctx, pa, pb, ns, R, st))) return rc;
            screen_score_kernel<<<(n + 255) / 256, 256, 0, st>>>(R, 0, ns, n, k, cstart, ssz, sbase, score);
            screen_select_kernel<<<k, 256, 0, st>>>(score, members, cstart, cnt, cbase, nbase, keep, cand);
            pairs += ns;
        }
        // candidate slots, their clusters, and chunks of at most `cap` pairs
        const int nslots = hcbase[k];
        hslot.assign(nslots, 0);
        for (int c = 0; c < k; ++c)
            for (int q = 0; q < hncand[c]; ++q) hslot[hcbase[c] + q] = c;
        DTWGB_CUDA(cudaMemcpyAsync(slot_cl, hslot.data(), sizeof(int32_t) * nslots, cudaMemcpyHostToDevice, st));
        int s0 = 0;
        while (s0 < nslots) {
            hspoff.assign(1, 0);
            int s1 = s0;
            while (s1 < nslots && (s1 == s0 || hspoff.back() + hcnt[hslot[s1]] <= cap)) {
                hspoff.push_back(hspoff.back() + hcnt[hslot[s1]]);
                ++s1;
            }
            const int64_t np = hspoff.back();
            DTWGB_CUDA(cudaMemcpyAsync(spoff, hspoff.data(), sizeof(int64_t) * hspoff.size(),
                                       cudaMemcpyHostToDevice, st));
            gen_update_pairs_kernel<<<(unsigned)((np + 255) / 256), 256, 0, st>>>(
                cand, slot_cl, spoff, s0, s1 - s0, np, members, cstart, pa, pb);
            if ((rc = dtw_list_run(&ctx, pa, pb, np, R, st))) return rc;
            cand_sum_kernel<<<s1 - s0, 256, 0, st>>>(R, spoff, slot_cl, cnt, s0, S);
            pairs += np;
            // the host vectors are reused by the next chunk: wait for the copies
            DTWGB_CUDA(cudaStreamSynchronize(st));
            s0 = s1;
        }
        DTWGB_CUDA(cudaMemsetAsync(flag, 0, sizeof(int32_t), st));
        lazy_update_kernel<<<(k + 31) / 32, 32, 0, st>>>(S, cand, cbase, ncand, k, M, Mn, flag);
        int32_t hflag = 0;
        DTWGB_CUDA(cudaMemcpyAsync(&hflag, flag, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        DTWGB_CUDA(cudaStreamSynchronize(st));
        iters = it;
        if (!hflag) {
            converged = true;  // labels and dmin already belong to M
            break;
        }
        std::swap(M, Mn);
    }
    if (!converged && (rc = assign())) return rc;
    cost_partial_kernel<<<kCostBlocks, 256, 0, st>>>(dmin, n, cpart);
    std::vector<double> hpart(kCostBlocks);
    DTWGB_CUDA(cudaMemcpyAsync(hpart.data(), cpart, sizeof(double) * kCostBlocks, cudaMemcpyDeviceToHost, st));
    DTWGB_CUDA(cudaMemcpyAsync(out_medoids, M, sizeof(int32_t) * k, cudaMemcpyDeviceToDevice, st));
    DTWGB_CUDA(cudaStreamSynchronize(st));
    double cost = 0.0;
    for (double v : hpart) cost += v;
    if (out_cost) *out_cost = cost;
    if (out_iters) *out_iters = iters;
    if (out_pairs) *out_pairs = pairs;
    return DTW_OK;
}
