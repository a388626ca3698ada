// encoder.cu -- forward, backward and Adam of the proposal encoder
// (dtwgb_encoder.h) on sm_103a.
//
// Activations are bfloat16, time-major [B][T][64].  The 64-channel
// convolutions are implicit GEMMs on the fifth-generation tensor cores
// (tcgen05.mma, bf16 operands from shared memory, f32 accumulators in TMEM):
// out[t][n] = sum_k sum_c in[t + s(k)][c] * W[k][n][c], s(k) = k - 3 forward
// and 3 - k for the input gradient (with the transposed weights).  A CTA keeps
// all 7 taps of the weights in shared memory and walks (series, 128-step tile)
// items.  Weight gradients are tcgen05 GEMMs over (series, time) reading the
// same time-major tiles as MN-major operands; per-CTA partial sums are added
// in a fixed order, so a step is deterministic.
// Conv1 (one input channel), pooling, the linear layer, the loss and Adam are
// small CUDA-core kernels.
#include <cuda_bf16.h>
#include <cudaTypedefs.h>  // PFN_cuTensorMapEncodeTiled

#include <cstring>
#include <vector>

#include "../../include/dtwgb_encoder.h"
#include "common.cuh"
#include "tc.cuh"

namespace dtwgb {
namespace {

using bf16 = __nv_bfloat16;
constexpr int C = 64, KW = 7;
constexpr int OFF_W1 = 0, OFF_B1 = 448, OFF_W2 = 512, OFF_B2 = 29184, OFF_W3 = 29248,
              OFF_B3 = 57920, OFF_WL = 57984, OFF_BL = 62080, NPAR = 62144;
constexpr int kMaxT = 832;     // longest series the encoder accepts

// GELU(z) = z Phi(z) and GELU'(z) = Phi(z) + z phi(z), Phi(z) = (1 + erf(z / sqrt 2)) / 2,
// phi(z) = exp(-z^2 / 2) / sqrt(2 pi).  erf by the rational approximation of Abramowitz &
// Stegun 7.1.26 (after Hastings): for x >= 0,
//   erfc(x) ~ t (a1 + t (a2 + t (a3 + t (a4 + t a5)))) exp(-x^2),  t = 1 / (1 + p x),
// |error| <= 1.5e-7.  With x = |z| / sqrt 2, 1 + erf(z / sqrt 2) is 2 - erfc(x) for z >= 0
// and erfc(x) itself for z < 0 (no cancellation in the negative tail), and exp(-x^2) is
// exp(-z^2 / 2), which GELU' needs too: one reciprocal and one exponential per element.
// Every result is stored as bfloat16 (2^-9 relative), far above the approximation error.
struct GeluParts {
    float one_plus_erf;  // 1 + erf(z / sqrt 2) = 2 Phi(z)
    float gauss;         // exp(-z^2 / 2)
};

__device__ __forceinline__ GeluParts gelu_parts(float z)
{
    const float x = fabsf(z) * 0.70710678118654752f;
    const float t = __fdividef(1.f, fmaf(0.3275911f, x, 1.f));
    float poly = fmaf(1.061405429f, t, -1.453152027f);
    poly = fmaf(poly, t, 1.421413741f);
    poly = fmaf(poly, t, -0.284496736f);
    poly = fmaf(poly, t, 0.254829592f);
    const float g = __expf(-x * x);
    const float ec = poly * t * g;  // erfc(x)
    return {z < 0.f ? ec : 2.f - ec, g};
}

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * gelu_parts(z).one_plus_erf; }

__device__ __forceinline__ float gelu_grad(float z)
{
    const GeluParts q = gelu_parts(z);
    return fmaf(z * q.gauss, 0.39894228040143268f, 0.5f * q.one_plus_erf);
}

__device__ __forceinline__ uint32_t pack2(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}

__device__ __forceinline__ float bfr(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

// Activations and their gradients are stored channel-group-blocked: element
// (series b, step t, channel c) at ((b * 8 + c / 8) * T + t) * 8 + c % 8, so the
// 16-byte rows of one channel group of one series are contiguous in time.
__device__ __forceinline__ int64_t aidx(int64_t b, int t, int c, int T)
{
    return ((b * 8 + (c >> 3)) * T + t) * 8 + (c & 7);
}

// ---------------------------------------------------------------- conv1

// z1[b][t][c] = b1[c] + sum_k W1[c][k] * xq[b][t+k-3]  (xq: x rounded to bf16).
// One block of 256 threads per 64-step tile of one series (T is a multiple of
// 64, so a tile never crosses series): x with its halo, W1 and b1 in shared
// memory; thread (c, row group) writes rows 4j + group, 128-byte rows.
__global__ void conv1_fwd_kernel(const float *__restrict__ x, const float *__restrict__ W1,
                                 const float *__restrict__ b1, int B, int T,
                                 bf16 *__restrict__ z1, bf16 *__restrict__ h1)
{
    __shared__ float xs[70], ws[KW * 64], bs[64];
    const int tiles = T / 64, tile = blockIdx.x;
    const int b = tile / tiles, t0 = (tile % tiles) * 64, tid = threadIdx.x;
    const float *xb = x + (int64_t)b * T;
    if (tid < 70) {
        const int t = t0 - 3 + tid;
        xs[tid] = (t >= 0 && t < T) ? bfr(xb[t]) : 0.f;
    }
    for (int i = tid; i < KW * 64; i += 256) ws[i] = W1[i];
    if (tid < 64) bs[tid] = b1[tid];
    __syncthreads();
    // thread (row r, channel group g) writes 8 channels: a warp covers 32 steps of one
    // group, 512 contiguous bytes
    for (int u = tid; u < 64 * 8; u += 256) {
        const int r = u & 63, g = u >> 6;
        uint32_t zw[4], hw[4];
#pragma unroll
        for (int e = 0; e < 8; e += 2) {
            float acc0 = bs[g * 8 + e], acc1 = bs[g * 8 + e + 1];
#pragma unroll
            for (int k = 0; k < KW; ++k) {
                acc0 = fmaf(ws[(g * 8 + e) * KW + k], xs[r + k], acc0);
                acc1 = fmaf(ws[(g * 8 + e + 1) * KW + k], xs[r + k], acc1);
            }
            zw[e / 2] = pack2(acc0, acc1);
            hw[e / 2] = pack2(gelu(acc0), gelu(acc1));
        }
        const int64_t idx = aidx(b, t0 + r, g * 8, T);
        if (z1) *reinterpret_cast<uint4 *>(z1 + idx) = make_uint4(zw[0], zw[1], zw[2], zw[3]);
        *reinterpret_cast<uint4 *>(h1 + idx) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
    }
}

// Partial sums of dW1 and db1 over the 64-step tiles tile = blockIdx.x,
// blockIdx.x + gridDim.x, ... (in that order): part[block][j], j = c * 7 + k
// for W1 (parameter order) and 448 + c for b1, so a fixed-order sum over the
// blocks lands on the parameter vector directly.  Warp w takes channel group w
// of every tile, lane l its rows l and l + 32: 16-byte loads of 8 channels, 512
// contiguous bytes per warp.  Each thread keeps its 8 channels x (7 taps +
// bias) over all of the block's tiles; a fixed butterfly then sums the 32
// lanes, so the partials are deterministic.
constexpr int kC1Blocks = 608;
__global__ void __launch_bounds__(256) conv1_wgrad_kernel(const bf16 *__restrict__ dz1,
                                                          const float *__restrict__ x, int B,
                                                          int T, float *__restrict__ part)
{
    __shared__ float xw[8][72];  // per warp: xq[t0 - 3 .. t0 + 66] of the current tile
    const unsigned FULL = 0xffffffffu;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tiles = T / 64, ntiles = B * tiles;
    float acc[8][8];
#pragma unroll
    for (int c = 0; c < 8; ++c)
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[c][k] = 0.f;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int b = tile / tiles, t0 = (tile % tiles) * 64;
        const uint4 q0 = __ldg(reinterpret_cast<const uint4 *>(dz1 + aidx(b, t0 + lane, warp * 8, T)));
        const uint4 q1 =
            __ldg(reinterpret_cast<const uint4 *>(dz1 + aidx(b, t0 + lane + 32, warp * 8, T)));
        const float *xb = x + (int64_t)b * T;
        __syncwarp();  // the previous tile's window is no longer read
        for (int i = lane; i < 70; i += 32) {
            const int t = t0 - 3 + i;
            xw[warp][i] = (t >= 0 && t < T) ? bfr(xb[t]) : 0.f;
        }
        __syncwarp();
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const uint4 q = h ? q1 : q0;
            const int r = lane + 32 * h;
            const uint32_t wd[4] = {q.x, q.y, q.z, q.w};
            float xv[KW];
#pragma unroll
            for (int k = 0; k < KW; ++k) xv[k] = xw[warp][r + k];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const __nv_bfloat162 v2 = *reinterpret_cast<const __nv_bfloat162 *>(&wd[e]);
                const float d0 = __low2float(v2), d1 = __high2float(v2);
#pragma unroll
                for (int k = 0; k < KW; ++k) {
                    acc[2 * e][k] = fmaf(d0, xv[k], acc[2 * e][k]);
                    acc[2 * e + 1][k] = fmaf(d1, xv[k], acc[2 * e + 1][k]);
                }
                acc[2 * e][7] += d0;
                acc[2 * e + 1][7] += d1;
            }
        }
    }
    // sum the 32 lanes (rows) by a fixed butterfly; every lane ends with the totals
#pragma unroll
    for (int c = 0; c < 8; ++c)
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            float v = acc[c][k];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(FULL, v, off);
            acc[c][k] = v;
        }
    // lane c (< 8) writes channel warp * 8 + c: 7 taps and the bias
    float *row = part + (int64_t)blockIdx.x * 512;
#pragma unroll
    for (int c = 0; c < 8; ++c)
        if (lane == c) {
            const int ch = warp * 8 + c;
#pragma unroll
            for (int k = 0; k < KW; ++k) row[ch * KW + k] = acc[c][k];
            row[448 + ch] = acc[c][7];
        }
}

// ------------------------------------------- 64-channel convs, tcgen05 / TMEM
//
// Tile = 128 time steps of one series.  out[t][n] = sum_k sum_c in[t + s(k)][c] *
// W[k][n][c] is 7 taps x 4 blocks of 16 channels = 28 MMAs of M = 128 (time)
// x N = 64 (outputs) x K = 16 into one f32 accumulator of 64 TMEM columns.
// The input tile is staged once with its 3-step halo; tap k's A operand is the
// same tile viewed s(k) + 3 rows lower (row stride 16 bytes, see tc.cuh).
//
// Persistent, warp-specialised CTA (10 warps):
//   warp 0      producer: the pre-tiled weights in one bulk copy, then per
//               tile one tensor-map copy of the 136 rows of all 8 channel
//               groups into a ring of 3 stages (rows outside [0, T) arrive as
//               zeros from the tensor map's bounds)
//   warp 1      MMA issuer: 28 tcgen05.mma per tile into one of 2 accumulators
//   warps 2-9   epilogue: warp w reads TMEM lanes 32(w%4).. (rows) and half of
//               the 64 columns, adds the bias and applies GELU (forward) or
//               multiplies by GELU'(z_prev) (input gradient), stores bf16
// mbarriers: full/empty per stage (TMA bytes / MMA completion), full/empty per
// accumulator (MMA completion / 8 epilogue warps).  Shared memory:
//   weights  7 taps x [8 channel groups][64 n][16 B]    57,344 B (LBO 1024, SBO 128)
//   inputs   3 x [8 channel groups][136 rows][16 B]     52,224 B (LBO 2176, SBO 128)
constexpr int kTcRows = 128;
constexpr int kTcR = 136;
constexpr int kTcStages = 3;
constexpr int kTcEpiWarps = 8;
constexpr int kTcThreads = 32 * (2 + kTcEpiWarps);
constexpr uint32_t kTcWBytes = KW * 64 * 64 * 2;
constexpr uint32_t kTcLbA = kTcR * 16, kTcLbW = 64 * 16, kTcSb = 128;
constexpr uint32_t kTcABytes = 8 * kTcLbA;
constexpr size_t kTcSmem = kTcWBytes + kTcStages * kTcABytes + 256 + 1024;
constexpr uint32_t kTcWaitLimit = 1u << 24;

template <bool BWD>
__global__ void __launch_bounds__(kTcThreads, 2)
    conv_tc_kernel(const __grid_constant__ CUtensorMap in_map, const bf16 *__restrict__ Wk,
                   const float *__restrict__ bias, const bf16 *__restrict__ zprev,
                   bf16 *__restrict__ out_z, bf16 *__restrict__ out, int B, int T,
                   int *__restrict__ err)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    unsigned char *Ws = base;
    unsigned char *As = base + kTcWBytes;
    uint64_t *full = reinterpret_cast<uint64_t *>(As + kTcStages * kTcABytes);
    uint64_t *empty = full + kTcStages;
    uint64_t *accf = empty + kTcStages;
    uint64_t *acce = accf + 2;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(acce + 3);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tslot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    uint64_t *wfull = acce + 2;
    if (tid == 0) {
        tc::mbar_init(wfull, 1);
        for (int q = 0; q < kTcStages; ++q) {
            tc::mbar_init(&full[q], 1);
            tc::mbar_init(&empty[q], 1);
        }
        for (int a = 0; a < 2; ++a) {
            tc::mbar_init(&accf[a], 1);
            tc::mbar_init(&acce[a], kTcEpiWarps);
        }
        *abort_flag = 0;
    }
    if (warp == 1) tc::tmem_alloc(tslot, 128);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    const int tiles = (T + kTcRows - 1) / kTcRows;
    const int64_t nitems = (int64_t)B * tiles;
    bool failed = false;

    if (warp == 0) {
        if (lane == 0) {
            // the weights arrive pre-tiled (tap k, channel group g, row n, 8 channels) in one copy
            tc::mbar_expect_tx(wfull, kTcWBytes);
            tc::bulk_load(Ws, Wk, kTcWBytes, wfull);
        }
        int i = 0;
        for (int64_t item = blockIdx.x; item < nitems; item += gridDim.x, ++i) {
            const int st = i % kTcStages;
            const uint32_t ph = (uint32_t)(i / kTcStages) & 1u;
            int ok = 1;
            if (lane == 0) ok = tc::mbar_wait(&empty[st], ph ^ 1u, kTcWaitLimit, abort_flag);
            if (!__shfl_sync(0xffffffffu, ok, 0)) {
                failed = true;
                break;
            }
            const int64_t b = item / tiles;
            const int t0 = (int)(item % tiles) * kTcRows;
            unsigned char *dst = As + st * kTcABytes;
            // rows t0 - 3 .. t0 + 132 of the 8 channel groups of series b
            if (lane == 0) {
                tc::mbar_expect_tx(&full[st], kTcABytes);
                tc::tensor_load_3d(dst, &in_map, 0, t0 - 3, (int)(b * 8), &full[st]);
            }
            __syncwarp();
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = tc::idesc_bf16_f32(kTcRows, 64);
            const uint32_t wbase = tc::smem_addr(Ws);
            if (!tc::mbar_wait(wfull, 0, kTcWaitLimit, abort_flag)) failed = true;
            int i = 0;
            for (int64_t item = blockIdx.x; item < nitems && !failed; item += gridDim.x, ++i) {
                const int st = i % kTcStages, a = i & 1;
                const uint32_t ph = (uint32_t)(i / kTcStages) & 1u, aph = (uint32_t)(i >> 1) & 1u;
                if (!tc::mbar_wait(&acce[a], aph ^ 1u, kTcWaitLimit, abort_flag) ||
                    !tc::mbar_wait(&full[st], ph, kTcWaitLimit, abort_flag)) {
                    failed = true;
                    break;
                }
                tc::fence_after_sync();
                const uint32_t abase = tc::smem_addr(As + st * kTcABytes);
                const uint32_t acc = tmem + (uint32_t)(a * 64);
#pragma unroll 1
                for (int k = 0; k < KW; ++k) {
                    const uint32_t shift = (uint32_t)(BWD ? 6 - k : k);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const uint64_t ad =
                            tc::desc_kmajor(abase + shift * 16 + 2 * q * kTcLbA, kTcLbA, kTcSb);
                        const uint64_t bd =
                            tc::desc_kmajor(wbase + k * 8192 + 2 * q * kTcLbW, kTcLbW, kTcSb);
                        tc::mma_bf16(acc, ad, bd, idesc, (k | q) != 0);
                    }
                }
                tc::commit(&empty[st]);
                tc::commit(&accf[a]);
            }
        }
    } else {
        const int q = warp & 3, hc = (warp - 2) >> 2;
        float bv[32];  // this warp's 32 bias values (forward)
#pragma unroll
        for (int e = 0; e < 32; ++e) bv[e] = BWD ? 0.f : bias[hc * 32 + e];
        int i = 0;
        for (int64_t item = blockIdx.x; item < nitems; item += gridDim.x, ++i) {
            const int a = i & 1;
            const uint32_t aph = (uint32_t)(i >> 1) & 1u;
            const int64_t b = item / tiles;
            const int t = (int)(item % tiles) * kTcRows + q * 32 + lane;
            const bool live = t < T;
            uint4 zq[4];  // z_prev of this row's 32 columns, fetched while the MMAs run
            if (BWD && live) {
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    zq[e] = *reinterpret_cast<const uint4 *>(zprev + aidx(b, t, hc * 32 + e * 8, T));
            }
            int ok = 1;
            if (lane == 0) ok = tc::mbar_wait(&accf[a], aph, kTcWaitLimit, abort_flag);
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) {
                failed = true;
                break;
            }
            tc::fence_after_sync();
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int n0 = hc * 32 + j * 16;
                float v[16];
                tc::ld16(tmem + (uint32_t)(a * 64 + n0) + ((uint32_t)(q * 32) << 16), v);
                if (!live) continue;
                uint32_t zw[8], hw[8];
                if (!BWD) {
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const float x0 = v[2 * e] + bv[j * 16 + 2 * e];
                        const float x1 = v[2 * e + 1] + bv[j * 16 + 2 * e + 1];
                        zw[e] = pack2(x0, x1);
                        hw[e] = pack2(gelu(x0), gelu(x1));
                    }
                    if (out_z) {
                        *reinterpret_cast<uint4 *>(out_z + aidx(b, t, n0, T)) =
                            make_uint4(zw[0], zw[1], zw[2], zw[3]);
                        *reinterpret_cast<uint4 *>(out_z + aidx(b, t, n0 + 8, T)) =
                            make_uint4(zw[4], zw[5], zw[6], zw[7]);
                    }
                } else {
                    const uint4 z0 = zq[2 * j], z1 = zq[2 * j + 1];
                    const uint32_t zr[8] = {z0.x, z0.y, z0.z, z0.w, z1.x, z1.y, z1.z, z1.w};
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const __nv_bfloat162 zz = *reinterpret_cast<const __nv_bfloat162 *>(&zr[e]);
                        hw[e] = pack2(v[2 * e] * gelu_grad(__low2float(zz)),
                                      v[2 * e + 1] * gelu_grad(__high2float(zz)));
                    }
                }
                *reinterpret_cast<uint4 *>(out + aidx(b, t, n0, T)) =
                    make_uint4(hw[0], hw[1], hw[2], hw[3]);
                *reinterpret_cast<uint4 *>(out + aidx(b, t, n0 + 8, T)) =
                    make_uint4(hw[4], hw[5], hw[6], hw[7]);
            }
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&acce[a]);
        }
    }
    if (failed) {
        *abort_flag = 1;
        atomicExch(err, 1);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 1) tc::tmem_dealloc(tmem, 128);
}

template <bool BWD>
int launch_conv_tc(const CUtensorMap &in_map, const bf16 *Wk, const float *bias,
                   const bf16 *zprev, bf16 *out_z, bf16 *out, int B, int T, int grid, int *err,
                   cudaStream_t st)
{
    conv_tc_kernel<BWD><<<grid, kTcThreads, kTcSmem, st>>>(in_map, Wk, bias, zprev, out_z, out, B,
                                                           T, err);
    DTWGB_CUDA(cudaGetLastError());
    return DTW_OK;
}

// ------------------------------------------- weight gradients, tcgen05 / TMEM
//
// dW[k][o][i] = sum_{b,t} dz[b][t][o] * h[b][t + k - 3][i] for the two 64-channel
// convolutions.  Per item (128 time steps of one series) and per K-step of 16
// time steps, four MMAs of M = 128 x N = 64 x K = 16, one per tap pair
// (k0, k0 + 1), k0 in {0, 2, 4, 6}:
//   D_p[(d, i)][o] += sum_t h[t + k0 + d - 3][i] * dz[t][o]      (d in {0, 1})
// Both operands are MN-major and read straight from the time-major tiles: the
// 16-byte rows run along the channels, consecutive rows along time (K).  The h
// tile is staged twice, the second copy one step later, as the M-halves d = 0
// and d = 1; tap pair k0 is a view k0 rows lower.  The four accumulators (256
// TMEM columns) sum over all of the CTA's items; the epilogue writes the CTA's
// partial dW (tap 7 of the last pair is discarded).  Warp 0 stages every tile
// with three tensor-map copies (h at t0 - 3 and t0 - 2, dz at t0, each the 8
// channel groups of one series; rows outside [0, T) arrive as zeros) into a
// 2-stage ring, warp 1 issues the MMAs, warps 2-5 read the accumulators at the
// end.  (With one bulk copy per channel-group column, 24 small copies per
// item, the copies and not the MMAs or the bandwidth bounded the kernel: 45
// against 25 us for S = 633, T = 256.)  Shared memory per stage:
//   h   16 column blocks (8 channel groups x 2 copies) x [136 rows][16 B]  34,816 B
//   dz   8 column blocks x [128 rows][16 B]                                  16,384 B
constexpr int kWgRows = 128;
constexpr int kWgStages = 2;  // 2 x 50 KB: fits beside one convolution CTA (108 KB)
constexpr uint32_t kWgLbH = 136 * 16, kWgLbZ = kWgRows * 16;
constexpr uint32_t kWgHBytes = 16 * kWgLbH, kWgZBytes = 8 * kWgLbZ;
constexpr uint32_t kWgStage = kWgHBytes + kWgZBytes;
constexpr int kWgThreads = 32 * 6;  // producer (warp 0), MMA issuer (warp 1), epilogue (2-5)
constexpr size_t kWgSmem = kWgStages * kWgStage + 128 + 1024;

__global__ void __launch_bounds__(kWgThreads, 1)
    wgrad_tc_kernel(const __grid_constant__ CUtensorMap h_map,
                    const __grid_constant__ CUtensorMap dz_map, int B, int T,
                    float *__restrict__ part, int *__restrict__ err)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *full = reinterpret_cast<uint64_t *>(base + kWgStages * kWgStage);
    uint64_t *empty = full + kWgStages;
    uint64_t *done = empty + kWgStages;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(done + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tslot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int q = 0; q < kWgStages; ++q) {
            tc::mbar_init(&full[q], 1);
            tc::mbar_init(&empty[q], 1);
        }
        tc::mbar_init(done, 1);
        *abort_flag = 0;
    }
    if (warp == 1) tc::tmem_alloc(tslot, 256);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    const int tiles = (T + kWgRows - 1) / kWgRows;
    const int64_t nitems = (int64_t)B * tiles;
    bool failed = false;

    if (warp == 0) {
        int i = 0;
        for (int64_t item = blockIdx.x; item < nitems; item += gridDim.x, ++i) {
            const int st = i % kWgStages;
            const uint32_t ph = (uint32_t)(i / kWgStages) & 1u;
            int ok = 1;
            if (lane == 0) ok = tc::mbar_wait(&empty[st], ph ^ 1u, kTcWaitLimit, abort_flag);
            if (!__shfl_sync(0xffffffffu, ok, 0)) {
                failed = true;
                break;
            }
            const int64_t b = item / tiles;
            const int t0 = (int)(item % tiles) * kWgRows;
            unsigned char *sh = base + st * kWgStage, *sz = sh + kWgHBytes;
            // h copies: block cp * 8 + g holds h[t0 - 3 + cp + r]; dz: block g holds dz[t0 + r]
            if (lane == 0) {
                tc::mbar_expect_tx(&full[st], kWgStage);
                tc::tensor_load_3d(sh, &h_map, 0, t0 - 3, (int)(b * 8), &full[st]);
                tc::tensor_load_3d(sh + 8 * kWgLbH, &h_map, 0, t0 - 2, (int)(b * 8), &full[st]);
                tc::tensor_load_3d(sz, &dz_map, 0, t0, (int)(b * 8), &full[st]);
            }
            __syncwarp();
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = tc::idesc_bf16_f32_mn(128, 64, true, true);
            int i = 0;
            for (int64_t item = blockIdx.x; item < nitems; item += gridDim.x, ++i) {
                const int st = i % kWgStages;
                const uint32_t ph = (uint32_t)(i / kWgStages) & 1u;
                if (!tc::mbar_wait(&full[st], ph, kTcWaitLimit, abort_flag)) {
                    failed = true;
                    break;
                }
                tc::fence_after_sync();
                const uint32_t hb = tc::smem_addr(base + st * kWgStage), zb = hb + kWgHBytes;
#pragma unroll 1
                for (int s16 = 0; s16 < kWgRows / 16; ++s16) {
                    const uint64_t bd = tc::desc_mnmajor(zb + s16 * 256, kWgLbZ, 128);
#pragma unroll
                    for (int p = 0; p < 4; ++p) {
                        const uint64_t ad =
                            tc::desc_mnmajor(hb + (uint32_t)(2 * p + s16 * 16) * 16, kWgLbH, 128);
                        tc::mma_bf16(tmem + (uint32_t)(p * 64), ad, bd, idesc, (i | s16) != 0);
                    }
                }
                tc::commit(&empty[st]);
            }
            tc::commit(done);
        }
    }
    if (warp >= 2 && !failed) {
        // epilogue: warp w reads lanes 32 (w % 4) .. : row m = (d, i), d = m / 64
        const int q = warp & 3, m = q * 32 + lane, d = m >> 6, ic = m & 63;
        int ok = 1;
        if (nitems > blockIdx.x) {
            if (lane == 0) ok = tc::mbar_wait(done, 0, kTcWaitLimit, abort_flag);
            ok = __shfl_sync(0xffffffffu, ok, 0);
        }
        if (!ok) {
            failed = true;
        } else {
            tc::fence_after_sync();
            float *dst = part + (int64_t)blockIdx.x * KW * 4096;
#pragma unroll 1
            for (int p = 0; p < 4; ++p) {
                const int k = 2 * p + d;
#pragma unroll 1
                for (int j = 0; j < 4; ++j) {
                    float v[16];
                    tc::ld16(tmem + (uint32_t)(p * 64 + j * 16) + ((uint32_t)(q * 32) << 16), v);
                    if (k < KW) {
#pragma unroll
                        for (int e = 0; e < 16; ++e)
                            dst[(k * 64 + j * 16 + e) * 64 + ic] =
                                nitems > blockIdx.x ? v[e] : 0.f;  // [k][o][i]
                    }
                }
            }
        }
    }
    if (failed) {
        *abort_flag = 1;
        atomicExch(err, 1);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 1) tc::tmem_dealloc(tmem, 256);
}

// grad[i] = sum over chunks of part[chunk][i], i < n, in a fixed order: block of
// 1024 threads = 32 outputs x 32 chunk partitions; partition q adds chunks
// q, q + 32, ... in order (four loads in flight), then the 32 partitions are
// added in order.  32 partitions keep the load chains short when there are
// many chunks (the first layer's tile partials, the bias sums over series).
constexpr int kRedParts = 32;
__global__ void __launch_bounds__(32 * kRedParts)
    chunk_reduce_kernel(const float *__restrict__ part, int chunks, int n, float *__restrict__ grad)
{
    __shared__ float sh[kRedParts][33];
    const int o = threadIdx.x & 31, q = threadIdx.x >> 5, i = blockIdx.x * 32 + o;
    float s = 0.f;
    if (i < n) {
        int c = q;
        for (; c + 3 * kRedParts < chunks; c += 4 * kRedParts) {
            const float a0 = part[(int64_t)c * n + i];
            const float a1 = part[(int64_t)(c + kRedParts) * n + i];
            const float a2 = part[(int64_t)(c + 2 * kRedParts) * n + i];
            const float a3 = part[(int64_t)(c + 3 * kRedParts) * n + i];
            s = (((s + a0) + a1) + a2) + a3;
        }
        for (; c < chunks; c += kRedParts) s += part[(int64_t)c * n + i];
    }
    sh[q][o] = s;
    __syncthreads();
    if (q == 0 && i < n) {
        float t = 0.f;
        for (int p = 0; p < kRedParts; ++p) t += sh[p][o];
        grad[i] = t;
    }
}


// partial channel sums of dz over one series: part[b][c] (fixed order: per
// thread over its rows, then the 32 lanes by shuffles, then the warps in order)
__global__ void colsum_kernel(const bf16 *__restrict__ dz, int T, float *__restrict__ part)
{
    __shared__ float sh[8][8][8];  // [group][warp][channel]
    const int b = blockIdx.x, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int g = 0; g < 8; ++g) {
        const uint4 *col = reinterpret_cast<const uint4 *>(dz + ((int64_t)b * 8 + g) * T * 8);
        float acc[8] = {};
        for (int t = threadIdx.x; t < T; t += 256) {
            const uint4 q = col[t];
            const uint32_t u[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const __nv_bfloat162 v = *reinterpret_cast<const __nv_bfloat162 *>(&u[e]);
                acc[2 * e] += __low2float(v);
                acc[2 * e + 1] += __high2float(v);
            }
        }
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            for (int o = 16; o > 0; o >>= 1) acc[e] += __shfl_xor_sync(0xffffffffu, acc[e], o);
            if (lane == 0) sh[g][w][e] = acc[e];
        }
    }
    __syncthreads();
    if (threadIdx.x < 64) {
        const int g = threadIdx.x >> 3, e = threadIdx.x & 7;
        float t = 0.f;
        for (int q = 0; q < 8; ++q) t += sh[g][q][e];
        part[(int64_t)b * 64 + threadIdx.x] = t;
    }
}

// ------------------------------------------------------- pooling, linear

// g[b][c] = mean_t h3[b][t][c]; e[b][o] = bl[o] + sum_c Wl[o][c] g[b][c].
// Block per series, warp w sums channel group w over time (16-byte rows).
__global__ void gap_linear_kernel(const bf16 *__restrict__ h3, const float *__restrict__ Wl,
                                  const float *__restrict__ bl, int T, float *__restrict__ gout,
                                  float *__restrict__ e)
{
    __shared__ float gs[64];
    __shared__ float wl[64][65];  // Wl[o][c], read coalesced
    const int b = blockIdx.x, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < 4096; i += blockDim.x) wl[i >> 6][i & 63] = Wl[i];
    const uint4 *col = reinterpret_cast<const uint4 *>(h3 + ((int64_t)b * 8 + w) * T * 8);
    float acc[8] = {};
#pragma unroll 8
    for (int t = lane; t < T; t += 32) {
        const uint4 q = col[t];
        const uint32_t u[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const __nv_bfloat162 v = *reinterpret_cast<const __nv_bfloat162 *>(&u[k]);
            acc[2 * k] += __low2float(v);
            acc[2 * k + 1] += __high2float(v);
        }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
        if (lane == 0) {
            const float gv = acc[k] / (float)T;
            gs[w * 8 + k] = gv;
            if (gout) gout[b * 64 + w * 8 + k] = gv;
        }
    }
    __syncthreads();
    if (threadIdx.x < 64) {
        const int c = threadIdx.x;
        float a2 = bl[c];
        for (int i = 0; i < 64; ++i) a2 = fmaf(wl[c][i], gs[i], a2);
        e[b * 64 + c] = a2;
    }
}

// Q[a][b] = 2 (d_ab - s_ab) / (P max(d_ab, 1e-12)), loss partial per block;
// one block of 256 threads per 32 x 32 tile of (a, b), both embedding tiles in
// shared memory; thread (ty, tx) takes a in {a0 + ty, a0 + ty + 16} and b in
// {b0 + tx, b0 + tx + 16}
constexpr int kPT = 32;
__global__ void pair_stats_kernel(const float *__restrict__ e, const float *__restrict__ target,
                                  int S, float *__restrict__ Q, float *__restrict__ lpart)
{
    __shared__ float ea[kPT][65], eb[kPT][65];
    __shared__ float sh[256];
    const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
    const int a0 = blockIdx.y * kPT, b0 = blockIdx.x * kPT;
    for (int i = threadIdx.x; i < kPT * 64; i += 256) {
        const int r = i >> 6, o = i & 63;
        ea[r][o] = a0 + r < S ? e[(a0 + r) * 64 + o] : 0.f;
        eb[r][o] = b0 + r < S ? e[(b0 + r) * 64 + o] : 0.f;
    }
    __syncthreads();
    const float P = 0.5f * (float)S * (float)(S - 1);
    float d2[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
    for (int o = 0; o < 64; ++o) {
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
            for (int v = 0; v < 2; ++v) {
                const float df = ea[ty + 16 * u][o] - eb[tx + 16 * v][o];
                d2[u][v] = fmaf(df, df, d2[u][v]);
            }
    }
    float l = 0.f;
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int v = 0; v < 2; ++v) {
            const int a = a0 + ty + 16 * u, b = b0 + tx + 16 * v;
            if (a < S && b < S) {
                float q = 0.f;
                if (a != b) {
                    const float d = sqrtf(d2[u][v]);
                    const float r = d - target[(int64_t)a * S + b];
                    q = 2.f * r / (P * fmaxf(d, 1e-12f));
                    if (a < b) l += r * r / P;
                }
                Q[(int64_t)a * S + b] = q;
            }
        }
    sh[threadIdx.x] = l;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) lpart[blockIdx.y * gridDim.x + blockIdx.x] = sh[0];
}

// fixed-order sum of the loss partials (strided per thread, then a tree)
__global__ void loss_reduce_kernel(const float *__restrict__ lpart, int n, float *__restrict__ loss,
                                   int *__restrict__ call_step)
{
    __shared__ float sh[256];
    float s = 0.f;
    for (int i = threadIdx.x; i < n; i += 256) s += lpart[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) loss[*call_step] = sh[0];
}

// dE[a][o] = sum_b Q[a][b] (e[a][o] - e[b][o]): two series per block of 512 threads
// (one resident wave at S = 633), per series 64 outputs x 4 partitions of b
// (b = part, part + 4, ... in order, sixteen loads in flight), the partitions
// combined in a fixed tree
__global__ void __launch_bounds__(512)
    embed_grad_kernel(const float *__restrict__ e, const float *__restrict__ Q, int S,
                      float *__restrict__ dE)
{
    __shared__ float sh[2][4][64];
    const int h = threadIdx.x >> 8, a = blockIdx.x * 2 + h;
    const int o = threadIdx.x & 63, part = (threadIdx.x >> 6) & 3;
    float acc = 0.f;
    if (a < S) {
        const float ea = e[a * 64 + o];
        const float *q = Q + (int64_t)a * S;
        int b = part;
        for (; b + 60 < S; b += 64) {
            float qv[16], ev[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                qv[u] = q[b + 4 * u];
                ev[u] = e[(b + 4 * u) * 64 + o];
            }
#pragma unroll
            for (int u = 0; u < 16; ++u) acc = fmaf(qv[u], ea - ev[u], acc);
        }
        for (; b < S; b += 4) acc = fmaf(q[b], ea - e[b * 64 + o], acc);
    }
    sh[h][part][o] = acc;
    __syncthreads();
    if (part == 0 && a < S)
        dE[a * 64 + o] = (sh[h][0][o] + sh[h][1][o]) + (sh[h][2][o] + sh[h][3][o]);
}

// The head's backward for series a = blockIdx.x, from dE:
//   dg[c]        = sum_o Wl[o][c] dE[a][o] / T
//   dz3[a][t][c] = dg[c] GELU'(z3[a][t][c])              (bf16)
//   cpart[a][c]  = sum_t dz3[a][t][c]                     (the stored bf16 values)
// The channel sums: per thread over its steps t = tid, tid + 128, ... in order,
// then over the threads in order (from shared memory, one thread per channel).
constexpr int kHbThreads = 128;
__global__ void __launch_bounds__(kHbThreads)
    head_bwd_kernel(const float *__restrict__ dE, const float *__restrict__ Wl,
                    const bf16 *__restrict__ z3, int T, bf16 *__restrict__ dz3,
                    float *__restrict__ cpart)
{
    __shared__ float de[64], dgs[64];
    __shared__ float red[kHbThreads][65];
    const int a = blockIdx.x;
    if (threadIdx.x < 64) de[threadIdx.x] = dE[a * 64 + threadIdx.x];
    __syncthreads();
    if (threadIdx.x < 64) {
        const int c = threadIdx.x;
        float dg = 0.f;
        for (int o = 0; o < 64; ++o) dg = fmaf(Wl[o * 64 + c], de[o], dg);
        dgs[c] = dg / (float)T;
    }
    __syncthreads();
    for (int g = 0; g < 8; ++g) {
        float v[8] = {};
        for (int t = threadIdx.x; t < T; t += kHbThreads) {
            const int64_t i = aidx(a, t, g * 8, T);
            const uint4 q = *reinterpret_cast<const uint4 *>(z3 + i);
            const uint32_t zi[4] = {q.x, q.y, q.z, q.w};
            uint32_t o[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const __nv_bfloat162 x = *reinterpret_cast<const __nv_bfloat162 *>(&zi[k]);
                o[k] = pack2(dgs[g * 8 + 2 * k] * gelu_grad(__low2float(x)),
                             dgs[g * 8 + 2 * k + 1] * gelu_grad(__high2float(x)));
                const __nv_bfloat162 y = *reinterpret_cast<const __nv_bfloat162 *>(&o[k]);
                v[2 * k] += __low2float(y);
                v[2 * k + 1] += __high2float(y);
            }
            *reinterpret_cast<uint4 *>(dz3 + i) = make_uint4(o[0], o[1], o[2], o[3]);
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) red[threadIdx.x][g * 8 + k] = v[k];
    }
    __syncthreads();
    if (threadIdx.x < 64) {
        float t = 0.f;
        for (int q = 0; q < kHbThreads; ++q) t += red[q][threadIdx.x];
        cpart[(int64_t)a * 64 + threadIdx.x] = t;
    }
}

// dWl[o][c] = sum_b dE[b][o] g[b][c]; dbl[o] = sum_b dE[b][o]; 8 partitions of b, in order
__global__ void linear_wgrad_kernel(const float *__restrict__ dE, const float *__restrict__ gin,
                                    int S, float *__restrict__ grad)
{
    __shared__ float sw[8][64], sb[8][64];
    const int o = blockIdx.x, c = threadIdx.x & 63, part = threadIdx.x >> 6;
    float s = 0.f, sbias = 0.f;
    for (int b = part; b < S; b += 8) {
        const float d = dE[b * 64 + o];
        s = fmaf(d, gin[b * 64 + c], s);
        sbias += d;
    }
    sw[part][c] = s;
    sb[part][c] = sbias;
    __syncthreads();
    if (part == 0) {
        float tw = 0.f, tb = 0.f;
        for (int q = 0; q < 8; ++q) {
            tw += sw[q][c];
            tb += sb[q][c];
        }
        grad[OFF_WL + o * 64 + c] = tw;
        if (c == 0) grad[OFF_BL + o] = tb;
    }
}

// ---------------------------------------------------------------- Adam

__global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ g,
                            float *__restrict__ m, float *__restrict__ v, const float *lr,
                            const int *step)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NPAR) return;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const int t = *step + 1;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / (1.f - powf(b1, (float)t)), vh = vi / (1.f - powf(b2, (float)t));
    p[i] -= *lr * mh / (sqrtf(vh) + eps);
}

__global__ void step_kernel(int *step, int *call_step)
{
    if (threadIdx.x == 0) {
        *step += 1;
        *call_step += 1;
    }
}

// bfloat16 copies of the weights for the forward/backward kernels:
// W1q, Wlq: float holding bf16-rounded values; W2/W3 [k][o][i] and the
// transposed [k][i][o]
__global__ void refresh_kernel(const float *__restrict__ p, float *__restrict__ W1q,
                               float *__restrict__ Wlq, bf16 *__restrict__ W2, bf16 *__restrict__ W2t,
                               bf16 *__restrict__ W3, bf16 *__restrict__ W3t)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 448) W1q[i] = bfr(p[OFF_W1 + i]);
    if (i < 4096) Wlq[i] = bfr(p[OFF_WL + i]);
    if (i < KW * 4096) {
        const int k = i / 4096, o = (i / 64) % 64, ii = i % 64;
        const bf16 w2 = __float2bfloat16_rn(p[OFF_W2 + i]), w3 = __float2bfloat16_rn(p[OFF_W3 + i]);
        // tiled for the tensor-core convolution: tap k, channel group g, row n, 8 channels
        W2[k * 4096 + (ii >> 3) * 512 + o * 8 + (ii & 7)] = w2;
        W3[k * 4096 + (ii >> 3) * 512 + o * 8 + (ii & 7)] = w3;
        W2t[k * 4096 + (o >> 3) * 512 + ii * 8 + (o & 7)] = w2;
        W3t[k * 4096 + (o >> 3) * 512 + ii * 8 + (o & 7)] = w3;
    }
}

// splitmix64 output number c (c >= 1) of the stream started at `seed`
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t c)
{
    uint64_t z = seed + c * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// He-style initialisation: parameter i = std_i * z_i, z_i standard normal by
// Box-Muller from outputs 2i+1 and 2i+2 of the splitmix64 stream of `seed`;
// std sqrt(2/7) (W1), sqrt(2/448) (W2, W3), sqrt(1/64) (Wl), biases zero.
__global__ void init_params_kernel(float *__restrict__ P, uint64_t seed)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NPAR) return;
    float sd;
    if (i < OFF_B1) sd = sqrtf(2.f / 7.f);
    else if (i < OFF_W2) sd = 0.f;
    else if (i < OFF_B2) sd = sqrtf(2.f / 448.f);
    else if (i < OFF_W3) sd = 0.f;
    else if (i < OFF_B3) sd = sqrtf(2.f / 448.f);
    else if (i < OFF_WL) sd = 0.f;
    else if (i < OFF_BL) sd = 0.125f;
    else sd = 0.f;
    const double u1 = (double)((splitmix64_at(seed, 2ull * i + 1) >> 11) + 1) * (1.0 / 9007199254740992.0);
    const double u2 = (double)(splitmix64_at(seed, 2ull * i + 2) >> 11) * (1.0 / 9007199254740992.0);
    const double z = sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
    P[i] = sd * (float)z;
}

// targets[a][b] = sqrt(D[a][b]) / mean over a != b of sqrt(D[a][b]); zero diagonal
__global__ void sqrt_sum_kernel(const float *__restrict__ D, int S, double *__restrict__ part)
{
    __shared__ double sh[256];
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < (int64_t)S * S;
         i += (int64_t)gridDim.x * 256)
        if (i / S != i % S) acc += sqrt((double)D[i]);
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void targets_kernel(const float *__restrict__ D, int S, const double *__restrict__ part,
                               int nparts, float *__restrict__ tgt)
{
    double tot = 0.0;
    for (int q = 0; q < nparts; ++q) tot += part[q];
    const double mean = tot / ((double)S * (double)(S - 1));
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (int64_t)S * S;
         i += (int64_t)gridDim.x * blockDim.x)
        tgt[i] = (i / S == i % S) ? 0.f : (float)(sqrt((double)D[i]) / mean);
}

template <typename T>
int dalloc(T **p, size_t n)
{
    if (cudaMalloc(p, sizeof(T) * (n ? n : 1)) != cudaSuccess) {
        *p = nullptr;
        set_error("encoder: device allocation of %zu bytes failed", sizeof(T) * n);
        return DTW_ENOMEM;
    }
    return DTW_OK;
}

}  // namespace
}  // namespace dtwgb

using namespace dtwgb;

struct dtw_encoder {
    int T = 0, max_batch = 0;
    // parameters, Adam state, gradients (float32) and bf16 working copies
    float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
    float *W1q = nullptr, *Wlq = nullptr;
    bf16 *W2 = nullptr, *W2t = nullptr, *W3 = nullptr, *W3t = nullptr;
    int *step = nullptr, *call_step = nullptr;
    int *tc_err = nullptr;  // set by a tensor-core kernel whose completion wait gave up
    // inference buffers (max_batch series)
    bf16 *ha = nullptr, *hb = nullptr;
    // tensor maps of the activations the tensor-core kernels stage: convolution
    // inputs (136-row boxes: a 128-step tile with its halo) and the weight
    // gradients' dz (128-row boxes)
    CUtensorMap m_ha{}, m_hb{}, m_h1{}, m_h2{}, m_dz3{}, m_dz2{}, m_dz3w{}, m_dz2w{};
    float *emb_g = nullptr;
    // training buffers (grown to the largest S seen)
    int S_cap = 0;
    bf16 *z1 = nullptr, *h1 = nullptr, *z2 = nullptr, *h2 = nullptr, *z3 = nullptr, *h3 = nullptr;
    bf16 *dz3 = nullptr, *dz2 = nullptr, *dz1 = nullptr;
    float *gv = nullptr, *e = nullptr, *dE = nullptr, *Q = nullptr, *lpart = nullptr;
    float *wpart = nullptr, *cpart = nullptr, *c1part = nullptr;
    // side stream for the step's independent reductions, with fork/join events
    cudaStream_t side = nullptr;
    cudaEvent_t ev_head = nullptr, ev_dz2 = nullptr, ev_join = nullptr;
    // captured training step
    cudaGraphExec_t exec = nullptr;
    const void *g_x = nullptr, *g_t = nullptr, *g_lr = nullptr, *g_loss = nullptr;
    int g_S = 0;
    int g_S_last = 0;  // S of the last training call (dtw_encoder_get_tensor)
};

namespace {

void free_train(dtw_encoder *E)
{
    for (bf16 *q : {E->z1, E->h1, E->z2, E->h2, E->z3, E->h3, E->dz3, E->dz2, E->dz1}) cudaFree(q);
    for (float *q : {E->gv, E->e, E->dE, E->Q, E->lpart, E->wpart, E->cpart, E->c1part}) cudaFree(q);
    E->z1 = E->h1 = E->z2 = E->h2 = E->z3 = E->h3 = E->dz3 = E->dz2 = E->dz1 = nullptr;
    E->gv = E->e = E->dE = E->Q = E->lpart = E->wpart = E->cpart = E->c1part = nullptr;
    E->S_cap = 0;
}


// Tensor map over a channel-group-blocked activation buffer of `nseries` series
// of T steps (element (b, t, c) at ((b * 8 + c / 8) * T + t) * 8 + c % 8):
// dimensions (8 channels, T steps, 8 * nseries channel-group columns), box
// (8, rows, 8) = `rows` steps of the 8 channel groups of one series.  Time
// coordinates outside [0, T) read zeros, which is the convolutions' padding.
int act_map(CUtensorMap *m, const bf16 *buf, int T, int nseries, int rows)
{
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q;
        void *fn = nullptr;
        DTWGB_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                    cudaEnableDefault, &q));
        if (q != cudaDriverEntryPointSuccess || !fn) {
            set_error("cuTensorMapEncodeTiled is not available from the driver");
            return DTW_ECUDA;
        }
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    const cuuint64_t dims[3] = {8, (cuuint64_t)T, (cuuint64_t)8 * (cuuint64_t)nseries};
    const cuuint64_t strides[2] = {16, (cuuint64_t)T * 16};  // bytes, dimensions 1 and 2
    const cuuint32_t box[3] = {8, (cuuint32_t)rows, 8}, estr[3] = {1, 1, 1};
    const CUresult r = encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<bf16 *>(buf), dims,
                              strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
        return DTW_ECUDA;
    }
    return DTW_OK;
}

// weight-gradient grid: one CTA per SM (each accumulates over its share of items)
int wgrad_grid()
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms < 1) sms = 1;
    }
    return sms;
}

int ensure_train(dtw_encoder *E, int S)
{
    if (S <= E->S_cap) return DTW_OK;
    if (E->exec) {
        cudaGraphExecDestroy(E->exec);
        E->exec = nullptr;
    }
    free_train(E);
    if (!E->side) {
        DTWGB_CUDA(cudaStreamCreateWithFlags(&E->side, cudaStreamNonBlocking));
        for (cudaEvent_t *ev : {&E->ev_head, &E->ev_dz2, &E->ev_join})
            DTWGB_CUDA(cudaEventCreateWithFlags(ev, cudaEventDisableTiming));
    }
    const size_t act = (size_t)S * E->T * C;
    int rc = DTW_OK;
    for (bf16 **q : {&E->z1, &E->h1, &E->z2, &E->h2, &E->z3, &E->h3, &E->dz3, &E->dz2, &E->dz1})
        if (!rc) rc = dalloc(q, act);
    if (!rc) rc = dalloc(&E->gv, (size_t)S * 64);
    if (!rc) rc = dalloc(&E->e, (size_t)S * 64);
    if (!rc) rc = dalloc(&E->dE, (size_t)S * 64);
    if (!rc) rc = dalloc(&E->Q, (size_t)S * S);
    if (!rc) rc = dalloc(&E->lpart, (size_t)((S + kPT - 1) / kPT) * ((S + kPT - 1) / kPT));
    if (!rc) rc = dalloc(&E->wpart, (size_t)wgrad_grid() * KW * 4096);
    if (!rc) rc = dalloc(&E->cpart, (size_t)S * 64);
    if (!rc) rc = dalloc(&E->c1part, (size_t)kC1Blocks * 512);
    const int T = E->T;
    if (!rc) rc = act_map(&E->m_h1, E->h1, T, S, kTcR);
    if (!rc) rc = act_map(&E->m_h2, E->h2, T, S, kTcR);
    if (!rc) rc = act_map(&E->m_dz3, E->dz3, T, S, kTcR);
    if (!rc) rc = act_map(&E->m_dz2, E->dz2, T, S, kTcR);
    if (!rc) rc = act_map(&E->m_dz3w, E->dz3, T, S, kWgRows);
    if (!rc) rc = act_map(&E->m_dz2w, E->dz2, T, S, kWgRows);
    if (rc) {
        free_train(E);
        return rc;
    }
    E->S_cap = S;
    return DTW_OK;
}

// persistent grid: resident blocks per SM (from the occupancy calculator) x SMs
int conv_grid(int B, int T)
{
    static int per_sm = 0, sms = 0;
    if (!per_sm) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, conv_tc_kernel<false>,
                                                          kTcThreads, kTcSmem) != cudaSuccess ||
            per_sm < 1)
            per_sm = 1;
    }
    const int items = B * ((T + kTcRows - 1) / kTcRows);
    const int cap = (per_sm > 2 ? per_sm : 2) * sms;  // two CTAs per SM fit by design
    return items < cap ? items : cap;
}

int set_smem_attrs(int T)
{
    static bool done = false;
    if (!done) {
        DTWGB_CUDA(cudaFuncSetAttribute(conv_tc_kernel<false>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem));
        DTWGB_CUDA(cudaFuncSetAttribute(conv_tc_kernel<true>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem));
        DTWGB_CUDA(cudaFuncSetAttribute(wgrad_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)kWgSmem));
        done = true;
    }
    (void)T;
    return DTW_OK;
}

// forward of B series through conv1..conv3 into h3 (z* stored if non-null)
// the training forward pass into the training buffers
int forward(dtw_encoder *E, const float *x, int B, cudaStream_t st)
{
    const int T = E->T;
    conv1_fwd_kernel<<<(unsigned)(B * (T / 64)), 256, 0, st>>>(x, E->W1q, E->p + OFF_B1, B, T,
                                                                E->z1, E->h1);
    const int grid = conv_grid(B, T);
    int rc = launch_conv_tc<false>(E->m_h1, E->W2, E->p + OFF_B2, nullptr, E->z2, E->h2, B, T,
                                   grid, E->tc_err, st);
    if (!rc)
        rc = launch_conv_tc<false>(E->m_h2, E->W3, E->p + OFF_B3, nullptr, E->z3, E->h3, B, T,
                                   grid, E->tc_err, st);
    return rc;
}

// one training step (forward, loss, backward, Adam, weight refresh)
int train_step(dtw_encoder *E, const float *x, int S, const float *targets, const float *lr,
               float *loss, cudaStream_t st)
{
    const int T = E->T;
    int rc = forward(E, x, S, st);
    if (rc) return rc;
    gap_linear_kernel<<<S, 256, 0, st>>>(E->h3, E->Wlq, E->p + OFF_BL, T, E->gv, E->e);
    const int pt = (S + kPT - 1) / kPT;
    pair_stats_kernel<<<dim3(pt, pt), 256, 0, st>>>(E->e, targets, S, E->Q, E->lpart);
    loss_reduce_kernel<<<1, 256, 0, st>>>(E->lpart, pt * pt, loss, E->call_step);
    // the embedding gradient, the head's backward with the channel sums of dz3; the
    // linear layer's and the biases' gradients then run on the side stream beside the
    // tensor-core kernels
    embed_grad_kernel<<<(S + 1) / 2, 512, 0, st>>>(E->e, E->Q, S, E->dE);
    head_bwd_kernel<<<S, kHbThreads, 0, st>>>(E->dE, E->Wlq, E->z3, T, E->dz3, E->cpart);
    DTWGB_CUDA(cudaEventRecord(E->ev_head, st));
    DTWGB_CUDA(cudaStreamWaitEvent(E->side, E->ev_head, 0));
    linear_wgrad_kernel<<<64, 512, 0, E->side>>>(E->dE, E->gv, S, E->g);
    chunk_reduce_kernel<<<2, 32 * kRedParts, 0, E->side>>>(E->cpart, S, 64, E->g + OFF_B3);
    const int wg = wgrad_grid();
    // weight gradients on the side stream, beside the input-gradient convolutions
    wgrad_tc_kernel<<<wg, kWgThreads, kWgSmem, E->side>>>(E->m_h2, E->m_dz3w, S, T, E->wpart,
                                                          E->tc_err);
    chunk_reduce_kernel<<<(KW * 4096 + 31) / 32, 32 * kRedParts, 0, E->side>>>(E->wpart, wg, KW * 4096,
                                                                 E->g + OFF_W3);
    // one input-gradient CTA per SM, so that a weight-gradient CTA fits beside it
    const int grid = conv_grid(S, T) < wg ? conv_grid(S, T) : wg;
    if ((rc = launch_conv_tc<true>(E->m_dz3, E->W3t, nullptr, E->z2, nullptr, E->dz2, S, T, grid,
                                   E->tc_err, st)))
        return rc;
    DTWGB_CUDA(cudaEventRecord(E->ev_dz2, st));
    DTWGB_CUDA(cudaStreamWaitEvent(E->side, E->ev_dz2, 0));
    colsum_kernel<<<S, 256, 0, E->side>>>(E->dz2, T, E->cpart);
    chunk_reduce_kernel<<<2, 32 * kRedParts, 0, E->side>>>(E->cpart, S, 64, E->g + OFF_B2);
    wgrad_tc_kernel<<<wg, kWgThreads, kWgSmem, E->side>>>(E->m_h1, E->m_dz2w, S, T, E->wpart,
                                                          E->tc_err);
    chunk_reduce_kernel<<<(KW * 4096 + 31) / 32, 32 * kRedParts, 0, E->side>>>(E->wpart, wg, KW * 4096,
                                                                 E->g + OFF_W2);
    DTWGB_CUDA(cudaEventRecord(E->ev_join, E->side));
    if ((rc = launch_conv_tc<true>(E->m_dz2, E->W2t, nullptr, E->z1, nullptr, E->dz1, S, T, grid,
                                   E->tc_err, st)))
        return rc;
    // layer 1
    const int nt = S * (T / 64);
    const int c1b = nt < kC1Blocks ? nt : kC1Blocks;
    conv1_wgrad_kernel<<<c1b, 256, 0, st>>>(E->dz1, x, S, T, E->c1part);
    chunk_reduce_kernel<<<512 / 32, 32 * kRedParts, 0, st>>>(E->c1part, c1b, 512, E->g + OFF_W1);
    // update, once the side stream's gradients are in
    DTWGB_CUDA(cudaStreamWaitEvent(st, E->ev_join, 0));
    adam_kernel<<<(NPAR + 255) / 256, 256, 0, st>>>(E->p, E->g, E->m, E->v, lr, E->step);
    step_kernel<<<1, 32, 0, st>>>(E->step, E->call_step);
    refresh_kernel<<<(KW * 4096 + 255) / 256, 256, 0, st>>>(E->p, E->W1q, E->Wlq, E->W2, E->W2t,
                                                            E->W3, E->W3t);
    DTWGB_CUDA(cudaGetLastError());
    return DTW_OK;
}

}  // namespace

extern "C" int32_t dtw_encoder_num_params(void) { return NPAR; }

extern "C" int dtw_encoder_create(int32_t T, int32_t max_batch, dtw_encoder **out)
{
    clear_error();
    if (!out) { set_error("NULL out"); return DTW_EINVAL; }
    *out = nullptr;
    if (T < 64 || T > kMaxT || T % 64) {
        set_error("T = %d must be a multiple of 64 in [64, %d]", T, kMaxT);
        return DTW_EINVAL;
    }
    if (max_batch < 2) { set_error("max_batch = %d must be >= 2", max_batch); return DTW_EINVAL; }
    dtw_encoder *E = new dtw_encoder();
    E->T = T;
    E->max_batch = max_batch;
    int rc = DTW_OK;
    for (float **q : {&E->p, &E->g, &E->m, &E->v})
        if (!rc) rc = dalloc(q, NPAR);
    if (!rc) rc = dalloc(&E->W1q, 448);
    if (!rc) rc = dalloc(&E->Wlq, 4096);
    for (bf16 **q : {&E->W2, &E->W2t, &E->W3, &E->W3t})
        if (!rc) rc = dalloc(q, KW * 4096);
    if (!rc) rc = dalloc(&E->step, 1);
    if (!rc) rc = dalloc(&E->call_step, 1);
    if (!rc) rc = dalloc(&E->tc_err, 1);
    if (!rc) rc = dalloc(&E->ha, (size_t)max_batch * T * C);
    if (!rc) rc = dalloc(&E->hb, (size_t)max_batch * T * C);
    if (!rc) rc = dalloc(&E->emb_g, (size_t)max_batch * 64);
    if (!rc) rc = act_map(&E->m_ha, E->ha, T, max_batch, kTcR);
    if (!rc) rc = act_map(&E->m_hb, E->hb, T, max_batch, kTcR);
    if (!rc) rc = set_smem_attrs(T);
    if (rc) {
        dtw_encoder_destroy(E);
        return rc;
    }
    for (float *q : {E->p, E->g, E->m, E->v}) cudaMemset(q, 0, sizeof(float) * NPAR);
    cudaMemset(E->step, 0, sizeof(int));
    cudaMemset(E->tc_err, 0, sizeof(int));
    refresh_kernel<<<(KW * 4096 + 255) / 256, 256>>>(E->p, E->W1q, E->Wlq, E->W2, E->W2t, E->W3,
                                                     E->W3t);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        dtw_encoder_destroy(E);
        return cuda_fail(e, "encoder init");
    }
    *out = E;
    return DTW_OK;
}

extern "C" int dtw_encoder_set_params(dtw_encoder *E, const float *host_params)
{
    clear_error();
    if (!E || !host_params) { set_error("NULL argument"); return DTW_EINVAL; }
    DTWGB_CUDA(cudaMemcpy(E->p, host_params, sizeof(float) * NPAR, cudaMemcpyHostToDevice));
    DTWGB_CUDA(cudaMemset(E->m, 0, sizeof(float) * NPAR));
    DTWGB_CUDA(cudaMemset(E->v, 0, sizeof(float) * NPAR));
    DTWGB_CUDA(cudaMemset(E->step, 0, sizeof(int)));
    refresh_kernel<<<(KW * 4096 + 255) / 256, 256>>>(E->p, E->W1q, E->Wlq, E->W2, E->W2t, E->W3,
                                                     E->W3t);
    DTWGB_CUDA(cudaDeviceSynchronize());
    return DTW_OK;
}

extern "C" int dtw_encoder_init_params(dtw_encoder *E, uint64_t seed)
{
    clear_error();
    if (!E) { set_error("NULL argument"); return DTW_EINVAL; }
    init_params_kernel<<<(NPAR + 255) / 256, 256>>>(E->p, seed);
    DTWGB_CUDA(cudaGetLastError());
    DTWGB_CUDA(cudaMemset(E->m, 0, sizeof(float) * NPAR));
    DTWGB_CUDA(cudaMemset(E->v, 0, sizeof(float) * NPAR));
    DTWGB_CUDA(cudaMemset(E->step, 0, sizeof(int)));
    refresh_kernel<<<(KW * 4096 + 255) / 256, 256>>>(E->p, E->W1q, E->Wlq, E->W2, E->W2t, E->W3,
                                                     E->W3t);
    DTWGB_CUDA(cudaDeviceSynchronize());
    return DTW_OK;
}

extern "C" int dtw_encoder_get_params(const dtw_encoder *E, float *host_params)
{
    clear_error();
    if (!E || !host_params) { set_error("NULL argument"); return DTW_EINVAL; }
    DTWGB_CUDA(cudaDeviceSynchronize());
    DTWGB_CUDA(cudaMemcpy(host_params, E->p, sizeof(float) * NPAR, cudaMemcpyDeviceToHost));
    return DTW_OK;
}

extern "C" int dtw_encoder_get_grads(const dtw_encoder *E, float *host_grads)
{
    clear_error();
    if (!E || !host_grads) { set_error("NULL argument"); return DTW_EINVAL; }
    DTWGB_CUDA(cudaDeviceSynchronize());
    DTWGB_CUDA(cudaMemcpy(host_grads, E->g, sizeof(float) * NPAR, cudaMemcpyDeviceToHost));
    return DTW_OK;
}

// The tensors of the last training step, unblocked to float32 on the host.
extern "C" int dtw_encoder_get_tensor(const dtw_encoder *E, int32_t which, float *host_out)
{
    clear_error();
    if (!E || !host_out) { set_error("NULL argument"); return DTW_EINVAL; }
    if (!E->S_cap) { set_error("no training step has run on this encoder"); return DTW_EINVAL; }
    const int S = E->g_S_last, T = E->T;
    const float *vec = nullptr;
    const bf16 *act = nullptr;
    switch (which) {
    case DTW_ENC_Z1: act = E->z1; break;
    case DTW_ENC_H1: act = E->h1; break;
    case DTW_ENC_Z2: act = E->z2; break;
    case DTW_ENC_H2: act = E->h2; break;
    case DTW_ENC_Z3: act = E->z3; break;
    case DTW_ENC_H3: act = E->h3; break;
    case DTW_ENC_DZ3: act = E->dz3; break;
    case DTW_ENC_DZ2: act = E->dz2; break;
    case DTW_ENC_DZ1: act = E->dz1; break;
    case DTW_ENC_E: vec = E->e; break;
    case DTW_ENC_DE: vec = E->dE; break;
    default: set_error("unknown tensor %d", which); return DTW_EINVAL;
    }
    DTWGB_CUDA(cudaDeviceSynchronize());
    if (vec) {
        DTWGB_CUDA(cudaMemcpy(host_out, vec, sizeof(float) * (size_t)S * 64, cudaMemcpyDeviceToHost));
        return DTW_OK;
    }
    const size_t n = (size_t)S * T * C;
    std::vector<uint16_t> raw(n);
    DTWGB_CUDA(cudaMemcpy(raw.data(), act, sizeof(uint16_t) * n, cudaMemcpyDeviceToHost));
    // blocked (b, c / 8, t, c % 8) -> (b, t, c); a bfloat16 is the top half of a float32
    for (int64_t b = 0; b < S; ++b)
        for (int g = 0; g < 8; ++g)
            for (int t = 0; t < T; ++t)
                for (int e = 0; e < 8; ++e) {
                    const uint32_t bits = (uint32_t)raw[((b * 8 + g) * T + t) * 8 + e] << 16;
                    std::memcpy(host_out + (b * T + t) * C + g * 8 + e, &bits, sizeof(float));
                }
    return DTW_OK;
}

extern "C" int dtw_encoder_embed(dtw_encoder *E, const float *x, int32_t B, float *emb, void *stream)
{
    clear_error();
    if (!E || !x || !emb) { set_error("NULL argument"); return DTW_EINVAL; }
    if (B < 1 || B > E->max_batch) { set_error("B = %d outside [1, %d]", B, E->max_batch); return DTW_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    // ha -> hb -> ha ping-pong: conv1 into ha, conv2 into hb, conv3 into ha
    const int T = E->T;
    conv1_fwd_kernel<<<(unsigned)(B * (T / 64)), 256, 0, st>>>(x, E->W1q, E->p + OFF_B1, B, T,
                                                                nullptr, E->ha);
    const int grid = conv_grid(B, T);
    int rc = launch_conv_tc<false>(E->m_ha, E->W2, E->p + OFF_B2, nullptr, nullptr, E->hb, B, T,
                                   grid, E->tc_err, st);
    if (!rc)
        rc = launch_conv_tc<false>(E->m_hb, E->W3, E->p + OFF_B3, nullptr, nullptr, E->ha, B, T,
                                   grid, E->tc_err, st);
    if (rc) return rc;
    gap_linear_kernel<<<B, 256, 0, st>>>(E->ha, E->Wlq, E->p + OFF_BL, T, nullptr, emb);
    DTWGB_CUDA(cudaGetLastError());
    return DTW_OK;
}

extern "C" int dtw_encoder_train(dtw_encoder *E, const float *x, int32_t S, const float *targets,
                                 const float *lr_dev, int32_t steps, float *loss_dev,
                                 int32_t use_graph, void *stream)
{
    clear_error();
    if (!E || !x || !targets || !lr_dev || !loss_dev) { set_error("NULL argument"); return DTW_EINVAL; }
    if (S < 2 || S > E->max_batch) { set_error("S = %d outside [2, %d]", S, E->max_batch); return DTW_EINVAL; }
    if (steps < 1) { set_error("steps = %d must be >= 1", steps); return DTW_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    int rc = ensure_train(E, S);
    if (rc) return rc;
    E->g_S_last = S;
    DTWGB_CUDA(cudaMemsetAsync(E->call_step, 0, sizeof(int), st));
    if (!use_graph) {
        for (int i = 0; i < steps; ++i)
            if ((rc = train_step(E, x, S, targets, lr_dev, loss_dev, st))) return rc;
        return DTW_OK;
    }
    if (E->exec && (E->g_x != x || E->g_t != targets || E->g_lr != lr_dev || E->g_loss != loss_dev ||
                    E->g_S != S)) {
        cudaGraphExecDestroy(E->exec);
        E->exec = nullptr;
    }
    if (!E->exec) {
        cudaStream_t cs;
        DTWGB_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t gph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
        if (e == cudaSuccess) rc = train_step(E, x, S, targets, lr_dev, loss_dev, cs);
        cudaError_t e2 = cudaStreamEndCapture(cs, &gph);
        cudaStreamDestroy(cs);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
        if (rc) {
            if (gph) cudaGraphDestroy(gph);
            return rc;
        }
        if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&E->exec, gph, 0);
        cudaGraphDestroy(gph);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
        E->g_x = x;
        E->g_t = targets;
        E->g_lr = lr_dev;
        E->g_loss = loss_dev;
        E->g_S = S;
    }
    for (int i = 0; i < steps; ++i) DTWGB_CUDA(cudaGraphLaunch(E->exec, st));
    return DTW_OK;
}

extern "C" int dtw_encoder_targets(const float *D, int32_t S, float *targets, void *stream)
{
    clear_error();
    if (!D || !targets) { set_error("NULL argument"); return DTW_EINVAL; }
    if (S < 2) { set_error("S = %d must be >= 2", S); return DTW_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    constexpr int kParts = 128;
    void *part = nullptr;
    int rc = scratch_alloc(&part, sizeof(double) * kParts, st);
    if (rc) return rc;
    sqrt_sum_kernel<<<kParts, 256, 0, st>>>(D, S, (double *)part);
    targets_kernel<<<256, 256, 0, st>>>(D, S, (const double *)part, kParts, targets);
    cudaError_t e = cudaGetLastError();
    scratch_free(part, st);
    if (e != cudaSuccess) return cuda_fail(e, "targets kernels");
    return DTW_OK;
}

extern "C" int dtw_encoder_check(dtw_encoder *E)
{
    clear_error();
    if (!E) { set_error("NULL argument"); return DTW_EINVAL; }
    int h = 0;
    DTWGB_CUDA(cudaDeviceSynchronize());
    DTWGB_CUDA(cudaMemcpy(&h, E->tc_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (h) {
        DTWGB_CUDA(cudaMemset(E->tc_err, 0, sizeof(int)));
        set_error("a tensor-core convolution gave up waiting for its MMAs; its outputs are invalid");
        return DTW_ETIMEOUT;
    }
    return DTW_OK;
}

extern "C" void dtw_encoder_destroy(dtw_encoder *E)
{
    if (!E) return;
    cudaDeviceSynchronize();
    if (E->exec) cudaGraphExecDestroy(E->exec);
    free_train(E);
    for (float *q : {E->p, E->g, E->m, E->v, E->W1q, E->Wlq, E->emb_g}) cudaFree(q);
    for (bf16 *q : {E->W2, E->W2t, E->W3, E->W3t, E->ha, E->hb}) cudaFree(q);
    cudaFree(E->step);
    cudaFree(E->call_step);
    cudaFree(E->tc_err);
    for (cudaEvent_t ev : {E->ev_head, E->ev_dz2, E->ev_join})
        if (ev) cudaEventDestroy(ev);
    if (E->side) cudaStreamDestroy(E->side);
    delete E;
}
