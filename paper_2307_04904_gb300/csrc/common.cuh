// common.cuh -- shared host/device helpers of the dtwgb library (errors,
// float primitives, triangle indexing).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>

#include "../../include/dtwgb.h"

namespace dtwgb {

// ---------------------------------------------------------------- errors

void set_error(const char *fmt, ...);
void clear_error();

// Returns DTW_ECUDA (and records the message) if `e` is an error.
int cuda_fail(cudaError_t e, const char *what);

// Stream-ordered scratch from the library's private per-device pool.
int scratch_alloc(void **p, size_t bytes, cudaStream_t st);
int scratch_free(void *p, cudaStream_t st);

#define DTWGB_CUDA(call)                                   \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return ::dtwgb::cuda_fail(e_, #call); \
    } while (0)

// ------------------------------------------------------- float primitives

__device__ __forceinline__ float finf() { return __int_as_float(0x7f800000); }

// min(a, b, c).  min is exact, so the grouping never changes the value; the
// three-input form of min.f32 (sm_100 and later) issues one instruction.
__device__ __forceinline__ float fmin3(float a, float b, float c)
{
#if defined(DTWGB_NO_MIN3)
    return fminf(fminf(a, b), c);
#else
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
#endif
}

// One DP cell: (x - y)^2 + m with d = x - y rounded to float and a single
// rounding for d*d + m (fused multiply-add).
__device__ __forceinline__ float dtw_cell(float x, float y, float m)
{
    float d = __fsub_rn(x, y);
    return __fmaf_rn(d, d, m);
}

// -------------------------------------------------------- pair indexing

// Upper-triangle index t in [0, p(p-1)/2) -> (a, b) with a < b, row-major:
// t = a*(2p-a-1)/2 + (b-a-1).  A double square root gives the row, an
// integer fix-up makes it exact.
__host__ __device__ __forceinline__ int64_t tri_row_start(int64_t a, int64_t p)
{
    return a * (2 * p - a - 1) / 2;
}

__host__ __device__ inline void tri_index(int64_t t, int64_t p, int64_t &a, int64_t &b)
{
    double q = (double)(2 * p - 1);
    double r = (q - sqrt(q * q - 8.0 * (double)t)) * 0.5;
    int64_t ai = (int64_t)r;
    if (ai < 0) ai = 0;
    if (ai > p - 2) ai = p - 2;
    while (ai > 0 && tri_row_start(ai, p) > t) --ai;
    while (ai < p - 2 && tri_row_start(ai + 1, p) <= t) ++ai;
    a = ai;
    b = t - tri_row_start(ai, p) + ai + 1;
}

}  // namespace dtwgb
