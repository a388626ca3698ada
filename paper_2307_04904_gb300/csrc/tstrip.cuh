// tstrip.cuh -- entry points of the transposed single-strip kernel (tstrip.cu)
// and the band edge masks it shares with the column-strip kernel (strip.cu).
#pragma once

#include "band_kernels.cuh"

namespace dtwgb {

// Transposed single strip (tstrip.cu) for pairs whose shorter series fits in
// one lane group: G = tstrip_lanes(n, K) lanes per pair (0 if n > 32 K); the
// queue's G is that of its pairs.
int launch_tstrip_queue(const QueueSrc &src, int K, cudaStream_t st);
int tstrip_lanes(int n, int K);
double cost_tstrip(int n, int m, int w, int K);

// Band edge masks in original coordinates (the strip kernels).  A lane owns
// K consecutive columns jl .. jl+K-1 and walks one row per step, so at step s
// of a block that starts on row i0 its slot t holds cell (i0 + s, jl + t),
// which lies in the band |i - j| <= w exactly when
// (unsigned)(d0 + s - t) <= 2w with d0 = i0 - jl + w.  The test depends on s
// and t only through t - s, so a block needs K + B - 1 masks, not K B: a
// window mk[t] = +0 for a cell in the band and +inf outside, set for step 0 and
// then moved one slot right per step (a register rename once unrolled) with one
// new mask entering slot 0.  Only K masks are live at a time.  A cell leaves
// the band by one addition on the FMA pipe instead of an integer test and a
// select on the ALU pipe; every cell value of a row inside the series is >= +0,
// so the sum is the select's value bit for bit.
template <int K>
__device__ __forceinline__ void edge_masks_init(const unsigned d0, const unsigned w2, float (&mk)[K])
{
#pragma unroll
    for (int t = 0; t < K; ++t) mk[t] = (d0 - (unsigned)t <= w2) ? 0.f : finf();
}

// the window of step s + 1 from that of step s
template <int K>
__device__ __forceinline__ void edge_masks_next(const unsigned d0, const unsigned w2, const int s,
                                                float (&mk)[K])
{
#pragma unroll
    for (int t = K - 1; t > 0; --t) mk[t] = mk[t - 1];
    mk[0] = (d0 + (unsigned)(s + 1) <= w2) ? 0.f : finf();
}

}  // namespace dtwgb
