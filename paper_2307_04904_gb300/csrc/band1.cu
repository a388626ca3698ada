// band1.cu -- instantiations and launcher of the one-pair-per-lane band kernel on the
// static pair stride (the work-queue instances are in band1q.cu, compiled in parallel).
#include "band_kernels.cuh"

namespace dtwgb {

template <int K, int MT>
int launch_static(const BandArgs &A, cudaStream_t st)
{
    StaticSrc src{A, A.G, A.log2G};
    return launch_kernel(dtw_band_kernel<K, MT, StaticSrc>, src, A.n_pairs, A.G, st, kThreads,
                         /*persistent=*/false);
}

int launch_band1(const BandArgs &A, int K, int MT, cudaStream_t st)
{
#define X(k, mt) \
    if (K == k && MT == mt) return launch_static<k, mt>(A, st);
    DTWGB_BAND_SHAPES(X)
#undef X
    return launch_band1_wide(A, K, MT, st);
}

}  // namespace dtwgb
