// band1w.cu -- the further slot counts of the one-pair-per-lane band kernel on
// the static pair stride (K = 9, 11, 14, 15, 17, 19, 21..24), in a translation
// unit of their own so that it compiles in parallel with band1.cu.
#include "band_kernels.cuh"

namespace dtwgb {

template <int K, int MT>
int launch_static_wide(const BandArgs &A, cudaStream_t st)
{
    StaticSrc src{A, A.G, A.log2G};
    return launch_kernel(dtw_band_kernel<K, MT, StaticSrc>, src, A.n_pairs, A.G, st, kThreads,
                         /*persistent=*/false);
}

int launch_band1_wide(const BandArgs &A, int K, int MT, cudaStream_t st)
{
#define X(k, mt) \
    if (K == k && MT == mt) return launch_static_wide<k, mt>(A, st);
    DTWGB_BAND_SHAPES_WIDE(X)
#undef X
    set_error("internal: no band kernel for K=%d, MT=%d", K, MT);
    return DTW_EUNSUPPORTED;
}

}  // namespace dtwgb
