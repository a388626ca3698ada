// band3r.cu -- instantiations and launcher of the three-row rotated-band kernel
// (band_multirow.cuh) on the static pair stride.
#include "band_multirow.cuh"

namespace dtwgb {

template <int H, int MT>
int launch_threerow_static(const BandArgs &A, cudaStream_t st)
{
    StaticSrc src{A, A.G, A.log2G};
    return launch_kernel(dtw_multirow_kernel<3, H, MT, StaticSrc>, src, A.n_pairs, A.G, st,
                         kMultiRowThreads, /*persistent=*/false);
}

int launch_threerow(const BandArgs &A, int H, int MT, cudaStream_t st)
{
#define X(h, mt) \
    if (H == h && MT == mt) return launch_threerow_static<h, mt>(A, st);
    DTWGB_THREEROW_SHAPES(X)
#undef X
    set_error("internal: no three-row band kernel for H=%d, MT=%d", H, MT);
    return DTW_EUNSUPPORTED;
}

}  // namespace dtwgb
