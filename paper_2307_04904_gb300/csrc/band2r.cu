// band2r.cu -- instantiations and launcher of the two-row rotated-band kernel
// (band_tworow.cuh) on the static pair stride.
#include "band_tworow.cuh"

namespace dtwgb {

template <int H, int MT>
int launch_tworow_static(const BandArgs &A, cudaStream_t st)
{
    StaticSrc src{A, A.G, A.log2G};
    return launch_kernel(dtw_tworow_kernel<H, MT, StaticSrc>, src, A.n_pairs, A.G, st,
                         kTwoRowThreads, /*persistent=*/false);
}

int launch_tworow(const BandArgs &A, int H, int MT, cudaStream_t st)
{
#define X(h, mt) \
    if (H == h && MT == mt) return launch_tworow_static<h, mt>(A, st);
    DTWGB_TWOROW_SHAPES(X)
#undef X
    set_error("internal: no two-row band kernel for H=%d, MT=%d", H, MT);
    return DTW_EUNSUPPORTED;
}

}  // namespace dtwgb
