// band2.cu -- instantiations and launcher of the two-pair-per-lane band kernel.
#include "band_kernels.cuh"

namespace dtwgb {

int launch_band2(const BandArgs &A, int K, int MT, cudaStream_t st)
{
    // compiled for K in {4, 8, 13, 16} with MT 1 or K (a full tail also serves a 4-slot one)
    if (K != 4 && K != 8 && K != 13 && K != 16) return launch_band1(A, K, MT, st);
    const bool full = MT != 1;
    switch (K) {
    case 4: return full ? launch_kernel(dtw_band2_kernel<4, 4>, A, A.n_pairs, A.G, st)
                   : launch_kernel(dtw_band2_kernel<4, 1>, A, A.n_pairs, A.G, st);
    case 8: return full ? launch_kernel(dtw_band2_kernel<8, 8>, A, A.n_pairs, A.G, st)
                    : launch_kernel(dtw_band2_kernel<8, 1>, A, A.n_pairs, A.G, st);
    case 13: return full ? launch_kernel(dtw_band2_kernel<13, 13>, A, A.n_pairs, A.G, st)
                    : launch_kernel(dtw_band2_kernel<13, 1>, A, A.n_pairs, A.G, st);
    case 16: return full ? launch_kernel(dtw_band2_kernel<16, 16>, A, A.n_pairs, A.G, st)
                    : launch_kernel(dtw_band2_kernel<16, 1>, A, A.n_pairs, A.G, st);
    default: set_error("internal: no band kernel for K=%d", K); return DTW_EUNSUPPORTED;
    }
}

}  // namespace dtwgb
