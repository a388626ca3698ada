// band1.cu -- instantiations and launchers of the one-pair-per-lane band kernel.
#include "band_kernels.cuh"

namespace dtwgb {

template <int K, int MT>
int launch_static(const BandArgs &A, cudaStream_t st)
{
    StaticSrc src{A, A.G, A.log2G};
    return launch_kernel(dtw_band_kernel<K, MT, StaticSrc>, src, A.n_pairs, A.G, st);
}

template <int K, int MT>
int launch_queue(const QueueSrc &src, cudaStream_t st)
{
    return launch_kernel(dtw_band_kernel<K, MT, QueueSrc>, src, src.n_items, src.G, st);
}

int launch_band1(const BandArgs &A, int K, int MT, cudaStream_t st)
{
    const bool full = MT != 1;
    switch (K) {
    case 4: return full ? launch_static<4, 4>(A, st) : launch_static<4, 1>(A, st);
    case 8: return full ? launch_static<8, 8>(A, st) : launch_static<8, 1>(A, st);
    case 13: return full ? launch_static<13, 13>(A, st) : launch_static<13, 1>(A, st);
    case 16: return full ? launch_static<16, 16>(A, st) : launch_static<16, 1>(A, st);
    default: set_error("internal: no band kernel for K=%d", K); return DTW_EUNSUPPORTED;
    }
}

int launch_band1_queue(const QueueSrc &src, int K, int MT, cudaStream_t st)
{
    const bool full = MT != 1;
    switch (K) {
    case 4: return full ? launch_queue<4, 4>(src, st) : launch_queue<4, 1>(src, st);
    case 8: return full ? launch_queue<8, 8>(src, st) : launch_queue<8, 1>(src, st);
    case 13: return full ? launch_queue<13, 13>(src, st) : launch_queue<13, 1>(src, st);
    case 16: return full ? launch_queue<16, 16>(src, st) : launch_queue<16, 1>(src, st);
    default: set_error("internal: no band kernel for K=%d", K); return DTW_EUNSUPPORTED;
    }
}

}  // namespace dtwgb
