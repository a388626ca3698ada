// band1q.cu -- instantiations and launcher of the one-pair-per-lane band kernel on the
// work queue of the batched launch (batch.cu).
#include "band_kernels.cuh"

namespace dtwgb {

template <int K, int MT>
int launch_queue(const QueueSrc &src, cudaStream_t st)
{
    return launch_kernel(dtw_band_kernel<K, MT, QueueSrc>, src, src.n_items, src.G, st);
}

int launch_band1_queue(const QueueSrc &src, int K, int MT, cudaStream_t st)
{
#define X(k, mt) \
    if (K == k && MT == mt) return launch_queue<k, mt>(src, st);
    DTWGB_BAND_SHAPES(X)
#undef X
    set_error("internal: no band kernel for K=%d, MT=%d", K, MT);
    return DTW_EUNSUPPORTED;
}

}  // namespace dtwgb
