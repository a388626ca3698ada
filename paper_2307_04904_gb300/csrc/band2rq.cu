// band2rq.cu -- the two-row rotated-band kernel on the work queues of a batch
// (batch.cu), in a translation unit of its own so that it compiles in parallel.
#include "band_tworow.cuh"

namespace dtwgb {

template <int H, int MT>
int launch_tworow_q(const QueueSrc &src, cudaStream_t st)
{
    return launch_kernel(dtw_tworow_kernel<H, MT, QueueSrc>, src, src.n_items, src.G, st,
                         kTwoRowThreads);
}

int launch_tworow_queue(const QueueSrc &src, int H, int MT, cudaStream_t st)
{
#define X(h, mt) \
    if (H == h && MT == mt) return launch_tworow_q<h, mt>(src, st);
    DTWGB_TWOROW_SHAPES(X)
#undef X
    set_error("internal: no two-row queue kernel for H=%d, MT=%d", H, MT);
    return DTW_EUNSUPPORTED;
}

}  // namespace dtwgb
