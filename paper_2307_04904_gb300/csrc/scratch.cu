// scratch.cu -- stream-ordered scratch memory for the library's own temporaries
// (padded series copies, k-medoids sums and flags).
//
// Every device gets one private cudaMemPool_t whose release threshold is
// unlimited, so memory freed at the end of a call stays mapped and the next
// call's cudaMallocFromPoolAsync is a cheap sub-allocation instead of a fresh
// mapping.  The pool never touches the device's default pool or torch's
// caching allocator.
#include <mutex>

#include "common.cuh"

namespace dtwgb {

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pools[kMaxDevices] = {};
}  // namespace

int scratch_pool(cudaMemPool_t *out)
{
    int dev = 0;
    DTWGB_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("device %d out of range", dev);
        return DTW_EUNSUPPORTED;
    }
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pools[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool;
        DTWGB_CUDA(cudaMemPoolCreate(&pool, &props));
        uint64_t keep = UINT64_MAX;
        DTWGB_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
        g_pools[dev] = pool;
    }
    *out = g_pools[dev];
    return DTW_OK;
}

int scratch_alloc(void **p, size_t bytes, cudaStream_t st)
{
    *p = nullptr;
    cudaMemPool_t pool;
    int rc = scratch_pool(&pool);
    if (rc) return rc;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMallocFromPoolAsync(p, bytes, pool, st);
    if (e != cudaSuccess) {
        *p = nullptr;
        set_error("scratch allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? DTW_ENOMEM : DTW_ECUDA;
    }
    return DTW_OK;
}

int scratch_free(void *p, cudaStream_t st)
{
    if (!p) return DTW_OK;
    DTWGB_CUDA(cudaFreeAsync(p, st));
    return DTW_OK;
}

}  // namespace dtwgb
