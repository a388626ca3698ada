// abi.cu -- error reporting and version of the dtwgb C ABI.
#include "common.cuh"

namespace dtwgb {

namespace {
thread_local char g_err[512] = "";
}

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

void clear_error() { g_err[0] = '\0'; }

int cuda_fail(cudaError_t e, const char *what)
{
    set_error("%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
    return DTW_ECUDA;
}

}  // namespace dtwgb

extern "C" const char *dtw_last_error(void) { return dtwgb::g_err; }

extern "C" const char *dtw_version(void) { return "0.1.0"; }
