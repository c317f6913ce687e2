// Status strings, error bookkeeping and device queries of the C ABI.
#include "common.cuh"

#include <cstdio>
#include <mutex>

namespace rbffd {

static thread_local char g_last_error[256] = "no error";

void set_cuda_error(cudaError_t e) {
    const char* name = cudaGetErrorName(e);
    const char* msg = cudaGetErrorString(e);
    snprintf(g_last_error, sizeof(g_last_error), "%s: %s", name ? name : "?", msg ? msg : "?");
}

int sm_count() {
    static int cached[64];
    static std::once_flag once[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
    std::call_once(once[dev], [&] {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0)
            v = 152;
        cached[dev] = v;
    });
    return cached[dev];
}

}  // namespace rbffd

extern "C" {

const char* rbffd_status_string(int s) {
    switch (s) {
        case RBFFD_OK: return "RBFFD_OK";
        case RBFFD_ERR_INVALID_ARG: return "RBFFD_ERR_INVALID_ARG";
        case RBFFD_ERR_CUDA: return "RBFFD_ERR_CUDA";
        case RBFFD_ERR_SINGULAR_STENCIL: return "RBFFD_ERR_SINGULAR_STENCIL";
        case RBFFD_ERR_NOT_CONVERGED: return "RBFFD_ERR_NOT_CONVERGED";
        case RBFFD_ERR_BREAKDOWN: return "RBFFD_ERR_BREAKDOWN";
        case RBFFD_ERR_TIMEOUT: return "RBFFD_ERR_TIMEOUT";
        case RBFFD_ERR_WORKSPACE: return "RBFFD_ERR_WORKSPACE";
        default: return "RBFFD_UNKNOWN_STATUS";
    }
}

const char* rbffd_last_cuda_error(void) { return rbffd::g_last_error; }

int rbffd_version(void) { return 100; }

}  // extern "C"
