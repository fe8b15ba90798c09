// Error reporting and the fixed-order FP64 reduction shared by all kernels.
#include <cstdarg>
#include <cstring>

#include "common.cuh"

namespace psps {

static thread_local std::string g_last_error = "no error";

void set_error(const std::string &msg) { g_last_error = msg; }

mbir_status fail(mbir_status code, const char *fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

namespace {
// One block sums n partials of each of K streams in a fixed order.
__global__ void reduce_partials_kernel(const double *__restrict__ partials, int n, int K, double *dst, int add) {
    __shared__ double sh[32];
    for (int k = 0; k < K; ++k) {
        double a = 0.0;
        for (int i = threadIdx.x; i < n; i += blockDim.x) a += partials[(size_t)k * n + i];
        for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = a;
        __syncthreads();
        if (threadIdx.x < 32) {
            a = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
            for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
            if (threadIdx.x == 0) dst[k] = add ? dst[k] + a : a;
        }
        __syncthreads();
    }
}
}  // namespace

mbir_status reduce_partials(const double *partials, int n, int K, double *dst, int add, cudaStream_t s) {
    reduce_partials_kernel<<<1, 256, 0, s>>>(partials, n, K, dst, add);
    PSPS_LAUNCH_CHECK();
    return MBIR_OK;
}

}  // namespace psps

extern "C" const char *mbir_last_error(void) { return psps::g_last_error.c_str(); }
