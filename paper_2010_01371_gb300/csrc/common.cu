// Error reporting and the fixed-order reduction of partial sums.
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
__global__ void reduce_partials_kernel(const dfloat *__restrict__ partials, int n, int K, double *dst, int add) {
    for (int k = 0; k < K; ++k) {
        const double a = block_sum_partials(partials + (size_t)k * n, n);
        if (threadIdx.x == 0) dst[k] = add ? dst[k] + a : a;
    }
}
}  // namespace

mbir_status reduce_partials(const dfloat *partials, int n, int K, double *dst, int add, cudaStream_t s) {
    reduce_partials_kernel<<<1, 256, 0, s>>>(partials, n, K, dst, add);
    PSPS_LAUNCH_CHECK();
    return MBIR_OK;
}

}  // namespace psps

extern "C" const char *mbir_last_error(void) { return psps::g_last_error.c_str(); }
