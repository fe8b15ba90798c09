// mbmd_objective_noalloc: the projection-domain PWLS data term computed with
// no device allocation at all.  It is for callers that cannot allocate device
// memory: code embedded in a host framework whose device memory belongs to
// another allocator (a caching allocator or a fixed pool that must not be
// bypassed), deployments held to a fixed device-memory budget, and loops that
// must not call cudaMalloc / cudaFree because those can block or implicitly
// synchronise the whole device.
//
// Its scratch (the FP32 copy of the spectral table and the per-block
// double-float partial sums) lives in the file-scope array below, 28,928 bytes, which
// every GPU that loads this library holds until the process exits.  In host
// code the array's name only stands in for the symbol and is never used as a
// pointer: the device address is looked up with cudaGetSymbolAddress on the
// first call on each device (with that device current) and handed to the
// kernels.  The call cannot be captured into a CUDA graph: it stages the
// spectral table from a stack array with a pageable copy, which a graph would
// replay from a buffer that no longer exists, so a stream that is capturing
// is rejected with MBIR_ERR_ARG before anything is enqueued.  All calls share
// the array, so calls that overlap on the GPU (different streams, or several
// host threads) race on it.
#include <mutex>

#include "model.cuh"

namespace psps {
namespace {

constexpr size_t kTableFloats = 256 * 4 + 8 * 256 + 8;  // Q[E][m], S[c][E], sigma[c] at the limits
constexpr size_t kTableBytes = ((kTableFloats * sizeof(float) + 255) / 256) * 256;
constexpr size_t kPartialBytes = sizeof(dfloat) * kModelMaxBlocks;
constexpr size_t kScratchBytes = kTableBytes + kPartialBytes;  // 28,928 bytes

static_assert(kScratchBytes == 28928, "keep the documented scratch size in step");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up on
// the first call per device).
mbir_status scratch_address(void **out) {
    int dev = 0;
    PSPS_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(MBIR_ERR_ARG, "mbmd_objective_noalloc: device %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fail(MBIR_ERR_CUDA, "mbmd_objective_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return MBIR_OK;
}

}  // namespace
}  // namespace psps

using namespace psps;

extern "C" mbir_status mbmd_objective_noalloc(int n_mat, int n_energy, int n_chan, const double *Q, const double *S,
                                              const float *l, const float *y, int64_t n_rays, double *objective,
                                              mbir_stream stream) {
    if (!Q || !S || !l || !y || !objective) return fail(MBIR_ERR_ARG, "mbmd_objective_noalloc: null argument");
    if (n_mat < 1 || n_mat > 4 || n_energy < 1 || n_energy > 256 || n_chan < 1 || n_chan > 8)
        return fail(MBIR_ERR_ARG,
                    "mbmd_objective_noalloc: n_mat=%d n_energy=%d n_chan=%d exceed the static scratch limits "
                    "(n_mat <= 4, n_energy <= 256, n_chan <= 8)",
                    n_mat, n_energy, n_chan);
    if (n_rays < 1) return fail(MBIR_ERR_ARG, "mbmd_objective_noalloc: n_rays must be >= 1");
    cudaStream_t s = (cudaStream_t)stream;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    const cudaError_t ce = cudaStreamIsCapturing(s, &cap);
    if (ce != cudaSuccess)
        return fail(MBIR_ERR_CUDA, "mbmd_objective_noalloc: cudaStreamIsCapturing: %s", cudaGetErrorString(ce));
    if (cap != cudaStreamCaptureStatusNone)
        return fail(MBIR_ERR_ARG, "mbmd_objective_noalloc: the stream is capturing a CUDA graph; this call cannot be "
                                  "captured (it stages its table with a pageable host copy)");
    const size_t nt = (size_t)n_energy * n_mat + (size_t)n_chan * n_energy + n_chan;
    float table[kTableFloats];  // host staging on the stack, no allocation
    for (size_t i = 0; i < (size_t)n_energy * n_mat; ++i) table[i] = (float)Q[i];
    for (int c = 0; c < n_chan; ++c) {
        double sig = 0.0;
        for (int e = 0; e < n_energy; ++e) {
            table[(size_t)n_energy * n_mat + (size_t)c * n_energy + e] = (float)S[(size_t)c * n_energy + e];
            sig += S[(size_t)c * n_energy + e];
        }
        table[(size_t)n_energy * n_mat + (size_t)n_chan * n_energy + c] = (float)sig;
    }
    void *base = nullptr;
    PSPS_TRY(scratch_address(&base));
    float *qs = (float *)base;
    dfloat *partials = (dfloat *)((unsigned char *)base + kTableBytes);
    // pageable source: the copy is staged before the call returns, so the
    // stack table may go out of scope afterwards
    PSPS_CUDA(cudaMemcpyAsync(qs, table, sizeof(float) * nt, cudaMemcpyHostToDevice, s));
    const SpecDev sp{n_mat, n_energy, n_chan, qs};
    const int nb = model_blocks(n_rays);  // <= kModelMaxBlocks: every block writes its own partial
    PSPS_TRY(launch_model_grad(sp, n_rays, l, y, nullptr, nullptr, nullptr, partials, nb, s));
    PSPS_TRY(reduce_partials(partials, nb, 1, objective, 0, s));
    return MBIR_OK;
}
