// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <string>

#include "../../include/mbir.h"

namespace psps {

// ----------------------------------------------------------------- errors
void set_error(const std::string &msg);
mbir_status fail(mbir_status code, const char *fmt, ...);

#define PSPS_CUDA(call)                                                                       \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            return ::psps::fail(e_ == cudaErrorMemoryAllocation ? MBIR_ERR_OOM : MBIR_ERR_CUDA, \
                                "%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e_)); \
        }                                                                                     \
    } while (0)

#define PSPS_TRY(expr)                         \
    do {                                       \
        mbir_status s_ = (expr);               \
        if (s_ != MBIR_OK) return s_;          \
    } while (0)

#define PSPS_LAUNCH_CHECK() PSPS_CUDA(cudaGetLastError())

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Device buffer owned by a handle (freed in the destructor).
template <class T>
struct DBuf {
    T *p = nullptr;
    size_t n = 0;
    DBuf() = default;
    DBuf(const DBuf &) = delete;
    DBuf &operator=(const DBuf &) = delete;
    ~DBuf() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    mbir_status alloc(size_t count) {
        release();
        if (count == 0) count = 1;
        cudaError_t e = cudaMalloc((void **)&p, count * sizeof(T));
        if (e != cudaSuccess) {
            p = nullptr;
            return fail(MBIR_ERR_OOM, "cudaMalloc(%zu bytes): %s", count * sizeof(T), cudaGetErrorString(e));
        }
        n = count;
        return MBIR_OK;
    }
    mbir_status zero(cudaStream_t s) {
        cudaError_t e = cudaMemsetAsync(p, 0, n * sizeof(T), s);
        if (e != cudaSuccess) return fail(MBIR_ERR_CUDA, "memset: %s", cudaGetErrorString(e));
        return MBIR_OK;
    }
};

// ------------------------------------------------------------- reductions
// Sums over rays and pixels are accumulated as double-floats: an unevaluated
// pair hi + lo of FP32 numbers updated with Knuth's TwoSum error-free
// transformation, which carries about twice FP32's precision with FP32
// additions only (FP64 arithmetic runs at a small fraction of the FP32 rate
// on this GPU).  Only the final few sums are converted to double.
struct dfloat {
    float hi, lo;
};

__device__ __forceinline__ void df_add(dfloat &a, float v) {
    const float s = a.hi + v;
    const float bp = s - a.hi;
    const float e = (a.hi - (s - bp)) + (v - bp);  // exact rounding error of a.hi + v
    a.hi = s;
    a.lo += e;
}

__device__ __forceinline__ void df_merge(dfloat &a, const dfloat &b) {
    df_add(a, b.hi);
    a.lo += b.lo;
}

__host__ __device__ inline double df_value(const dfloat &a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ dfloat df_shfl_down(const dfloat &a, int o) {
    return dfloat{__shfl_down_sync(0xffffffffu, a.hi, o), __shfl_down_sync(0xffffffffu, a.lo, o)};
}

// Block-level sum of K double-floats per thread (fixed order); thread 0
// writes the block's partial sums to out[k * gridDim.x + blockIdx.x].
// blockDim.x must be a multiple of 32 and <= 1024.
template <int K>
__device__ __forceinline__ void block_sum_store(dfloat (&v)[K], dfloat *out) {
    __shared__ dfloat sh[K][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        dfloat a = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) df_merge(a, df_shfl_down(a, o));
        if (lane == 0) sh[k][wid] = a;
    }
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            dfloat a = lane < nw ? sh[k][lane] : dfloat{0.f, 0.f};
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) df_merge(a, df_shfl_down(a, o));
            if (lane == 0) out[(size_t)k * gridDim.x + blockIdx.x] = a;
        }
    }
}

// Fixed-order sum of n double-float partials by one whole block (ld.cg: the
// partials may come from other blocks of the same kernel); the result is
// valid in thread 0.
__device__ inline double block_sum_partials(const dfloat *p, int n) {
    __shared__ dfloat sh[32];
    dfloat a{0.f, 0.f};
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const float2 v = __ldcg(reinterpret_cast<const float2 *>(p + i));
        df_merge(a, dfloat{v.x, v.y});
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) df_merge(a, df_shfl_down(a, o));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = a;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0) {
        dfloat t{0.f, 0.f};
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) df_merge(t, sh[w]);
        r = df_value(t);
    }
    __syncthreads();
    return r;
}

// K such sums in one pass (stream k at p + k * n), so that the block pays
// the load latency once; the results are valid in thread 0.
template <int K>
__device__ inline void block_sum_partials_k(const dfloat *p, int n, double (&out)[K]) {
    __shared__ dfloat sh[K][32];
    dfloat a[K];
#pragma unroll
    for (int k = 0; k < K; ++k) a[k] = dfloat{0.f, 0.f};
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const float2 v = __ldcg(reinterpret_cast<const float2 *>(p + (size_t)k * n + i));
            df_merge(a[k], dfloat{v.x, v.y});
        }
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) df_merge(a[k], df_shfl_down(a[k], o));
        if ((threadIdx.x & 31) == 0) sh[k][threadIdx.x >> 5] = a[k];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            dfloat t{0.f, 0.f};
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) df_merge(t, sh[k][w]);
            out[k] = df_value(t);
        }
    }
    __syncthreads();
}

// Joseph sample split shared by every forward projector and transpose
// (identical arithmetic on both sides, so each pair is an exact transpose up
// to the summation order): with h = f - 1/2 = i * df + (f0 - 1/2) and
// |h| < 2^22, h + 1.5 * 2^23 rounds to the integer nearest h, which is
// floor(f) except at integer f, where it may give floor(f) - 1 with fraction
// 1 — the same two weights on the same pixel, since the linear interpolation
// is continuous there.  Returns the lower interpolation index; f gets the
// weight of the upper one.  No conversion instructions are used.
constexpr float kSplitMagic = 12582912.0f;  // 1.5 * 2^23

__device__ __forceinline__ int joseph_split(float h, float &f) {
    const float rn = h + kSplitMagic;
    f = (h - (rn - kSplitMagic)) + 0.5f;
    return __float_as_int(rn) - __float_as_int(kSplitMagic);
}

// Sum `n` partials (fixed order, one block) into dst[0..K) (dst += if add).
mbir_status reduce_partials(const dfloat *partials, int n, int K, double *dst, int add, cudaStream_t s);

// ------------------------------------------------------------ handles
struct RayTable2D {
    // Per ray (2-D): interpolation coordinate at driving index 0, its
    // increment per driving index, weight (pixel size / |u_axis|), driving
    // axis (0 = x, 1 = y) and the conservative range of driving indices.
    float *f0 = nullptr, *df = nullptr, *w = nullptr;
    int *axis_lo_hi = nullptr;  // packed: axis | (lo << 1) | (hi << 16) [lo,hi < 32768]
};

}  // namespace psps

struct mbir_plan {
    mbir_geometry g;
    int n_mat_max = 1;
    int64_t n_rays = 0, n_pix = 0;
    // 2-D per-ray Joseph set-up
    psps::DBuf<float4> ray;       // (f0, df, w, bits(axis,lo,hi))
    // 2-D per-view constants for the pixel-driven transpose
    psps::DBuf<float4> view;      // parallel: (cos, sin, -, -); fan: (sx, sy, beta + pi, -)
    int back_mode = 0;            // 0 tile scatter (default), 1 pixel / voxel gather, 2 ray-driven atomics, 3 split-table gather (3-D)
    int back_views = 60;          // views per CTA of the tile transpose
    int fwd_mode = 1;             // 0 tile sums, 1 one thread per ray (default), 2 shared-memory strips
    int strip_bins = 64;          // strip forward: bins per CTA (32, 64, 128 or 256; 256 / it views)
    // 3-D per-ray Joseph set-up (cone_ray, computed once): (fb_mid, dfb,
    // fc_mid, dfc) in `ray` and (weight, bits(axis | lo << 2 | hi << 17)) in
    // ray3b; per view, the set of driving axes its rays use (bit a)
    psps::DBuf<float2> ray3b;
    psps::DBuf<int> view_axes;
    psps::DBuf<float> wsino;      // 3-D gather: weighted sinogram, up to 4 channels interleaved
    // scratch: packed / transposed image copies for the forward projector
    // (3-D: one copy per driving axis)
    psps::DBuf<float> xrow, xcol, xcol3;
    // 2-D tile transpose: per channel, max_i |s_i| as float bits, and the
    // largest ray weight: M = w_max max|s| bounds every |w_i s_i| and sets
    // the fixed-point scale of the shared-memory accumulators
    psps::DBuf<unsigned> wmax;
    float w_max = 0.f;
    // 2-D tile transpose: 64-bit fixed-point image sums ([n_mat_max][n_pix])
    psps::DBuf<long long> xfix;
    // bound on the rays of one view that add to one tile accumulator (0: none
    // known; 2-D: the CTA's candidate count bounds it then; 3-D: the tile
    // transpose is replaced by the direct gather)
    int cell_rays = 0;
    // 3-D tile transpose: the number of leading channels of the next calls
    // that also accumulate each term's remainder (two words per voxel: terms
    // held to 2^-12 of the fixed-point unit); set around a call by the
    // gradient numerators' callers
    int tile_fine = 0;
    // 3-D tile transpose: tile depth (16 or 8 voxels; 8 x 8 across)
    int cone_tile = 16;
};

struct mbmd_spectrum {
    int n_mat = 1, n_energy = 1, n_chan = 1;
    psps::DBuf<float> qs;   // device: Q[E][m] then S[c][E] then sigma[c]
    // optional detector blur (outer operator B S): taps b[-r..r] along rows
    // of blur_row consecutive rays; r = 0: none
    int blur_r = 0, blur_row = 1;
    float blur_b[7] = {};
    // optional correlated noise: Sigma_y = D^1/2 C D^1/2, C[j][k] = a^|j-k|
    // within rows of noise_row consecutive rays; a = 0: diagonal
    float noise_a = 0.f;
    int noise_row = 1;
    double *hQ = nullptr, *hS = nullptr;  // host FP64 copies
    ~mbmd_spectrum() {
        delete[] hQ;
        delete[] hS;
    }
};

namespace psps {
// projector internals (projector.cu)
mbir_status project(mbir_plan *p, const float *x, float *l, int n_mat, cudaStream_t s);
mbir_status backproject(mbir_plan *p, const float *sino, float *x, int n_mat, int accumulate, cudaStream_t s);
// cone-beam (cone.cu)
mbir_status cone_setup(mbir_plan *p);
// Floats of each zero-bordered packed volume copy the cone forward reads
// (4 per voxel, the largest of the three driving-axis layouts).
int64_t cone_pack_floats(const mbir_geometry &g);
mbir_status project_cone(mbir_plan *p, const float *x, float *l, int n_mat, cudaStream_t s);
mbir_status backproject_cone(mbir_plan *p, const float *sino, float *x, int n_mat, int accumulate, cudaStream_t s);
}  // namespace psps
