// Orthonormal 2-D Haar transform U_DWT (Mallat pyramid, full depth) for the
// wavelet preconditioner M = M0 U^T Lambda^-1/2 U M0 (Eq. 34), its transpose,
// and the sign-free |U| used for the separable-curvature bound.
//
// Level step on the current low-pass block (h x h): every 2x2 group
//   (a b / c d) -> LL=(a+b+c+d)/2, HL=(a-b+c-d)/2, LH=(a+b-c-d)/2, HH=(a-b-c+d)/2
// with HL stored at (i, h/2+j), LH at (h/2+i, j), HH at (h/2+i, h/2+j) and LL
// recursing in the top-left corner; |U| uses +1/2 for every tap.
//
// GPU design: the first log2(T) levels (T = min(32, n)) are local to T x T
// tiles, so one CTA per tile runs them in shared memory and writes every
// detail coefficient straight to its Mallat position (optionally pre-scaled
// by m0 on input and scaled by Lambda^-1/2 on output); one CTA then finishes
// the (n/T) x (n/T) low-pass block.  The inverse runs the same in reverse.
// Square power-of-two images only (n <= 2048).
//
// 3-D volumes [z][y][x] (cubes n^3, n a power of two <= 256): every 2x2x2
// group v[dz][dy][dx] of the current low-pass block goes to the eight outputs
//   c[sz][sy][sx] = 2^-3/2 sum (-1)^(sz dz + sy dy + sx dx) v[dz][dy][dx]
// (three in-place +/- butterflies, one per axis), stored in octant
// (sz, sy, sx) of the block; the pyramid recurses on octant (0, 0, 0).  The
// sign matrix is symmetric and, scaled, orthogonal, so the inverse step runs
// the same butterflies on the octants.  The first log2(T) levels (T =
// min(16, n)) are local to T^3 tiles in shared memory; one CTA per channel
// finishes the (n/T)^3 low-pass block.
#include "haar.cuh"

namespace psps {
namespace {

constexpr int kT = 32;
constexpr int kThreads = 256;

__device__ __forceinline__ void fwd4(float a, float b, float c, float d, bool ab, float &ll, float &hl, float &lh,
                                     float &hh) {
    if (ab) {
        ll = hl = lh = hh = 0.5f * (a + b + c + d);
    } else {
        ll = 0.5f * ((a + b) + (c + d));
        hl = 0.5f * ((a - b) + (c - d));
        lh = 0.5f * ((a + b) - (c + d));
        hh = 0.5f * ((a - b) - (c - d));
    }
}

__device__ __forceinline__ void inv4(float ll, float hl, float lh, float hh, bool ab, float &a, float &b, float &c,
                                     float &d) {
    if (ab) {
        a = b = c = d = 0.5f * (ll + hl + lh + hh);
    } else {
        a = 0.5f * ((ll + hl) + (lh + hh));
        b = 0.5f * ((ll - hl) + (lh - hh));
        c = 0.5f * ((ll + hl) - (lh + hh));
        d = 0.5f * ((ll - hl) - (lh - hh));
    }
}

// Forward over the tile levels.  grid: (n/T, n/T, channels).
__global__ void __launch_bounds__(kThreads)
    fwd_tile_kernel(int n, int T, const float *__restrict__ in, float *__restrict__ coef,
                    const float *__restrict__ pre, const float *__restrict__ scale, unsigned abs_mask) {
    __shared__ float A[kT * kT];
    const int ch = blockIdx.z;
    const bool ab = (abs_mask >> ch) & 1u;
    const int64_t nn = (int64_t)n * n;
    const float *src = in + ch * nn;
    float *dst = coef + ch * nn;
    const int ty = blockIdx.y, tx = blockIdx.x;
    for (int k = threadIdx.x; k < T * T; k += blockDim.x) {
        const int r = k / T, c = k % T;
        const int64_t gi = (int64_t)(ty * T + r) * n + tx * T + c;
        float v = src[gi];
        if (pre) v *= pre[gi];
        A[r * T + c] = v;
    }
    __syncthreads();
    int h = T, Ng = n;
    while (h >= 2) {
        const int h2 = h / 2, N2 = Ng / 2;
        float ll[4];
        int cnt = 0;
        // each thread handles up to 4 groups (h2*h2 <= 256 when T = 32)
        for (int g = threadIdx.x; g < h2 * h2; g += blockDim.x, ++cnt) {
            const int i = g / h2, j = g % h2;
            float L, HL, LH, HH;
            fwd4(A[(2 * i) * T + 2 * j], A[(2 * i) * T + 2 * j + 1], A[(2 * i + 1) * T + 2 * j],
                 A[(2 * i + 1) * T + 2 * j + 1], ab, L, HL, LH, HH);
            const int gi = ty * h2 + i, gj = tx * h2 + j;
            const int64_t o_hl = (int64_t)gi * n + N2 + gj, o_lh = (int64_t)(N2 + gi) * n + gj,
                          o_hh = (int64_t)(N2 + gi) * n + N2 + gj;
            if (scale) {
                HL *= scale[o_hl];
                LH *= scale[o_lh];
                HH *= scale[o_hh];
            }
            dst[o_hl] = HL;
            dst[o_lh] = LH;
            dst[o_hh] = HH;
            ll[cnt & 3] = L;
        }
        __syncthreads();
        cnt = 0;
        for (int g = threadIdx.x; g < h2 * h2; g += blockDim.x, ++cnt) {
            const int i = g / h2, j = g % h2;
            A[i * T + j] = ll[cnt & 3];
        }
        __syncthreads();
        h = h2;
        Ng = N2;
    }
    if (threadIdx.x == 0) dst[(int64_t)ty * n + tx] = A[0];
}

// Inverse over the tile levels: reads the tile's low-pass value at (ty, tx)
// and its detail coefficients, writes pixels (times post, if given).
__global__ void __launch_bounds__(kThreads)
    inv_tile_kernel(int n, int T, const float *__restrict__ coef, float *__restrict__ out,
                    const float *__restrict__ post, unsigned abs_mask) {
    __shared__ float A[kT * kT];
    const int ch = blockIdx.z;
    const bool ab = (abs_mask >> ch) & 1u;
    const int64_t nn = (int64_t)n * n;
    const float *src = coef + ch * nn;
    float *dst = out + ch * nn;
    const int ty = blockIdx.y, tx = blockIdx.x;
    if (threadIdx.x == 0) A[0] = src[(int64_t)ty * n + tx];
    __syncthreads();
    int h = 2, Ng = 2 * n / T;
    while (h <= T) {
        const int h2 = h / 2, N2 = Ng / 2;
        float a4[4][4];
        int cnt = 0;
        for (int g = threadIdx.x; g < h2 * h2; g += blockDim.x, ++cnt) {
            const int i = g / h2, j = g % h2;
            const int gi = ty * h2 + i, gj = tx * h2 + j;
            const float L = A[i * T + j];
            const float HL = src[(int64_t)gi * n + N2 + gj];
            const float LH = src[(int64_t)(N2 + gi) * n + gj];
            const float HH = src[(int64_t)(N2 + gi) * n + N2 + gj];
            inv4(L, HL, LH, HH, ab, a4[cnt & 3][0], a4[cnt & 3][1], a4[cnt & 3][2], a4[cnt & 3][3]);
        }
        __syncthreads();
        cnt = 0;
        for (int g = threadIdx.x; g < h2 * h2; g += blockDim.x, ++cnt) {
            const int i = g / h2, j = g % h2;
            A[(2 * i) * T + 2 * j] = a4[cnt & 3][0];
            A[(2 * i) * T + 2 * j + 1] = a4[cnt & 3][1];
            A[(2 * i + 1) * T + 2 * j] = a4[cnt & 3][2];
            A[(2 * i + 1) * T + 2 * j + 1] = a4[cnt & 3][3];
        }
        __syncthreads();
        h *= 2;
        Ng *= 2;
    }
    for (int k = threadIdx.x; k < T * T; k += blockDim.x) {
        const int r = k / T, c = k % T;
        const int64_t gi = (int64_t)(ty * T + r) * n + tx * T + c;
        float v = A[r * T + c];
        if (post) v *= post[gi];
        dst[gi] = v;
    }
}

// The (C x C) low-pass block, C = n/T, in one CTA per channel.  mode bit 0:
// run the remaining forward levels; bit 1: scale every coefficient of the
// block by `scale`; bit 2: run the inverse levels.  In place on coef.
__global__ void coarse_kernel(int n, int C, float *__restrict__ coef, const float *__restrict__ scale, int mode,
                              unsigned abs_mask) {
    extern __shared__ float B[];  // C*C + C*C
    float *tmp = B + C * C;
    const int ch = blockIdx.x;
    const bool ab = (abs_mask >> ch) & 1u;
    float *c0 = coef + (int64_t)ch * n * n;
    for (int k = threadIdx.x; k < C * C; k += blockDim.x) B[k] = c0[(int64_t)(k / C) * n + k % C];
    __syncthreads();
    if (mode & 1) {
        for (int h = C; h >= 2; h /= 2) {
            const int h2 = h / 2;
            for (int g = threadIdx.x; g < h2 * h2; g += blockDim.x) {
                const int i = g / h2, j = g % h2;
                float L, HL, LH, HH;
                fwd4(B[(2 * i) * C + 2 * j], B[(2 * i) * C + 2 * j + 1], B[(2 * i + 1) * C + 2 * j],
                     B[(2 * i + 1) * C + 2 * j + 1], ab, L, HL, LH, HH);
                tmp[i * C + j] = L;
                tmp[i * C + h2 + j] = HL;
                tmp[(h2 + i) * C + j] = LH;
                tmp[(h2 + i) * C + h2 + j] = HH;
            }
            __syncthreads();
            for (int g = threadIdx.x; g < h * h; g += blockDim.x) B[(g / h) * C + g % h] = tmp[(g / h) * C + g % h];
            __syncthreads();
        }
    }
    if (mode & 2) {
        for (int k = threadIdx.x; k < C * C; k += blockDim.x) B[k] *= scale[(int64_t)(k / C) * n + k % C];
        __syncthreads();
    }
    if (mode & 4) {
        for (int h = 2; h <= C; h *= 2) {
            const int h2 = h / 2;
            for (int g = threadIdx.x; g < h2 * h2; g += blockDim.x) {
                const int i = g / h2, j = g % h2;
                float a, b, c, d;
                inv4(B[i * C + j], B[i * C + h2 + j], B[(h2 + i) * C + j], B[(h2 + i) * C + h2 + j], ab, a, b, c, d);
                tmp[(2 * i) * C + 2 * j] = a;
                tmp[(2 * i) * C + 2 * j + 1] = b;
                tmp[(2 * i + 1) * C + 2 * j] = c;
                tmp[(2 * i + 1) * C + 2 * j + 1] = d;
            }
            __syncthreads();
            for (int g = threadIdx.x; g < h * h; g += blockDim.x) B[(g / h) * C + g % h] = tmp[(g / h) * C + g % h];
            __syncthreads();
        }
    }
    for (int k = threadIdx.x; k < C * C; k += blockDim.x) c0[(int64_t)(k / C) * n + k % C] = B[k];
}


// ---------------------------------------------------------------- 3-D
constexpr int kT3 = 16;
constexpr int kMaxC3 = 16;  // coarse block side: n / kT3 for n <= 256
constexpr float kR3 = 0.353553390593273762f;  // 2^-3/2

// In place on v[dz*4 + dy*2 + dx]: afterwards v[sz*4 + sy*2 + sx] holds the
// output of octant (sz, sy, sx); the same call inverts it.
__device__ __forceinline__ void bfly8(float (&v)[8], bool ab) {
    if (ab) {
        float t = 0.f;
#pragma unroll
        for (int q = 0; q < 8; ++q) t += v[q];
        t *= kR3;
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = t;
        return;
    }
#pragma unroll
    for (int stride = 1; stride < 8; stride *= 2)
#pragma unroll
        for (int q = 0; q < 8; ++q)
            if (!(q & stride)) {
                const float a = v[q], b = v[q + stride];
                v[q] = a + b;
                v[q + stride] = a - b;
            }
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] *= kR3;
}

__device__ __forceinline__ int64_t at3(int n, int z, int y, int x) { return ((int64_t)z * n + y) * n + x; }

// Forward over the tile levels.  grid: (C, C, C * channels), C = n / T.
__global__ void __launch_bounds__(kThreads)
    fwd3_tile_kernel(int n, int T, int C, const float *__restrict__ in, float *__restrict__ coef,
                     const float *__restrict__ pre, const float *__restrict__ scale, unsigned abs_mask) {
    __shared__ float A[kT3 * kT3 * kT3];
    const int ch = blockIdx.z / C, tz = blockIdx.z % C, ty = blockIdx.y, tx = blockIdx.x;
    const bool ab = (abs_mask >> ch) & 1u;
    const int64_t nnn = (int64_t)n * n * n;
    const float *src = in + ch * nnn;
    float *dst = coef + ch * nnn;
    for (int q = threadIdx.x; q < T * T * T; q += blockDim.x) {
        const int z = q / (T * T), y = (q / T) % T, x = q % T;
        const int64_t gi = at3(n, tz * T + z, ty * T + y, tx * T + x);
        float v = src[gi];
        if (pre) v *= pre[gi];
        A[q] = v;
    }
    __syncthreads();
    int h = T, Ng = n;
    while (h >= 2) {
        const int h2 = h / 2, N2 = Ng / 2;
        float ll[2];
        int cnt = 0;
        // at most (16/2)^3 = 512 groups: two per thread
        for (int g = threadIdx.x; g < h2 * h2 * h2; g += blockDim.x, ++cnt) {
            const int i = g / (h2 * h2), j = (g / h2) % h2, k = g % h2;
            float v[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) v[q] = A[((2 * i + (q >> 2)) * T + 2 * j + ((q >> 1) & 1)) * T + 2 * k + (q & 1)];
            bfly8(v, ab);
            const int gz = tz * h2 + i, gy = ty * h2 + j, gx = tx * h2 + k;
#pragma unroll
            for (int q = 1; q < 8; ++q) {
                const int64_t o = at3(n, (q >> 2) * N2 + gz, ((q >> 1) & 1) * N2 + gy, (q & 1) * N2 + gx);
                dst[o] = scale ? v[q] * scale[o] : v[q];
            }
            ll[cnt & 1] = v[0];
        }
        __syncthreads();
        cnt = 0;
        for (int g = threadIdx.x; g < h2 * h2 * h2; g += blockDim.x, ++cnt) {
            const int i = g / (h2 * h2), j = (g / h2) % h2, k = g % h2;
            A[(i * T + j) * T + k] = ll[cnt & 1];
        }
        __syncthreads();
        h = h2;
        Ng = N2;
    }
    if (threadIdx.x == 0) dst[at3(n, tz, ty, tx)] = A[0];
}

// Inverse over the tile levels: the tile's low-pass value at (tz, ty, tx)
// and its detail coefficients to voxels (times post, if given).
__global__ void __launch_bounds__(kThreads)
    inv3_tile_kernel(int n, int T, int C, const float *__restrict__ coef, float *__restrict__ out,
                     const float *__restrict__ post, unsigned abs_mask) {
    __shared__ float A[kT3 * kT3 * kT3];
    const int ch = blockIdx.z / C, tz = blockIdx.z % C, ty = blockIdx.y, tx = blockIdx.x;
    const bool ab = (abs_mask >> ch) & 1u;
    const int64_t nnn = (int64_t)n * n * n;
    const float *src = coef + ch * nnn;
    float *dst = out + ch * nnn;
    if (threadIdx.x == 0) A[0] = src[at3(n, tz, ty, tx)];
    __syncthreads();
    int h = 2, Ng = 2 * n / T;
    while (h <= T) {
        const int h2 = h / 2, N2 = Ng / 2;
        float a8[2][8];
        int cnt = 0;
        for (int g = threadIdx.x; g < h2 * h2 * h2; g += blockDim.x, ++cnt) {
            const int i = g / (h2 * h2), j = (g / h2) % h2, k = g % h2;
            const int gz = tz * h2 + i, gy = ty * h2 + j, gx = tx * h2 + k;
            float v[8];
            v[0] = A[(i * T + j) * T + k];
#pragma unroll
            for (int q = 1; q < 8; ++q) v[q] = src[at3(n, (q >> 2) * N2 + gz, ((q >> 1) & 1) * N2 + gy, (q & 1) * N2 + gx)];
            bfly8(v, ab);
#pragma unroll
            for (int q = 0; q < 8; ++q) a8[cnt & 1][q] = v[q];
        }
        __syncthreads();
        cnt = 0;
        for (int g = threadIdx.x; g < h2 * h2 * h2; g += blockDim.x, ++cnt) {
            const int i = g / (h2 * h2), j = (g / h2) % h2, k = g % h2;
#pragma unroll
            for (int q = 0; q < 8; ++q)
                A[((2 * i + (q >> 2)) * T + 2 * j + ((q >> 1) & 1)) * T + 2 * k + (q & 1)] = a8[cnt & 1][q];
        }
        __syncthreads();
        h *= 2;
        Ng *= 2;
    }
    for (int q = threadIdx.x; q < T * T * T; q += blockDim.x) {
        const int z = q / (T * T), y = (q / T) % T, x = q % T;
        const int64_t gi = at3(n, tz * T + z, ty * T + y, tx * T + x);
        float v = A[q];
        if (post) v *= post[gi];
        dst[gi] = v;
    }
}

// The C^3 low-pass block in one CTA per channel (modes as coarse_kernel).
__global__ void coarse3_kernel(int n, int C, float *__restrict__ coef, const float *__restrict__ scale, int mode,
                               unsigned abs_mask) {
    extern __shared__ float B[];  // C^3 + C^3
    const int C3 = C * C * C;
    float *tmp = B + C3;
    const int ch = blockIdx.x;
    const bool ab = (abs_mask >> ch) & 1u;
    float *c0 = coef + (int64_t)ch * n * n * n;
    for (int q = threadIdx.x; q < C3; q += blockDim.x) B[q] = c0[at3(n, q / (C * C), (q / C) % C, q % C)];
    __syncthreads();
    if (mode & 1) {
        for (int h = C; h >= 2; h /= 2) {
            const int h2 = h / 2;
            for (int g = threadIdx.x; g < h2 * h2 * h2; g += blockDim.x) {
                const int i = g / (h2 * h2), j = (g / h2) % h2, k = g % h2;
                float v[8];
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    v[q] = B[((2 * i + (q >> 2)) * C + 2 * j + ((q >> 1) & 1)) * C + 2 * k + (q & 1)];
                bfly8(v, ab);
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    tmp[(((q >> 2) * h2 + i) * C + ((q >> 1) & 1) * h2 + j) * C + (q & 1) * h2 + k] = v[q];
            }
            __syncthreads();
            for (int g = threadIdx.x; g < h * h * h; g += blockDim.x) {
                const int idx = ((g / (h * h)) * C + (g / h) % h) * C + g % h;
                B[idx] = tmp[idx];
            }
            __syncthreads();
        }
    }
    if (mode & 2) {
        for (int q = threadIdx.x; q < C3; q += blockDim.x) B[q] *= scale[at3(n, q / (C * C), (q / C) % C, q % C)];
        __syncthreads();
    }
    if (mode & 4) {
        for (int h = 2; h <= C; h *= 2) {
            const int h2 = h / 2;
            for (int g = threadIdx.x; g < h2 * h2 * h2; g += blockDim.x) {
                const int i = g / (h2 * h2), j = (g / h2) % h2, k = g % h2;
                float v[8];
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    v[q] = B[(((q >> 2) * h2 + i) * C + ((q >> 1) & 1) * h2 + j) * C + (q & 1) * h2 + k];
                bfly8(v, ab);
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    tmp[((2 * i + (q >> 2)) * C + 2 * j + ((q >> 1) & 1)) * C + 2 * k + (q & 1)] = v[q];
            }
            __syncthreads();
            for (int g = threadIdx.x; g < h * h * h; g += blockDim.x) {
                const int idx = ((g / (h * h)) * C + (g / h) % h) * C + g % h;
                B[idx] = tmp[idx];
            }
            __syncthreads();
        }
    }
    for (int q = threadIdx.x; q < C3; q += blockDim.x) c0[at3(n, q / (C * C), (q / C) % C, q % C)] = B[q];
}

}  // namespace

bool haar_supported(int nx, int ny, int nz) {
    if (nz > 1) {
        if (nx != ny || ny != nz || nx < 2 || nx > kT3 * kMaxC3) return false;
        return (nx & (nx - 1)) == 0;
    }
    if (nx != ny || nx < 2 || nx > 2048) return false;
    return (nx & (nx - 1)) == 0;
}

namespace {
struct Haar3Launch {
    int T, C;
    size_t smem;
    explicit Haar3Launch(int n) : T(n < kT3 ? n : kT3), C(n / (n < kT3 ? n : kT3)), smem(2 * sizeof(float) * C * C * C) {}
};
}  // namespace

mbir_status haar_forward(int n, int channels, const float *in, float *coef, const float *pre, const float *scale,
                         unsigned abs_mask, cudaStream_t s, int nz) {
    if (nz > 1) {
        const Haar3Launch L(n);
        fwd3_tile_kernel<<<dim3(L.C, L.C, L.C * channels), kThreads, 0, s>>>(n, L.T, L.C, in, coef, pre, scale,
                                                                              abs_mask);
        PSPS_LAUNCH_CHECK();
        coarse3_kernel<<<channels, kThreads, L.smem, s>>>(n, L.C, coef, scale, scale ? 3 : 1, abs_mask);
        PSPS_LAUNCH_CHECK();
        return MBIR_OK;
    }
    const int T = n < kT ? n : kT, C = n / T;
    fwd_tile_kernel<<<dim3(C, C, channels), kThreads, 0, s>>>(n, T, in, coef, pre, scale, abs_mask);
    PSPS_LAUNCH_CHECK();
    coarse_kernel<<<channels, kThreads, 2 * C * C * sizeof(float), s>>>(n, C, coef, scale, scale ? 3 : 1, abs_mask);
    PSPS_LAUNCH_CHECK();
    return MBIR_OK;
}

mbir_status haar_inverse(int n, int channels, float *coef, float *out, const float *post, unsigned abs_mask,
                         cudaStream_t s, int nz) {
    if (nz > 1) {
        const Haar3Launch L(n);
        coarse3_kernel<<<channels, kThreads, L.smem, s>>>(n, L.C, coef, nullptr, 4, abs_mask);
        PSPS_LAUNCH_CHECK();
        inv3_tile_kernel<<<dim3(L.C, L.C, L.C * channels), kThreads, 0, s>>>(n, L.T, L.C, coef, out, post, abs_mask);
        PSPS_LAUNCH_CHECK();
        return MBIR_OK;
    }
    const int T = n < kT ? n : kT, C = n / T;
    coarse_kernel<<<channels, kThreads, 2 * C * C * sizeof(float), s>>>(n, C, coef, nullptr, 4, abs_mask);
    PSPS_LAUNCH_CHECK();
    inv_tile_kernel<<<dim3(C, C, channels), kThreads, 0, s>>>(n, T, coef, out, post, abs_mask);
    PSPS_LAUNCH_CHECK();
    return MBIR_OK;
}

mbir_status haar_apply(int n, int channels, const float *in, float *tmp, float *out, const float *pre,
                       const float *post, const float *scale, unsigned abs_mask, cudaStream_t s, int nz) {
    if (nz > 1) {
        const Haar3Launch L(n);
        fwd3_tile_kernel<<<dim3(L.C, L.C, L.C * channels), kThreads, 0, s>>>(n, L.T, L.C, in, tmp, pre, scale,
                                                                              abs_mask);
        PSPS_LAUNCH_CHECK();
        coarse3_kernel<<<channels, kThreads, L.smem, s>>>(n, L.C, tmp, scale, 7, abs_mask);
        PSPS_LAUNCH_CHECK();
        inv3_tile_kernel<<<dim3(L.C, L.C, L.C * channels), kThreads, 0, s>>>(n, L.T, L.C, tmp, out, post, abs_mask);
        PSPS_LAUNCH_CHECK();
        return MBIR_OK;
    }
    const int T = n < kT ? n : kT, C = n / T;
    fwd_tile_kernel<<<dim3(C, C, channels), kThreads, 0, s>>>(n, T, in, tmp, pre, scale, abs_mask);
    PSPS_LAUNCH_CHECK();
    coarse_kernel<<<channels, kThreads, 2 * C * C * sizeof(float), s>>>(n, C, tmp, scale, 7, abs_mask);
    PSPS_LAUNCH_CHECK();
    inv_tile_kernel<<<dim3(C, C, channels), kThreads, 0, s>>>(n, T, tmp, out, post, abs_mask);
    PSPS_LAUNCH_CHECK();
    return MBIR_OK;
}

}  // namespace psps
