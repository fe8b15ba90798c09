// Shared-memory batched FFT for the Fourier preconditioners (Eqs. 28-33,
// 56-57): M v = m0 .* U^H (s .* U (m0 .* v)) with U the unitary 2-D DFT over
// the image grid (periodic, per material) and s a real spectrum
// (Lambda~^-1/2, or the spectrum of the absolute kernel for |M|).
//
// One kernel runs radix-2 Stockham passes (self-sorting, natural order) on B
// transforms of length N held in shared memory; loads and stores are
// coalesced for both row transforms (unit element stride) and column
// transforms (unit batch stride).  A 2-D apply is three launches:
//   rows forward (real input, times m0) -> columns forward, spectral
//   multiply, columns inverse -> rows inverse (real part, 1/(nx ny), times m0).
// Twiddles e^{-2 pi i k/N} are generated in FP64 on the host, stored FP32.
// Power-of-two sizes up to 1024.
#include <cmath>
#include <vector>

#include "fft.cuh"

namespace psps {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Stockham radix-2 over B transforms of length N in shared memory X (result
// left in the returned buffer).  dir = -1 forward (e^{-i}), +1 inverse.
__device__ float2 *stockham(float2 *X, float2 *Y, int N, int B, int dir, const float2 *__restrict__ tw) {
    const int half = N / 2;
    for (int Ns = 1; Ns < N; Ns *= 2) {
        const int tstep = N / (2 * Ns);
        for (int t = threadIdx.x; t < B * half; t += blockDim.x) {
            const int b = t / half, j = t % half;
            const float2 v0 = X[b * N + j];
            float2 w = tw[(j % Ns) * tstep];
            if (dir > 0) w.y = -w.y;
            const float2 v1 = cmul(X[b * N + j + half], w);
            const int idx = (j / Ns) * 2 * Ns + (j % Ns);
            Y[b * N + idx] = make_float2(v0.x + v1.x, v0.y + v1.y);
            Y[b * N + idx + Ns] = make_float2(v0.x - v1.x, v0.y - v1.y);
        }
        __syncthreads();
        float2 *t = X;
        X = Y;
        Y = t;
    }
    return X;
}

struct Pass {
    int N, B;            // transform length, transforms per CTA
    int64_t ks, bs;      // element stride, batch stride (in elements)
    int nbatch;          // total transforms per channel
    int64_t ch_stride;   // elements per channel
};

__device__ __forceinline__ void lin(const Pass &p, int idx, int &b, int &k) {
    if (p.ks == 1) {
        b = idx / p.N;
        k = idx % p.N;
    } else {
        k = idx / p.B;
        b = idx % p.B;
    }
}

// mode 0: forward, real input (times pre) -> complex Z
// mode 3: forward, complex Z in place
// mode 1: forward, spectral multiply by spec[k * spec_ks + b * spec_bs] (real),
//         inverse; complex Z in place
// mode 2: inverse, complex Z -> real output (times post, times norm)
// mode 4: inverse, complex Z in place
__global__ void __launch_bounds__(kThreads)
    fft_pass_kernel(Pass p, int mode, const float *__restrict__ rin, float2 *__restrict__ Z, float *__restrict__ rout,
                    const float *__restrict__ pre_post, const float *__restrict__ spec, int64_t spec_ks, int64_t spec_bs,
                    float norm, const float2 *__restrict__ tw) {
    extern __shared__ float2 sm[];
    float2 *X = sm, *Y = sm + p.N * p.B;
    const int ch = blockIdx.y;
    const int b0 = blockIdx.x * p.B;
    const int nb = min(p.B, p.nbatch - b0);
    const int64_t cbase = ch * p.ch_stride;
    for (int idx = threadIdx.x; idx < p.N * p.B; idx += blockDim.x) {
        int b, k;
        lin(p, idx, b, k);
        if (b >= nb) continue;
        const int64_t off = (int64_t)(b0 + b) * p.bs + (int64_t)k * p.ks;
        float2 v;
        if (mode == 0) {
            float r = rin[cbase + off];
            if (pre_post) r *= pre_post[off];
            v = make_float2(r, 0.f);
        } else {
            v = Z[cbase + off];
        }
        X[b * p.N + k] = v;
    }
    __syncthreads();
    float2 *R;
    if (mode == 0 || mode == 3) {
        R = stockham(X, Y, p.N, p.B, -1, tw);
    } else if (mode == 1) {
        R = stockham(X, Y, p.N, p.B, -1, tw);
        for (int idx = threadIdx.x; idx < p.N * p.B; idx += blockDim.x) {
            const int b = idx / p.N, k = idx % p.N;
            if (b >= nb) continue;
            const float s = spec[(int64_t)k * spec_ks + (int64_t)(b0 + b) * spec_bs];
            R[idx].x *= s;
            R[idx].y *= s;
        }
        __syncthreads();
        R = stockham(R, R == X ? Y : X, p.N, p.B, +1, tw);
    } else {  // modes 2 and 4
        R = stockham(X, Y, p.N, p.B, +1, tw);
    }
    for (int idx = threadIdx.x; idx < p.N * p.B; idx += blockDim.x) {
        int b, k;
        lin(p, idx, b, k);
        if (b >= nb) continue;
        const int64_t off = (int64_t)(b0 + b) * p.bs + (int64_t)k * p.ks;
        const float2 v = R[b * p.N + k];
        if (mode == 2) {
            float r = v.x * norm;
            if (pre_post) r *= pre_post[off];
            rout[cbase + off] = r;
        } else {
            Z[cbase + off] = v;
        }
    }
}

int pick_B(int N) {
    // about 4096 complex values per CTA in each of the two buffers
    int B = 4096 / N;
    return B < 1 ? 1 : B;
}

}  // namespace

bool fft_supported(int n) { return n >= 2 && n <= 1024 && (n & (n - 1)) == 0; }

mbir_status FftPlan::init(int nx_, int ny_) {
    nx = nx_;
    ny = ny_;
    if (!fft_supported(nx) || !fft_supported(ny))
        return fail(MBIR_ERR_UNIMPLEMENTED, "FFT sizes must be powers of two in 2..1024 (got %d x %d)", nx, ny);
    for (int a = 0; a < 2; ++a) {
        const int N = a == 0 ? nx : ny;
        std::vector<float2> h(N);
        for (int k = 0; k < N; ++k) {
            const double ang = -2.0 * M_PI * (double)k / (double)N;
            h[k] = make_float2((float)cos(ang), (float)sin(ang));
        }
        DBuf<float2> &t = a == 0 ? twx : twy;
        PSPS_TRY(t.alloc(N));
        PSPS_CUDA(cudaMemcpy(t.p, h.data(), sizeof(float2) * N, cudaMemcpyHostToDevice));
    }
    static bool attr_done = false;
    if (!attr_done) {
        PSPS_CUDA(cudaFuncSetAttribute(fft_pass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * 4096 * 8 + 1024));
        attr_done = true;
    }
    return MBIR_OK;
}

mbir_status FftPlan::forward(int channels, const float *in, float2 *Z, cudaStream_t s) const {
    const int64_t npix = (int64_t)nx * ny;
    {
        Pass p{nx, pick_B(nx), 1, nx, ny, npix};
        const size_t sm = 2 * sizeof(float2) * p.N * p.B;
        fft_pass_kernel<<<dim3((unsigned)cdiv(ny, p.B), channels), kThreads, sm, s>>>(p, 0, in, Z, nullptr, nullptr,
                                                                                    nullptr, 0, 0, 1.f, twx.p);
        PSPS_LAUNCH_CHECK();
    }
    {
        Pass p{ny, pick_B(ny), nx, 1, nx, npix};
        const size_t sm = 2 * sizeof(float2) * p.N * p.B;
        fft_pass_kernel<<<dim3((unsigned)cdiv(nx, p.B), channels), kThreads, sm, s>>>(p, 3, nullptr, Z, nullptr, nullptr,
                                                                                    nullptr, 0, 0, 1.f, twy.p);
        PSPS_LAUNCH_CHECK();
    }
    return MBIR_OK;
}

mbir_status FftPlan::inverse(int channels, float2 *Z, float *out, const float *post, cudaStream_t s) const {
    const int64_t npix = (int64_t)nx * ny;
    {
        Pass p{ny, pick_B(ny), nx, 1, nx, npix};
        const size_t sm = 2 * sizeof(float2) * p.N * p.B;
        fft_pass_kernel<<<dim3((unsigned)cdiv(nx, p.B), channels), kThreads, sm, s>>>(p, 4, nullptr, Z, nullptr, nullptr,
                                                                                    nullptr, 0, 0, 1.f, twy.p);
        PSPS_LAUNCH_CHECK();
    }
    {
        Pass p{nx, pick_B(nx), 1, nx, ny, npix};
        const size_t sm = 2 * sizeof(float2) * p.N * p.B;
        fft_pass_kernel<<<dim3((unsigned)cdiv(ny, p.B), channels), kThreads, sm, s>>>(
            p, 2, nullptr, Z, out, post, nullptr, 0, 0, (float)(1.0 / (double)npix), twx.p);
        PSPS_LAUNCH_CHECK();
    }
    return MBIR_OK;
}

mbir_status FftPlan::filter(int channels, const float *in, float2 *Z, float *out, const float *m0, const float *spec,
                            cudaStream_t s) const {
    const int64_t npix = (int64_t)nx * ny;
    // rows: ny transforms of length nx, element stride 1, batch stride nx
    {
        Pass p{nx, pick_B(nx), 1, nx, ny, npix};
        const size_t sm = 2 * sizeof(float2) * p.N * p.B;
        fft_pass_kernel<<<dim3((unsigned)cdiv(ny, p.B), channels), kThreads, sm, s>>>(p, 0, in, Z, nullptr, m0, nullptr,
                                                                                    0, 0, 1.f, twx.p);
        PSPS_LAUNCH_CHECK();
    }
    // columns: nx transforms of length ny, element stride nx, batch stride 1
    {
        Pass p{ny, pick_B(ny), nx, 1, nx, npix};
        const size_t sm = 2 * sizeof(float2) * p.N * p.B;
        fft_pass_kernel<<<dim3((unsigned)cdiv(nx, p.B), channels), kThreads, sm, s>>>(p, 1, nullptr, Z, nullptr, nullptr,
                                                                                    spec, nx, 1, 1.f, twy.p);
        PSPS_LAUNCH_CHECK();
    }
    {
        Pass p{nx, pick_B(nx), 1, nx, ny, npix};
        const size_t sm = 2 * sizeof(float2) * p.N * p.B;
        fft_pass_kernel<<<dim3((unsigned)cdiv(ny, p.B), channels), kThreads, sm, s>>>(
            p, 2, nullptr, Z, out, m0, nullptr, 0, 0, (float)(1.0 / (double)npix), twx.p);
        PSPS_LAUNCH_CHECK();
    }
    return MBIR_OK;
}

}  // namespace psps
