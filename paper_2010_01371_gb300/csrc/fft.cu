// Shared-memory batched FFT for the Fourier preconditioners (Eqs. 28-33,
// 56-57): M v = m0 .* U^H (s .* U (m0 .* v)) with U the unitary 2-D DFT over
// the image grid (periodic, per material) and s a real spectrum
// (Lambda~^-1/2, or the spectrum of the absolute kernel for |M|).
//
// One kernel runs mixed-radix Stockham passes (self-sorting, natural order;
// radices 4, 2, 3, 5, 7) on B transforms of length N held in shared memory;
// loads and stores are coalesced for both row transforms (unit element
// stride) and column transforms (unit batch stride).  Pass s with radix R
// after a product Ns of the earlier radices maps, for j < N/R, the inputs
// X[j + r N/R] (r < R), times the twiddles e^{-/+2 pi i r (j mod Ns)/(Ns R)},
// through an R-point DFT to Y[(j div Ns) Ns R + (j mod Ns) + r Ns].
// A 2-D apply is three launches:
//   rows forward (real input, times m0) -> columns forward, spectral
//   multiply, columns inverse -> rows inverse (real part, 1/(nx ny), times m0).
// Twiddles e^{-2 pi i k/N} and the R-point roots of unity are generated in
// FP64 on the host and stored FP32.  Sizes 2^a 3^b 5^c 7^d up to 1024.
#include <cmath>
#include <vector>

#include "fft.cuh"

namespace psps {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Roots of unity of the small DFTs, stored after the N twiddles of a table:
// offsets of the R = 3, 5, 7 roots e^{-2 pi i k/R}, k < R.
constexpr int kRoot3 = 0, kRoot5 = 3, kRoot7 = 8, kRoots = 15;
constexpr int kMaxPasses = 12;

// R-point DFT of v in place; root[k] = e^{-2 pi i k/R} (conjugated for the
// inverse, dir = +1).
template <int R>
__device__ __forceinline__ void small_dft(float2 (&v)[R], int dir, const float2 *__restrict__ root) {
    if constexpr (R == 2) {
        const float2 a = v[0], b = v[1];
        v[0] = make_float2(a.x + b.x, a.y + b.y);
        v[1] = make_float2(a.x - b.x, a.y - b.y);
    } else if constexpr (R == 4) {
        const float2 a = make_float2(v[0].x + v[2].x, v[0].y + v[2].y);
        const float2 b = make_float2(v[0].x - v[2].x, v[0].y - v[2].y);
        const float2 c = make_float2(v[1].x + v[3].x, v[1].y + v[3].y);
        const float2 e = make_float2(v[1].x - v[3].x, v[1].y - v[3].y);
        // d = e * (i dir): e^{dir 2 pi i / 4} = i dir
        const float2 d = dir > 0 ? make_float2(-e.y, e.x) : make_float2(e.y, -e.x);
        v[0] = make_float2(a.x + c.x, a.y + c.y);
        v[2] = make_float2(a.x - c.x, a.y - c.y);
        v[1] = make_float2(b.x + d.x, b.y + d.y);
        v[3] = make_float2(b.x - d.x, b.y - d.y);
    } else {
        float2 w[R];
#pragma unroll
        for (int k = 0; k < R; ++k) {
            w[k] = root[k];
            if (dir > 0) w[k].y = -w[k].y;
        }
        float2 out[R];
#pragma unroll
        for (int m = 0; m < R; ++m) {
            float2 acc = v[0];
#pragma unroll
            for (int r = 1; r < R; ++r) {
                const float2 t = cmul(v[r], w[(m * r) % R]);
                acc.x += t.x;
                acc.y += t.y;
            }
            out[m] = acc;
        }
#pragma unroll
        for (int m = 0; m < R; ++m) v[m] = out[m];
    }
}

template <int R>
__device__ __forceinline__ void stockham_pass(const float2 *__restrict__ X, float2 *__restrict__ Y, int N, int B,
                                              int Ns, int dir, const float2 *__restrict__ tw,
                                              const float2 *__restrict__ root) {
    const int NR = N / R;
    const int tstep = N / (Ns * R);
    for (int t = threadIdx.x; t < B * NR; t += blockDim.x) {
        const int b = t / NR, j = t - b * NR;
        const int jm = j % Ns;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            v[r] = X[b * N + j + r * NR];
            if (r > 0) {
                float2 w = tw[jm * r * tstep];
                if (dir > 0) w.y = -w.y;
                v[r] = cmul(v[r], w);
            }
        }
        small_dft<R>(v, dir, root);
        const int idx = (j / Ns) * Ns * R + jm;
#pragma unroll
        for (int r = 0; r < R; ++r) Y[b * N + idx + r * Ns] = v[r];
    }
}

struct Radices {
    int n = 0;
    int r[kMaxPasses] = {};
};

// Stockham over B transforms of length N in shared memory X (result left in
// the returned buffer).  dir = -1 forward (e^{-i}), +1 inverse.
__device__ float2 *stockham(float2 *X, float2 *Y, int N, int B, int dir, const Radices &rad,
                            const float2 *__restrict__ tw) {
    const float2 *roots = tw + N;
    int Ns = 1;
    for (int s = 0; s < rad.n; ++s) {
        const int R = rad.r[s];
        switch (R) {
            case 4: stockham_pass<4>(X, Y, N, B, Ns, dir, tw, roots); break;
            case 2: stockham_pass<2>(X, Y, N, B, Ns, dir, tw, roots); break;
            case 3: stockham_pass<3>(X, Y, N, B, Ns, dir, tw, roots + kRoot3); break;
            case 5: stockham_pass<5>(X, Y, N, B, Ns, dir, tw, roots + kRoot5); break;
            default: stockham_pass<7>(X, Y, N, B, Ns, dir, tw, roots + kRoot7); break;
        }
        __syncthreads();
        float2 *t = X;
        X = Y;
        Y = t;
        Ns *= R;
    }
    return X;
}

struct Pass {
    int N, B;            // transform length, transforms per CTA
    int64_t ks, bs;      // element stride, batch stride (in elements)
    int nbatch;          // total transforms per channel
    int64_t ch_stride;   // elements per channel
    Radices rad;         // radix of each Stockham pass
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
        R = stockham(X, Y, p.N, p.B, -1, p.rad, tw);
    } else if (mode == 1) {
        R = stockham(X, Y, p.N, p.B, -1, p.rad, tw);
        for (int idx = threadIdx.x; idx < p.N * p.B; idx += blockDim.x) {
            const int b = idx / p.N, k = idx % p.N;
            if (b >= nb) continue;
            const float s = spec[(int64_t)k * spec_ks + (int64_t)(b0 + b) * spec_bs];
            R[idx].x *= s;
            R[idx].y *= s;
        }
        __syncthreads();
        R = stockham(R, R == X ? Y : X, p.N, p.B, +1, p.rad, tw);
    } else {  // modes 2 and 4
        R = stockham(X, Y, p.N, p.B, +1, p.rad, tw);
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

// Transforms per CTA: at most ~4096 complex values per buffer, and few
// enough that the grid has about two CTAs per SM (small images would
// otherwise run on a handful of CTAs).  Strided (column) transforms read B
// consecutive elements per row: keep at least four (one 32-byte sector) when
// the buffer allows.
int pick_B(int N, int64_t transforms, bool strided) {
    const int cap = 4096 / N < 1 ? 1 : 4096 / N;
    int B = cap;
    const int64_t want = cdiv(transforms, 2 * 152);
    if (want < B) B = (int)want;
    if (strided && B < 4) B = cap < 4 ? cap : 4;
    return B < 1 ? 1 : B;
}

// Radix plan of N: radix-4 passes while 4 divides N, one radix-2 pass for an
// odd power of two, then 3, 5, 7.  False if another prime divides N.
bool factor(int N, Radices &rad) {
    rad.n = 0;
    while (N % 4 == 0 && rad.n < kMaxPasses) rad.r[rad.n++] = 4, N /= 4;
    if (N % 2 == 0 && rad.n < kMaxPasses) rad.r[rad.n++] = 2, N /= 2;
    for (int R : {3, 5, 7})
        while (N % R == 0 && rad.n < kMaxPasses) rad.r[rad.n++] = R, N /= R;
    return N == 1;
}

Pass make_pass(int N, int64_t ks, int64_t bs, int nbatch, int64_t ch_stride, int64_t transforms) {
    Pass p{N, pick_B(N, transforms, ks != 1), ks, bs, nbatch, ch_stride, {}};
    factor(N, p.rad);
    return p;
}

}  // namespace

bool fft_supported(int n) {
    Radices r;
    return n >= 2 && n <= 1024 && factor(n, r);
}

mbir_status FftPlan::init(int nx_, int ny_, int nz_) {
    nx = nx_;
    ny = ny_;
    nz = nz_;
    if (!fft_supported(nx) || !fft_supported(ny) || (nz > 1 && !fft_supported(nz)))
        return fail(MBIR_ERR_UNIMPLEMENTED, "FFT sizes must be 2^a 3^b 5^c 7^d in 2..1024 (got %d x %d x %d)", nx, ny,
                    nz);
    for (int a = 0; a < 3; ++a) {
        const int N = a == 0 ? nx : (a == 1 ? ny : nz);
        if (a == 2 && nz <= 1) break;
        std::vector<float2> h(N + kRoots);
        for (int k = 0; k < N; ++k) {
            const double ang = -2.0 * M_PI * (double)k / (double)N;
            h[k] = make_float2((float)cos(ang), (float)sin(ang));
        }
        const int radix[3] = {3, 5, 7}, off[3] = {kRoot3, kRoot5, kRoot7};
        for (int q = 0; q < 3; ++q)
            for (int k = 0; k < radix[q]; ++k) {
                const double ang = -2.0 * M_PI * (double)k / (double)radix[q];
                h[N + off[q] + k] = make_float2((float)cos(ang), (float)sin(ang));
            }
        DBuf<float2> &t = a == 0 ? twx : (a == 1 ? twy : twz);
        PSPS_TRY(t.alloc(N + kRoots));
        PSPS_CUDA(cudaMemcpy(t.p, h.data(), sizeof(float2) * h.size(), cudaMemcpyHostToDevice));
    }
    static bool attr_done = false;
    if (!attr_done) {
        PSPS_CUDA(cudaFuncSetAttribute(fft_pass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * 4096 * 8 + 1024));
        attr_done = true;
    }
    return MBIR_OK;
}

// One pass of 1-D transforms along axis 0 (x, rows), 1 (y, columns) or 2 (z)
// of [channels][nz][ny][nx] data; see fft_pass_kernel for the modes.  A
// spectral multiply (mode 1) reads spec[z][y][x].
mbir_status FftPlan::run(int axis, int mode, int channels, const float *rin, float2 *Z, float *rout,
                         const float *pre_post, const float *spec, cudaStream_t s) const {
    const int64_t plane = (int64_t)nx * ny, nvox = plane * nz;
    Pass p;
    dim3 grid;
    int64_t sks = 0, sbs = 0;
    const float2 *tw;
    if (axis == 0) {
        p = make_pass(nx, 1, nx, ny * nz, nvox, (int64_t)ny * nz * channels);
        grid = dim3((unsigned)cdiv((int64_t)ny * nz, p.B), channels);
        tw = twx.p;
    } else if (axis == 1) {
        // every z-plane of every channel is its own batch
        p = make_pass(ny, nx, 1, nx, plane, (int64_t)nx * nz * channels);
        grid = dim3((unsigned)cdiv(nx, p.B), channels * nz);
        sks = nx, sbs = 1;
        tw = twy.p;
    } else {
        p = make_pass(nz, plane, 1, (int)plane, nvox, plane * channels);
        grid = dim3((unsigned)cdiv(plane, p.B), channels);
        sks = plane, sbs = 1;
        tw = twz.p;
    }
    const size_t sm = 2 * sizeof(float2) * p.N * p.B;
    fft_pass_kernel<<<grid, kThreads, sm, s>>>(p, mode, rin, Z, rout, pre_post, spec, sks, sbs,
                                               (float)(1.0 / (double)nvox), tw);
    PSPS_LAUNCH_CHECK();
    return MBIR_OK;
}

mbir_status FftPlan::forward(int channels, const float *in, float2 *Z, cudaStream_t s) const {
    PSPS_TRY(run(0, 0, channels, in, Z, nullptr, nullptr, nullptr, s));
    PSPS_TRY(run(1, 3, channels, nullptr, Z, nullptr, nullptr, nullptr, s));
    if (nz > 1) PSPS_TRY(run(2, 3, channels, nullptr, Z, nullptr, nullptr, nullptr, s));
    return MBIR_OK;
}

mbir_status FftPlan::inverse(int channels, float2 *Z, float *out, const float *post, cudaStream_t s) const {
    if (nz > 1) PSPS_TRY(run(2, 4, channels, nullptr, Z, nullptr, nullptr, nullptr, s));
    PSPS_TRY(run(1, 4, channels, nullptr, Z, nullptr, nullptr, nullptr, s));
    return run(0, 2, channels, nullptr, Z, out, post, nullptr, s);
}

mbir_status FftPlan::filter(int channels, const float *in, float2 *Z, float *out, const float *pre, const float *post,
                            const float *spec, cudaStream_t s) const {
    PSPS_TRY(run(0, 0, channels, in, Z, nullptr, pre, nullptr, s));
    if (nz > 1) {
        PSPS_TRY(run(1, 3, channels, nullptr, Z, nullptr, nullptr, nullptr, s));
        PSPS_TRY(run(2, 1, channels, nullptr, Z, nullptr, nullptr, spec, s));   // forward, multiply, inverse in z
        PSPS_TRY(run(1, 4, channels, nullptr, Z, nullptr, nullptr, nullptr, s));
    } else {
        PSPS_TRY(run(1, 1, channels, nullptr, Z, nullptr, nullptr, spec, s));   // forward, multiply, inverse in y
    }
    return run(0, 2, channels, nullptr, Z, out, post, nullptr, s);
}

}  // namespace psps
