// Quadratic roughness penalty R(x) = 1/2 x^T R x with R = beta (x) Gamma
// (Eqs. 26, 50-52): Gamma_jj = |N_j|, Gamma_jj' = -1 for the 4 (2-D) or 6
// (3-D) grid neighbours inside the image; beta is n_mat x n_mat.  The matrix
// form is used (Eq. 49 counts every neighbour pair twice relative to it).
#include "penalty.cuh"

namespace psps {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ float gamma_at(const float *__restrict__ v, int64_t j, int ix, int iy, int iz, int nx,
                                          int ny, int nz, float sign) {
    const float c = v[j];
    float acc = 0.f;
    int cnt = 0;
    const int64_t sx = 1, sy = nx, sz = (int64_t)nx * ny;
    if (ix > 0) { acc += v[j - sx]; ++cnt; }
    if (ix < nx - 1) { acc += v[j + sx]; ++cnt; }
    if (iy > 0) { acc += v[j - sy]; ++cnt; }
    if (iy < ny - 1) { acc += v[j + sy]; ++cnt; }
    if (iz > 0) { acc += v[j - sz]; ++cnt; }
    if (iz < nz - 1) { acc += v[j + sz]; ++cnt; }
    return (float)cnt * c + sign * acc;
}

// Writes Rx (if rx_out) and reduces sum x.Rx, p.Rx, p.Rp (double-float
// partials).
// abs_mode: |R| v instead (positive taps, |beta|), no reductions.
__global__ void __launch_bounds__(kThreads)
    penalty_kernel(PenaltyDev pd, int nx, int ny, int nz, const float *__restrict__ x, const float *__restrict__ p,
                   float *__restrict__ rx_out, int accumulate, int abs_mode, dfloat *__restrict__ partials) {
    const int64_t npix = (int64_t)nx * ny * nz;
    dfloat s0{0.f, 0.f}, s1{0.f, 0.f}, s2{0.f, 0.f};
    const float sign = abs_mode ? 1.f : -1.f;
    const int64_t plane = (int64_t)nx * ny;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < npix; j += (int64_t)gridDim.x * blockDim.x) {
        // one 64-bit division per pixel; the in-plane split is 32-bit
        const int iz = (int)(j / plane);
        const int jp = (int)(j - (int64_t)iz * plane);
        const int iy = jp / nx;
        const int ix = jp - iy * nx;
        float gx[4] = {0, 0, 0, 0}, gp[4] = {0, 0, 0, 0};
        for (int k = 0; k < pd.nm; ++k) {
            if (x) gx[k] = gamma_at(x + k * npix, j, ix, iy, iz, nx, ny, nz, sign);
            if (p) gp[k] = gamma_at(p + k * npix, j, ix, iy, iz, nx, ny, nz, sign);
        }
        for (int k = 0; k < pd.nm; ++k) {
            float rx = 0.f, rp = 0.f;
            for (int k2 = 0; k2 < pd.nm; ++k2) {
                const float b = abs_mode ? fabsf(pd.beta[k * 4 + k2]) : pd.beta[k * 4 + k2];
                rx = fmaf(b, gx[k2], rx);
                rp = fmaf(b, gp[k2], rp);
            }
            if (rx_out) {
                float *o = rx_out + k * npix + j;
                *o = accumulate ? *o + rx : rx;
            }
            if (partials) {
                const float xv = x ? x[k * npix + j] : 0.f;
                const float pv = p ? p[k * npix + j] : 0.f;
                df_add(s0, xv * rx);
                df_add(s1, pv * rx);
                df_add(s2, pv * rp);
            }
        }
    }
    if (partials) {
        dfloat v[3] = {s0, s1, s2};
        block_sum_store<3>(v, partials);
    }
}

}  // namespace

mbir_status launch_penalty(const PenaltyDev &pd, int nx, int ny, int nz, const float *x, const float *p, float *rx_out,
                           int accumulate, int abs_mode, dfloat *partials, int nblocks, cudaStream_t s) {
    penalty_kernel<<<nblocks, kThreads, 0, s>>>(pd, nx, ny, nz, x, p, rx_out, accumulate, abs_mode, partials);
    PSPS_LAUNCH_CHECK();
    return MBIR_OK;
}

int penalty_blocks(int64_t npix) {
    int64_t b = cdiv(npix, kThreads);
    return (int)(b < 1024 ? (b < 1 ? 1 : b) : 1024);
}

}  // namespace psps
