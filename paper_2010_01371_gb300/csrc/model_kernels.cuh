// Templated per-ray kernels of the spectral model (model.cu): the data term
// with SPS numerators and the fused line-search evaluation, plain and with
// rays coupled along detector rows.  Each material count is instantiated in
// its own translation unit (model_inst.cu compiled once per count and
// family), so the 96 kernel variants compile in parallel.
#pragma once
#include <cmath>

#include "model.cuh"

namespace psps {
namespace {

constexpr int kMaxE = 256, kMaxC = 8;

__device__ __forceinline__ void load_spec(const SpecDev &sp, float *sh) {
    const int n = sp.ne * sp.nm + sp.nc * sp.ne + sp.nc;
    for (int i = threadIdx.x; i < n; i += blockDim.x) sh[i] = sp.qs[i];
    __syncthreads();
}

// Channel counts are compile-time upper bounds CM (1, 2, 4, 8) with the
// actual count nc <= CM tested inside fully unrolled loops, so the per-channel
// accumulators stay in registers.
// t = exp(-z) through the base-2 exponential: exp2f(-z log2 e), with
// log2 e = 1 / ln 2.  exp2f maps to the SFU's base-2 exponential (2 ulp);
// the product adds a relative error of about |z| 2^-24 to t.
__device__ __forceinline__ float transmission(float z) { return exp2f(z * -1.4426950408889634f); }

template <int NM, int CM>
__global__ void __launch_bounds__(kModelThreads)
    model_grad_kernel(SpecDev sp, int64_t n_rays, const float *__restrict__ l, const float *__restrict__ y,
                      const float *__restrict__ gamma, float *__restrict__ g, float *__restrict__ kappa,
                      dfloat *__restrict__ partials) {
    extern __shared__ float sh[];
    load_spec(sp, sh);
    const float *Q = sh;
    const float *S = sh + sp.ne * NM;
    const float *sig = S + sp.nc * sp.ne;
    const int nc = sp.nc, ne = sp.ne;
    dfloat obj{0.f, 0.f};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_rays; i += (int64_t)gridDim.x * blockDim.x) {
        float lm[NM];
#pragma unroll
        for (int m = 0; m < NM; ++m) lm[m] = l[(int64_t)m * n_rays + i];
        float yb[CM];
#pragma unroll
        for (int c = 0; c < CM; ++c) yb[c] = 0.f;
        for (int e = 0; e < ne; ++e) {
            float z = 0.f;
#pragma unroll
            for (int m = 0; m < NM; ++m) z = fmaf(Q[e * NM + m], lm[m], z);
            const float t = transmission(z);
#pragma unroll
            for (int c = 0; c < CM; ++c)
                if (c < nc) yb[c] = fmaf(S[c * ne + e], t, yb[c]);
        }
        float wr[CM], ws[CM];
#pragma unroll
        for (int c = 0; c < CM; ++c) {
            wr[c] = ws[c] = 0.f;
            if (c < nc) {
                const float yc = y[(int64_t)c * n_rays + i];
                const float w = 1.f / fmaxf(yc, 1.f);
                const float r = yb[c] - yc;
                wr[c] = w * r;
                df_add(obj, 0.5f * wr[c] * r);
                ws[c] = w * sig[c];
            }
        }
        if (g || kappa) {
            float gm[NM], km[NM], gam[NM];
#pragma unroll
            for (int m = 0; m < NM; ++m) {
                gm[m] = km[m] = 0.f;
                gam[m] = kappa ? gamma[(int64_t)m * n_rays + i] : 0.f;
            }
            for (int e = 0; e < ne; ++e) {
                float z = 0.f, gE = 0.f;
#pragma unroll
                for (int m = 0; m < NM; ++m) {
                    z = fmaf(Q[e * NM + m], lm[m], z);
                    gE = fmaf(Q[e * NM + m], gam[m], gE);
                }
                const float t = transmission(z);
                float v = 0.f, eta = 0.f;
#pragma unroll
                for (int c = 0; c < CM; ++c)
                    if (c < nc) {
                        v = fmaf(S[c * ne + e], wr[c], v);
                        eta = fmaf(S[c * ne + e], ws[c], eta);
                    }
                const float tv = t * v;
                float cE = 0.f;
                if (kappa) {
                    const float rho = v - eta * t;
                    const float u = fmaxf(1.f, t);
                    cE = fmaxf(0.f, (2.f * eta * u + rho) * u);
                }
#pragma unroll
                for (int m = 0; m < NM; ++m) {
                    gm[m] = fmaf(-Q[e * NM + m], tv, gm[m]);
                    km[m] = fmaf(Q[e * NM + m], gE * cE, km[m]);
                }
            }
#pragma unroll
            for (int m = 0; m < NM; ++m) {
                if (g) g[(int64_t)m * n_rays + i] = gm[m];
                if (kappa) kappa[(int64_t)m * n_rays + i] = km[m];
            }
        }
    }
    dfloat v[1] = {obj};
    block_sum_store<1>(v, partials);
}

template <int NM, int CM, int MODE>
__global__ void __launch_bounds__(kModelThreads)
    ls_fused_kernel(SpecDev sp, int64_t n_rays, const float *__restrict__ l, const float *__restrict__ q,
                    const float *__restrict__ y, DevLS *ls, LsCfg cfg, int last, dfloat *__restrict__ partials) {
    if (MODE == 1 && ls->done) return;  // same value for every block
    extern __shared__ float sh[];
    load_spec(sp, sh);
    const float *Q = sh;
    const float *S = sh + sp.ne * NM;
    const int nc = sp.nc, ne = sp.ne;
    const int nh = cfg.n_halve < kMaxHalve ? cfg.n_halve : kMaxHalve;
    constexpr int NACC = MODE == 0 ? 4 : 2 * kMaxHalve;
    dfloat acc[NACC];
#pragma unroll
    for (int k = 0; k < NACC; ++k) acc[k] = dfloat{0.f, 0.f};
    if constexpr (MODE == 0) {
        const float alpha = (float)ls->alpha;
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_rays;
             i += (int64_t)gridDim.x * blockDim.x) {
            float la[NM], qm[NM];
            float zlo = 3.0e38f;
#pragma unroll
            for (int m = 0; m < NM; ++m) {
                qm[m] = q[(int64_t)m * n_rays + i];
                la[m] = fmaf(alpha, qm[m], l[(int64_t)m * n_rays + i]);
            }
            float yb[CM], d1[CM], d2[CM];
#pragma unroll
            for (int c = 0; c < CM; ++c) yb[c] = d1[c] = d2[c] = 0.f;
            for (int e = 0; e < ne; ++e) {
                float z = 0.f, dz = 0.f;
#pragma unroll
                for (int m = 0; m < NM; ++m) {
                    z = fmaf(Q[e * NM + m], la[m], z);
                    dz = fmaf(Q[e * NM + m], qm[m], dz);
                }
                zlo = fminf(zlo, z);
                const float t = transmission(z);
                const float tdz = t * dz;
#pragma unroll
                for (int c = 0; c < CM; ++c)
                    if (c < nc) {
                        const float s = S[c * ne + e];
                        yb[c] = fmaf(s, t, yb[c]);
                        d1[c] = fmaf(-s, tdz, d1[c]);
                        d2[c] = fmaf(s, tdz * dz, d2[c]);
                    }
            }
            float f = 0.f, f1 = 0.f, f2 = 0.f;
#pragma unroll
            for (int c = 0; c < CM; ++c)
                if (c < nc) {
                    const float yc = y[(int64_t)c * n_rays + i];
                    const float w = 1.f / fmaxf(yc, 1.f);
                    const float r = yb[c] - yc;
                    f = fmaf(0.5f * w * r, r, f);
                    f1 = fmaf(w * r, d1[c], f1);
                    f2 = fmaf(w, fmaf(d1[c], d1[c], r * d2[c]), f2);
                }
            df_add(acc[0], f);
            df_add(acc[1], f1);
            df_add(acc[2], f2);
            if (!(zlo >= cfg.z_min)) df_add(acc[3], 1.f);
        }
        block_sum_store<4>(acc, partials);
    } else {
        const double a0 = ls->best_a;
        float alphas[kMaxHalve];
        double ak = a0;
#pragma unroll
        for (int k = 0; k < kMaxHalve; ++k) {
            ak *= 0.5;
            alphas[k] = (float)ak;
        }
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_rays;
             i += (int64_t)gridDim.x * blockDim.x) {
            float lm[NM], qm[NM], yc[CM], wh[CM];
#pragma unroll
            for (int m = 0; m < NM; ++m) {
                qm[m] = q[(int64_t)m * n_rays + i];
                lm[m] = l[(int64_t)m * n_rays + i];
            }
#pragma unroll
            for (int c = 0; c < CM; ++c) {
                yc[c] = c < nc ? y[(int64_t)c * n_rays + i] : 0.f;
                wh[c] = 0.5f / fmaxf(yc[c], 1.f);
            }
#pragma unroll
            for (int k = 0; k < kMaxHalve; ++k) {
                if (k >= nh) break;
                float yb[CM];
#pragma unroll
                for (int c = 0; c < CM; ++c) yb[c] = 0.f;
                float zlo = 3.0e38f;
                for (int e = 0; e < ne; ++e) {
                    float z = 0.f;
#pragma unroll
                    for (int m = 0; m < NM; ++m) z = fmaf(Q[e * NM + m], fmaf(alphas[k], qm[m], lm[m]), z);
                    zlo = fminf(zlo, z);
                    const float t = transmission(z);
#pragma unroll
                    for (int c = 0; c < CM; ++c)
                        if (c < nc) yb[c] = fmaf(S[c * ne + e], t, yb[c]);
                }
                float f = 0.f;
#pragma unroll
                for (int c = 0; c < CM; ++c)
                    if (c < nc) {
                        const float r = yb[c] - yc[c];
                        f = fmaf(wh[c] * r, r, f);
                    }
                df_add(acc[k], f);
                if (!(zlo >= cfg.z_min)) df_add(acc[kMaxHalve + k], 1.f);
            }
        }
        block_sum_store<NACC>(acc, partials);
    }
    if (!last_block_arrive(&ls->ticket)) return;
    const int nb = gridDim.x;
    if constexpr (MODE == 0) {
        double sums[4];
        block_sum_partials_k<4>(partials, nb, sums);
        if (threadIdx.x == 0) {
            ls_newton_control(ls, sums[0], sums[1], sums[2], sums[3], last, cfg);
            ls->ticket = 0;
        }
    } else {
        double sums[2 * kMaxHalve];
        block_sum_partials_k<2 * kMaxHalve>(partials, nb, sums);
        if (threadIdx.x == 0) {
            ls_halve_control(ls, sums, sums + kMaxHalve, nh);
            ls->ticket = 0;
        }
    }
}

// ---------------------------------------------------------------- blur
// With a detector blur B in the outer operator (B S, Eq. 1) the mean counts
// of a ray mix the unblurred counts of its row neighbours, and the SPS
// quantities of Eqs. 8 and 10 become, per ray i and energy E,
//   eta = sum_c S[c][E] sigma_c [B^T (w_c .* B 1)]_i
//   rho = sum_c S[c][E] [B^T (w_c .* r_c)]_i - eta t_E,   r = B S t - y.
// The blurred path runs in passes: unblurred counts per ray, then the
// blurred residual and its weights, then the numerators from B^T of those.

// [B v]_i (dir = +1) or [B^T v]_i (dir = -1), one channel, within the row.
__device__ __forceinline__ float blur_at(const BlurDev &B, const float *__restrict__ v, int64_t i, int dir) {
    const int j = (int)(i % B.row);
    float s = 0.f;
    for (int k = -B.r; k <= B.r; ++k) {
        const int jj = j + dir * k;
        if (jj >= 0 && jj < B.row) s = fmaf(B.b[k + B.r], v[i + dir * k], s);
    }
    return s;
}

// (B 1)_j at row position j (rows of `row` rays).
__device__ __forceinline__ float blur_ones(const BlurDev &B, int row, int j) {
    float s = 0.f;
    for (int k = -B.r; k <= B.r; ++k)
        if (j + k >= 0 && j + k < row) s += B.b[k + B.r];
    return s;
}

// w^1/2 = max(y, 1)^-1/2 of one ray's counts.
__device__ __forceinline__ float sqrt_weight(float y) { return sqrtf(1.f / fmaxf(y, 1.f)); }

// [W v]_j for one row of cells with W = D^-1/2 C^-1 D^-1/2: v holds the
// values of consecutive cells (shared memory), tid this cell, j its position
// in the row, yc the channel's counts (global) and i this cell's ray.  C^-1 is
// (1 / (1 - a^2)) times 1 (row ends) or 1 + a^2 on the diagonal and -a next
// to it.
__device__ __forceinline__ float noise_apply(const NoiseDev &N, int row, const float *__restrict__ v, int tid, int j,
                                             const float *__restrict__ yc, int64_t i) {
    const bool lo = j > 0, hi = j + 1 < row;
    const float a = N.a;
    const float s0 = sqrt_weight(yc[i]);
    float acc = ((lo && hi) ? fmaf(a, a, 1.f) : 1.f) * s0 * v[tid];
    if (lo) acc = fmaf(-a * sqrt_weight(yc[i - 1]), v[tid - 1], acc);
    if (hi) acc = fmaf(-a * sqrt_weight(yc[i + 1]), v[tid + 1], acc);
    return s0 * acc / fmaf(-a, a, 1.f);
}

// eta weight of one channel at ray i (row position j):
// [B^T (|W| (B 1))]_i, with |W| = diag(w) without correlated noise; y is the
// channel's counts (global memory), the row's neighbours of i are read from it.
__device__ __forceinline__ float coupled_eta_weight(const SpecDev &sp, int row, const float *__restrict__ y,
                                                    int64_t i, int j) {
    const BlurDev &B = sp.blur;
    const float a = sp.noise.a;
    float s = 0.f;
    for (int k = -B.r; k <= B.r; ++k) {
        const int jj = j - k;
        if (jj < 0 || jj >= row) continue;
        const int64_t p = i - k;
        float v;
        if (a > 0.f) {
            const bool lo = jj > 0, hi = jj + 1 < row;
            const float s0 = sqrt_weight(y[p]);
            float acc = ((lo && hi) ? fmaf(a, a, 1.f) : 1.f) * s0 * blur_ones(B, row, jj);
            if (lo) acc = fmaf(a * sqrt_weight(y[p - 1]), blur_ones(B, row, jj - 1), acc);
            if (hi) acc = fmaf(a * sqrt_weight(y[p + 1]), blur_ones(B, row, jj + 1), acc);
            v = s0 * acc / fmaf(-a, a, 1.f);
        } else {
            v = blur_ones(B, row, jj) / fmaxf(y[p], 1.f);
        }
        s = fmaf(B.b[k + B.r], v, s);
    }
    return s;
}

// Data term and numerators with rays coupled along detector rows (a blur B
// in the outer operator and / or correlated noise W), in one kernel: a block
// takes segments of T = blockDim - 2H rays with H = 2 rb + rn halo rays on
// each side (rb the blur radius, rn = 1 with correlated noise).
// Phase 1: unblurred counts y0 of every ray of the extended segment (shared
// memory).  Phase 2: blurred residual r = B y0 - y (rays within rb + rn of
// the segment).  Phase 2b: weighted residual qw = W r (rays within rb; with
// diagonal noise qw = w r comes with phase 2) and the data term
// 1/2 r^T W r of the segment's own rays.  Phase 3 (own rays): u_c =
// [B^T qw_c]_i replaces w_c r_c and sigma_c [B^T (|W| B 1)]_i replaces
// w_c sigma_c in the numerators, with a second pass over the energies.
// [B v] and [B^T v] at thread tid's ray from a shared-memory column of
// consecutive rays (j = the ray's position in its row of `row` rays).
__device__ __forceinline__ float blur_col(const BlurDev &Bd, int row, const float *__restrict__ col, int tid, int j) {
    float s = 0.f;
    for (int k = -Bd.r; k <= Bd.r; ++k) {
        const int jj = j + k;
        if (jj >= 0 && jj < row) s = fmaf(Bd.b[k + Bd.r], col[tid + k], s);
    }
    return s;
}

__device__ __forceinline__ float blur_colT(const BlurDev &Bd, int row, const float *__restrict__ col, int tid, int j) {
    float s = 0.f;
    for (int k = -Bd.r; k <= Bd.r; ++k) {
        const int jj = j - k;
        if (jj >= 0 && jj < row) s = fmaf(Bd.b[k + Bd.r], col[tid - k], s);
    }
    return s;
}

template <int NM, int CM>
__global__ void __launch_bounds__(kModelThreads)
    model_grad_rows_kernel(SpecDev sp, int64_t n_rays, const float *__restrict__ l, const float *__restrict__ y,
                           const float *__restrict__ gamma, float *__restrict__ g, float *__restrict__ kappa,
                           dfloat *__restrict__ partials) {
    extern __shared__ float sh[];
    load_spec(sp, sh);
    const float *Q = sh;
    const float *S = sh + sp.ne * NM;
    const float *sig = S + sp.nc * sp.ne;
    const int nc = sp.nc, ne = sp.ne;
    const int B = blockDim.x, tid = threadIdx.x;
    const int rb = sp.blur.r, rn = sp.noise.a > 0.f ? 1 : 0, H = 2 * rb + rn, T = B - 2 * H;
    const int row = rb > 0 ? sp.blur.row : sp.noise.row;
    float *y0s = sh + (sp.ne * sp.nm + sp.nc * sp.ne + sp.nc);  // [CM][B] unblurred counts
    float *qws = y0s + CM * B;                                  // [CM][B] weighted residuals
    float *rs = qws + CM * B;                                   // [CM][B] residuals (rn only)
    const bool grads = g || kappa;
    const int64_t nseg = (n_rays + T - 1) / T;
    dfloat obj{0.f, 0.f};
    for (int64_t seg = blockIdx.x; seg < nseg; seg += gridDim.x) {
        const int64_t i = seg * T - H + tid;
        const bool valid = i >= 0 && i < n_rays;
        const bool own = valid && tid >= H && tid < H + T;
        const int j = valid ? (int)(i % row) : 0;
        float lm[NM];
#pragma unroll
        for (int m = 0; m < NM; ++m) lm[m] = valid ? l[(int64_t)m * n_rays + i] : 0.f;
        {
            float yb[CM];
#pragma unroll
            for (int c = 0; c < CM; ++c) yb[c] = 0.f;
            if (valid)
                for (int e = 0; e < ne; ++e) {
                    float z = 0.f;
#pragma unroll
                    for (int m = 0; m < NM; ++m) z = fmaf(Q[e * NM + m], lm[m], z);
                    const float t = transmission(z);
#pragma unroll
                    for (int c = 0; c < CM; ++c)
                        if (c < nc) yb[c] = fmaf(S[c * ne + e], t, yb[c]);
                }
#pragma unroll
            for (int c = 0; c < CM; ++c)
                if (c < nc) y0s[c * B + tid] = yb[c];
        }
        __syncthreads();
        if (valid && tid >= rb && tid < B - rb) {
            float f = 0.f;
#pragma unroll
            for (int c = 0; c < CM; ++c)
                if (c < nc) {
                    const float yc = y[(int64_t)c * n_rays + i];
                    const float w = 1.f / fmaxf(yc, 1.f);
                    const float rr = blur_col(sp.blur, row, y0s + c * B, tid, j) - yc;
                    if (rn) {
                        rs[c * B + tid] = rr;
                    } else {
                        qws[c * B + tid] = w * rr;
                        f = fmaf(0.5f * w * rr, rr, f);
                    }
                }
            if (!rn && own) df_add(obj, f);
        }
        __syncthreads();
        if (rn) {
            if (valid && tid >= rb + 1 && tid < B - rb - 1) {
                float f = 0.f;
#pragma unroll
                for (int c = 0; c < CM; ++c)
                    if (c < nc) {
                        const float qv = noise_apply(sp.noise, row, rs + c * B, tid, j, y + (int64_t)c * n_rays, i);
                        qws[c * B + tid] = qv;
                        f = fmaf(0.5f * rs[c * B + tid], qv, f);
                    }
                if (own) df_add(obj, f);
            }
            __syncthreads();
        }
        if (grads && own) {
            float gm[NM], km[NM], gam[NM];
#pragma unroll
            for (int m = 0; m < NM; ++m) {
                gm[m] = km[m] = 0.f;
                gam[m] = kappa ? gamma[(int64_t)m * n_rays + i] : 0.f;
            }
            float u[CM], ws[CM];
#pragma unroll
            for (int c = 0; c < CM; ++c) {
                u[c] = ws[c] = 0.f;
                if (c < nc) {
                    u[c] = blur_colT(sp.blur, row, qws + c * B, tid, j);
                    ws[c] = kappa ? sig[c] * coupled_eta_weight(sp, row, y + (int64_t)c * n_rays, i, j) : 0.f;
                }
            }
            for (int e = 0; e < ne; ++e) {
                float z = 0.f, gE = 0.f;
#pragma unroll
                for (int m = 0; m < NM; ++m) {
                    z = fmaf(Q[e * NM + m], lm[m], z);
                    gE = fmaf(Q[e * NM + m], gam[m], gE);
                }
                const float t = transmission(z);
                float v = 0.f, eta = 0.f;
#pragma unroll
                for (int c = 0; c < CM; ++c)
                    if (c < nc) {
                        v = fmaf(S[c * ne + e], u[c], v);
                        eta = fmaf(S[c * ne + e], ws[c], eta);
                    }
                const float tv = t * v;
                float cE = 0.f;
                if (kappa) {
                    const float rho = v - eta * t;
                    const float uh = fmaxf(1.f, t);
                    cE = fmaxf(0.f, (2.f * eta * uh + rho) * uh);
                }
#pragma unroll
                for (int m = 0; m < NM; ++m) {
                    gm[m] = fmaf(-Q[e * NM + m], tv, gm[m]);
                    km[m] = fmaf(Q[e * NM + m], gE * cE, km[m]);
                }
            }
#pragma unroll
            for (int m = 0; m < NM; ++m) {
                if (g) g[(int64_t)m * n_rays + i] = gm[m];
                if (kappa) kappa[(int64_t)m * n_rays + i] = km[m];
            }
        }
        __syncthreads();
    }
    if (partials) {
        dfloat v[1] = {obj};
        block_sum_store<1>(v, partials);
    }
}

// Line search with rays coupled along detector rows (blur and / or
// correlated noise), one kernel per evaluation: a block takes segments of
// T = blockDim - 2H consecutive rays plus H = rb + rn halo rays on each side.
// Every thread evaluates the unblurred counts of one ray of the extended
// segment (and, for the Newton evaluation, their first two alpha-derivatives)
// into shared memory; the rays within rn of the segment blur them along their
// row; the segment's own rays then add the data terms (with correlated noise
// through W applied to the blurred residuals and derivatives of their row
// neighbours) and count the rays that leave the domain z >= z_min.  Partials
// and the last block's control are those of ls_fused_kernel.
template <int NM, int CM, int MODE>
__global__ void __launch_bounds__(kModelThreads)
    ls_rows_kernel(SpecDev sp, int64_t n_rays, const float *__restrict__ l, const float *__restrict__ q,
                   const float *__restrict__ y, DevLS *ls, LsCfg cfg, int last, dfloat *__restrict__ partials) {
    if (MODE == 1 && ls->done) return;  // same value for every block
    extern __shared__ float sh[];
    load_spec(sp, sh);
    const float *Q = sh;
    const float *S = sh + sp.ne * NM;
    const int nc = sp.nc, ne = sp.ne;
    // [NV][CM][blockDim] with NV = 3 values per channel and ray (mode 0) or 1
    float *buf = sh + (sp.ne * sp.nm + sp.nc * sp.ne + sp.nc);
    const int B = blockDim.x, tid = threadIdx.x;
    const int rb = sp.blur.r, rn = sp.noise.a > 0.f ? 1 : 0, H = rb + rn, T = B - 2 * H;
    const int row = rb > 0 ? sp.blur.row : sp.noise.row;
    const int64_t nseg = (n_rays + T - 1) / T;
    const int nh = cfg.n_halve < kMaxHalve ? cfg.n_halve : kMaxHalve;
    constexpr int NACC = MODE == 0 ? 4 : 2 * kMaxHalve;
    dfloat acc[NACC];
#pragma unroll
    for (int k = 0; k < NACC; ++k) acc[k] = dfloat{0.f, 0.f};
    float alphas[kMaxHalve];
    {
        double ak = MODE == 0 ? 0.0 : ls->best_a;
#pragma unroll
        for (int k = 0; k < kMaxHalve; ++k) {
            ak *= 0.5;
            alphas[k] = (float)ak;
        }
    }
    const float alpha = MODE == 0 ? (float)ls->alpha : 0.f;
    for (int64_t seg = blockIdx.x; seg < nseg; seg += gridDim.x) {
        const int64_t i = seg * T - H + tid;
        const bool valid = i >= 0 && i < n_rays;
        const bool own = valid && tid >= H && tid < H + T;
        const bool near = valid && tid >= rb && tid < B - rb;  // blurred values needed here
        const int j = valid ? (int)(i % row) : 0;
        float lm[NM], qm[NM];
#pragma unroll
        for (int m = 0; m < NM; ++m) {
            qm[m] = valid ? q[(int64_t)m * n_rays + i] : 0.f;
            lm[m] = valid ? l[(int64_t)m * n_rays + i] : 0.f;
        }
#pragma unroll
        for (int k = 0; k < (MODE == 0 ? 1 : kMaxHalve); ++k) {
            if (MODE == 1 && k >= nh) break;  // same for every thread
            float v0[CM], v1[CM], v2[CM];
#pragma unroll
            for (int c = 0; c < CM; ++c) v0[c] = v1[c] = v2[c] = 0.f;
            float zlo = 3.0e38f;
            if (valid) {
                const float ak = MODE == 0 ? alpha : alphas[k];
                float la[NM];
#pragma unroll
                for (int m = 0; m < NM; ++m) la[m] = fmaf(ak, qm[m], lm[m]);
                for (int e = 0; e < ne; ++e) {
                    float z = 0.f, dz = 0.f;
#pragma unroll
                    for (int m = 0; m < NM; ++m) {
                        z = fmaf(Q[e * NM + m], la[m], z);
                        if (MODE == 0) dz = fmaf(Q[e * NM + m], qm[m], dz);
                    }
                    zlo = fminf(zlo, z);
                    const float t = transmission(z);
                    const float tdz = t * dz;
#pragma unroll
                    for (int c = 0; c < CM; ++c)
                        if (c < nc) {
                            const float sv = S[c * ne + e];
                            v0[c] = fmaf(sv, t, v0[c]);
                            if (MODE == 0) {
                                v1[c] = fmaf(-sv, tdz, v1[c]);
                                v2[c] = fmaf(sv, tdz * dz, v2[c]);
                            }
                        }
                }
            }
#pragma unroll
            for (int c = 0; c < CM; ++c)
                if (c < nc) {
                    buf[c * B + tid] = v0[c];
                    if (MODE == 0) {
                        buf[(CM + c) * B + tid] = v1[c];
                        buf[(2 * CM + c) * B + tid] = v2[c];
                    }
                }
            if (own && !(zlo >= cfg.z_min)) df_add(acc[MODE == 0 ? 3 : kMaxHalve + k], 1.f);
            __syncthreads();
            // blurred residual and derivatives at the rays within rn of the
            // segment (registers first: the neighbours still read buf)
            float r0[CM], r1[CM], r2[CM], sw[CM];
#pragma unroll
            for (int c = 0; c < CM; ++c) {
                r0[c] = r1[c] = r2[c] = 0.f;
                sw[c] = 0.f;
                if (c < nc && near) {
                    const float yc = y[(int64_t)c * n_rays + i];
                    sw[c] = 1.f / fmaxf(yc, 1.f);
                    r0[c] = blur_col(sp.blur, row, buf + c * B, tid, j) - yc;
                    if (MODE == 0) {
                        r1[c] = blur_col(sp.blur, row, buf + (CM + c) * B, tid, j);
                        r2[c] = blur_col(sp.blur, row, buf + (2 * CM + c) * B, tid, j);
                    }
                }
            }
            if (rn) {
                __syncthreads();
                if (near)
#pragma unroll
                    for (int c = 0; c < CM; ++c)
                        if (c < nc) {
                            buf[c * B + tid] = r0[c];
                            if (MODE == 0) buf[(CM + c) * B + tid] = r1[c];
                        }
                __syncthreads();
            }
            if (own) {
                float f = 0.f, f1 = 0.f, f2 = 0.f;
#pragma unroll
                for (int c = 0; c < CM; ++c)
                    if (c < nc) {
                        // W r and W r' at this ray (diagonal: w r, w r')
                        float wr, wd;
                        if (rn) {
                            const float *yc = y + (int64_t)c * n_rays;
                            wr = noise_apply(sp.noise, row, buf + c * B, tid, j, yc, i);
                            wd = MODE == 0 ? noise_apply(sp.noise, row, buf + (CM + c) * B, tid, j, yc, i) : 0.f;
                        } else {
                            wr = sw[c] * r0[c];
                            wd = sw[c] * r1[c];
                        }
                        f = fmaf(0.5f * r0[c], wr, f);
                        if (MODE == 0) {
                            f1 = fmaf(r1[c], wr, f1);
                            f2 = fmaf(r1[c], wd, fmaf(r2[c], wr, f2));
                        }
                    }
                if (MODE == 0) {
                    df_add(acc[0], f);
                    df_add(acc[1], f1);
                    df_add(acc[2], f2);
                } else {
                    df_add(acc[k], f);
                }
            }
            __syncthreads();
        }
    }
    block_sum_store<NACC>(acc, partials);
    if (!last_block_arrive(&ls->ticket)) return;
    const int nb = gridDim.x;
    if constexpr (MODE == 0) {
        double sums[4];
        block_sum_partials_k<4>(partials, nb, sums);
        if (threadIdx.x == 0) {
            ls_newton_control(ls, sums[0], sums[1], sums[2], sums[3], last, cfg);
            ls->ticket = 0;
        }
    } else {
        double sums[2 * kMaxHalve];
        block_sum_partials_k<2 * kMaxHalve>(partials, nb, sums);
        if (threadIdx.x == 0) {
            ls_halve_control(ls, sums, sums + kMaxHalve, nh);
            ls->ticket = 0;
        }
    }
}

}  // namespace
}  // namespace psps
