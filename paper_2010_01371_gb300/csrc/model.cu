// Polyenergetic forward model (Eq. 1 with B -> S, A -> Q or QA), the PWLS data
// term (Eq. 3, Sigma_y = diag(max(y,1))), the SPS gradient and curvature
// numerators per ray (Eqs. 5-11) and the line-search terms, all per ray.
//
// Per ray i with material line integrals l_m:
//   z_E = sum_m Q[E][m] l_m,  t_E = exp(-z_E),  y_bar_c = sum_E S[c][E] t_E
//   r_c = y_bar_c - y_c,  w_c = 1/max(y_c, 1)
//   data term        1/2 sum_c w_c r_c^2                       (double-float sum)
//   gradient num.    g_m = -sum_E Q[E][m] t_E v_E,  v_E = sum_c S[c][E] w_c r_c
//   curvature        eta_E = sum_c S[c][E] w_c sigma_c (sigma_c = sum_E S[c][E]),
//                    rho_E = v_E - eta_E t_E   (Eq. 10 with the current t where
//                    the paper prints x^(n)), u = max(1, t_E),
//                    c_E = max(0, 2 eta_E u^2 + rho_E u): the largest second
//                    derivative of 1/2 eta e^{-2z} + rho e^{-z} on z >= min(0, z^n)
//   curvature num.   kappa_m = sum_E Q[E][m] gamma_E c_E,  gamma_E = sum_m Q[E][m] gamma_m
// Exponentials and per-ray sums run in FP32 (exp(-z) as exp2f(-z log2 e));
// the objective and line-search sums over rays are double-float reductions.
// With a detector blur B (outer operator B S) or correlated noise (a
// tridiagonal W = Sigma_y^-1 along detector rows) the kernels work on row
// segments with halo rays so that B, B^T and W act on shared-memory copies.
#include <cmath>
#include <type_traits>
#include <vector>

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

// Blurred residual r = B y0 - y: weighted residual qw = w r (if qw) and the
// data term 1/2 sum w r^2 (block partials); ybar = B y0 when asked.
__global__ void __launch_bounds__(kModelThreads)
    blur_resid_kernel(SpecDev sp, int64_t n_rays, const float *__restrict__ y0, const float *__restrict__ y,
                      float *__restrict__ qw, float *__restrict__ ybar, dfloat *__restrict__ partials) {
    dfloat obj{0.f, 0.f};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_rays; i += (int64_t)gridDim.x * blockDim.x)
        for (int c = 0; c < sp.nc; ++c) {
            const float yb = blur_at(sp.blur, y0 + (int64_t)c * n_rays, i, +1);
            if (ybar) ybar[(int64_t)c * n_rays + i] = yb;
            if (!y) continue;
            const float yc = y[(int64_t)c * n_rays + i];
            const float w = 1.f / fmaxf(yc, 1.f);
            const float r = yb - yc;
            if (qw) qw[(int64_t)c * n_rays + i] = w * r;
            df_add(obj, 0.5f * w * r * r);
        }
    if (partials) {
        dfloat v[1] = {obj};
        block_sum_store<1>(v, partials);
    }
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
    constexpr int NV = MODE == 0 ? 3 : 1;                       // values per channel and ray
    float *buf = sh + (sp.ne * sp.nm + sp.nc * sp.ne + sp.nc);  // [NV][CM][blockDim]
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

__global__ void forward_model_kernel(SpecDev sp, int64_t n_rays, const float *__restrict__ l, float *__restrict__ ybar) {
    extern __shared__ float sh[];
    load_spec(sp, sh);
    const float *Q = sh;
    const float *S = sh + sp.ne * sp.nm;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_rays; i += (int64_t)gridDim.x * blockDim.x) {
        float lm[4];
        for (int m = 0; m < sp.nm; ++m) lm[m] = l[(int64_t)m * n_rays + i];
        float yb[kMaxC];
        for (int c = 0; c < sp.nc; ++c) yb[c] = 0.f;
        for (int e = 0; e < sp.ne; ++e) {
            float z = 0.f;
            for (int m = 0; m < sp.nm; ++m) z = fmaf(Q[e * sp.nm + m], lm[m], z);
            const float t = transmission(z);
            for (int c = 0; c < sp.nc; ++c) yb[c] = fmaf(S[c * sp.ne + e], t, yb[c]);
        }
        for (int c = 0; c < sp.nc; ++c) ybar[(int64_t)c * n_rays + i] = yb[c];
    }
}

// FP64 per-ray set-up of the preconditioner build: D from the data and the
// Fisher blocks F_i = J^T W J, J[c][m] = sum_E S[c][E] t_E Q[E][m].
// Standard CT (one energy, one channel): t = y / S.  Otherwise t_E =
// exp(-Q[E][0] l_w) with l_w from 10 Gauss-Newton steps (from 0, clamped
// at >= 0) on the single-material (water, material 0) PWLS misfit.
__global__ void fisher_kernel(int nm, int ne, int nc, const double *__restrict__ Q, const double *__restrict__ S,
                              int64_t n_rays, const float *__restrict__ y, float *__restrict__ F) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_rays) return;
    double yc[kMaxC], w[kMaxC];
    for (int c = 0; c < nc; ++c) {
        yc[c] = y[(int64_t)c * n_rays + i];
        w[c] = 1.0 / fmax(yc[c], 1.0);
    }
    double J[kMaxC][4];
    if (ne == 1 && nc == 1 && nm == 1) {
        const double t = yc[0] / S[0];
        J[0][0] = S[0] * t * Q[0];
    } else {
        double lw = 0.0;
        for (int it = 0; it < 10; ++it) {
            double yb[kMaxC], d[kMaxC];
            for (int c = 0; c < nc; ++c) yb[c] = d[c] = 0.0;
            for (int e = 0; e < ne; ++e) {
                const double q = Q[e * nm];
                const double t = exp(-q * lw);
                for (int c = 0; c < nc; ++c) {
                    yb[c] += S[c * ne + e] * t;
                    d[c] -= S[c * ne + e] * q * t;
                }
            }
            double gs = 0.0, hs = 0.0;
            for (int c = 0; c < nc; ++c) {
                gs += w[c] * (yb[c] - yc[c]) * d[c];
                hs += w[c] * d[c] * d[c];
            }
            const double step = hs > 0 ? gs / hs : 0.0;
            lw = fmax(lw - step, 0.0);
        }
        for (int c = 0; c < nc; ++c)
            for (int m = 0; m < nm; ++m) J[c][m] = 0.0;
        for (int e = 0; e < ne; ++e) {
            const double t = exp(-Q[e * nm] * lw);
            for (int c = 0; c < nc; ++c) {
                const double st = S[c * ne + e] * t;
                for (int m = 0; m < nm; ++m) J[c][m] += st * Q[e * nm + m];
            }
        }
    }
    int k = 0;
    for (int a = 0; a < nm; ++a)
        for (int b = a; b < nm; ++b, ++k) {
            double v = 0.0;
            for (int c = 0; c < nc; ++c) v += w[c] * J[c][a] * J[c][b];
            F[(int64_t)k * n_rays + i] = (float)v;
        }
}

size_t spec_smem(SpecDev sp) { return sizeof(float) * (size_t)(sp.ne * sp.nm + sp.nc * sp.ne + sp.nc); }

}  // namespace

// Smallest channel bound CM in {1, 2, 4, 8} with nc <= CM.
inline int channel_bound(int nc) { return nc <= 1 ? 1 : nc <= 2 ? 2 : nc <= 4 ? 4 : 8; }

template <int NM, int CM>
void model_grad_launch(SpecDev sp, int64_t n_rays, const float *l, const float *y, const float *gamma, float *g,
                       float *kappa, dfloat *partials, int nblocks, size_t smem, cudaStream_t s) {
    model_grad_kernel<NM, CM><<<nblocks, kModelThreads, smem, s>>>(sp, n_rays, l, y, gamma, g, kappa, partials);
}

template <int NM>
void model_grad_launch_nm(SpecDev sp, int64_t n_rays, const float *l, const float *y, const float *gamma, float *g,
                          float *kappa, dfloat *partials, int nblocks, size_t smem, cudaStream_t s) {
    switch (channel_bound(sp.nc)) {
        case 1: model_grad_launch<NM, 1>(sp, n_rays, l, y, gamma, g, kappa, partials, nblocks, smem, s); break;
        case 2: model_grad_launch<NM, 2>(sp, n_rays, l, y, gamma, g, kappa, partials, nblocks, smem, s); break;
        case 4: model_grad_launch<NM, 4>(sp, n_rays, l, y, gamma, g, kappa, partials, nblocks, smem, s); break;
        default: model_grad_launch<NM, 8>(sp, n_rays, l, y, gamma, g, kappa, partials, nblocks, smem, s); break;
    }
}

// Calls F::template run<NM, CM>() for the material count and channel bound
// of the spectrum.
template <class F>
mbir_status dispatch_nm_cm(const SpecDev &sp, F &&f) {
    const int cm = channel_bound(sp.nc);
    auto with_cm = [&](auto nm_tag) {
        constexpr int NM = decltype(nm_tag)::value;
        switch (cm) {
            case 1: f.template run<NM, 1>(); break;
            case 2: f.template run<NM, 2>(); break;
            case 4: f.template run<NM, 4>(); break;
            default: f.template run<NM, 8>(); break;
        }
    };
    switch (sp.nm) {
        case 1: with_cm(std::integral_constant<int, 1>{}); break;
        case 2: with_cm(std::integral_constant<int, 2>{}); break;
        case 3: with_cm(std::integral_constant<int, 3>{}); break;
        case 4: with_cm(std::integral_constant<int, 4>{}); break;
        default: return fail(MBIR_ERR_ARG, "n_mat %d unsupported", sp.nm);
    }
    PSPS_LAUNCH_CHECK();
    return MBIR_OK;
}

struct BlurModelLaunch {
    SpecDev sp;
    int64_t n;
    const float *l, *y, *gamma;
    float *g, *kappa;
    dfloat *partials;
    int nblocks;
    size_t smem;
    cudaStream_t s;
    template <int NM, int CM>
    void run() {
        const size_t sm = smem + sizeof(float) * (sp.noise.a > 0.f ? 3 : 2) * CM * kModelThreads;
        model_grad_rows_kernel<NM, CM><<<nblocks, kModelThreads, sm, s>>>(sp, n, l, y, gamma, g, kappa, partials);
    }
};

mbir_status launch_model_grad(SpecDev sp, int64_t n_rays, const float *l, const float *y, const float *gamma,
                              float *g, float *kappa, dfloat *partials, int nblocks, cudaStream_t s) {
    const size_t smem = spec_smem(sp);
    if (row_coupled(sp)) {
        BlurModelLaunch L{sp, n_rays, l, y, gamma, g, kappa, partials, nblocks, smem, s};
        return dispatch_nm_cm(sp, L);
    }
    switch (sp.nm) {
        case 1: model_grad_launch_nm<1>(sp, n_rays, l, y, gamma, g, kappa, partials, nblocks, smem, s); break;
        case 2: model_grad_launch_nm<2>(sp, n_rays, l, y, gamma, g, kappa, partials, nblocks, smem, s); break;
        case 3: model_grad_launch_nm<3>(sp, n_rays, l, y, gamma, g, kappa, partials, nblocks, smem, s); break;
        case 4: model_grad_launch_nm<4>(sp, n_rays, l, y, gamma, g, kappa, partials, nblocks, smem, s); break;
        default: return fail(MBIR_ERR_ARG, "n_mat %d unsupported", sp.nm);
    }
    PSPS_LAUNCH_CHECK();
    return MBIR_OK;
}

template <int NM, int CM>
void ls_fused_launch(SpecDev sp, int64_t n_rays, const float *l, const float *q, const float *y, DevLS *ls, LsCfg cfg,
                     int mode, int last, dfloat *partials, int nblocks, size_t smem, cudaStream_t s) {
    if (mode == 0)
        ls_fused_kernel<NM, CM, 0><<<nblocks, kModelThreads, smem, s>>>(sp, n_rays, l, q, y, ls, cfg, last, partials);
    else
        ls_fused_kernel<NM, CM, 1><<<nblocks, kModelThreads, smem, s>>>(sp, n_rays, l, q, y, ls, cfg, last, partials);
}

template <int NM>
void ls_fused_launch_nm(SpecDev sp, int64_t n_rays, const float *l, const float *q, const float *y, DevLS *ls,
                        LsCfg cfg, int mode, int last, dfloat *partials, int nblocks, size_t smem, cudaStream_t s) {
    switch (channel_bound(sp.nc)) {
        case 1: ls_fused_launch<NM, 1>(sp, n_rays, l, q, y, ls, cfg, mode, last, partials, nblocks, smem, s); break;
        case 2: ls_fused_launch<NM, 2>(sp, n_rays, l, q, y, ls, cfg, mode, last, partials, nblocks, smem, s); break;
        case 4: ls_fused_launch<NM, 4>(sp, n_rays, l, q, y, ls, cfg, mode, last, partials, nblocks, smem, s); break;
        default: ls_fused_launch<NM, 8>(sp, n_rays, l, q, y, ls, cfg, mode, last, partials, nblocks, smem, s); break;
    }
}

struct BlurLsLaunch {
    SpecDev sp;
    int64_t n;
    const float *l, *q, *y;
    DevLS *ls;
    LsCfg cfg;
    dfloat *partials;
    int mode, last, nblocks;
    size_t smem;
    cudaStream_t s;
    template <int NM, int CM>
    void run() {
        const size_t sm = smem + sizeof(float) * (mode == 0 ? 3 : 1) * CM * kModelThreads;
        if (mode == 0)
            ls_rows_kernel<NM, CM, 0><<<nblocks, kModelThreads, sm, s>>>(sp, n, l, q, y, ls, cfg, last, partials);
        else
            ls_rows_kernel<NM, CM, 1><<<nblocks, kModelThreads, sm, s>>>(sp, n, l, q, y, ls, cfg, last, partials);
    }
};

mbir_status launch_ls_fused(SpecDev sp, int64_t n_rays, const float *l, const float *q, const float *y, DevLS *ls,
                            LsCfg cfg, int mode, int last, dfloat *partials, int nblocks, cudaStream_t s) {
    const size_t smem = spec_smem(sp);
    if (row_coupled(sp)) {
        BlurLsLaunch L{sp, n_rays, l, q, y, ls, cfg, partials, mode, last, nblocks, smem, s};
        return dispatch_nm_cm(sp, L);
    }
    switch (sp.nm) {
        case 1: ls_fused_launch_nm<1>(sp, n_rays, l, q, y, ls, cfg, mode, last, partials, nblocks, smem, s); break;
        case 2: ls_fused_launch_nm<2>(sp, n_rays, l, q, y, ls, cfg, mode, last, partials, nblocks, smem, s); break;
        case 3: ls_fused_launch_nm<3>(sp, n_rays, l, q, y, ls, cfg, mode, last, partials, nblocks, smem, s); break;
        case 4: ls_fused_launch_nm<4>(sp, n_rays, l, q, y, ls, cfg, mode, last, partials, nblocks, smem, s); break;
        default: return fail(MBIR_ERR_ARG, "n_mat %d unsupported", sp.nm);
    }
    PSPS_LAUNCH_CHECK();
    return MBIR_OK;
}

mbir_status launch_forward_model(SpecDev sp, int64_t n_rays, const float *l, float *ybar, cudaStream_t s,
                                 float *y0) {
    if (sp.blur.r > 0) {
        if (!y0) return fail(MBIR_ERR_ARG, "the blurred forward model needs a scratch buffer");
        forward_model_kernel<<<model_blocks(n_rays), kModelThreads, spec_smem(sp), s>>>(sp, n_rays, l, y0);
        PSPS_LAUNCH_CHECK();
        blur_resid_kernel<<<model_blocks(n_rays), kModelThreads, 0, s>>>(sp, n_rays, y0, nullptr, nullptr, ybar,
                                                                        nullptr);
        PSPS_LAUNCH_CHECK();
        return MBIR_OK;
    }
    forward_model_kernel<<<model_blocks(n_rays), kModelThreads, spec_smem(sp), s>>>(sp, n_rays, l, ybar);
    PSPS_LAUNCH_CHECK();
    return MBIR_OK;
}

mbir_status launch_fisher_blocks(const mbmd_spectrum *spec, int64_t n_rays, const float *y, float *F, cudaStream_t s) {
    DBuf<double> q, sbuf;
    PSPS_TRY(q.alloc((size_t)spec->n_energy * spec->n_mat));
    PSPS_TRY(sbuf.alloc((size_t)spec->n_chan * spec->n_energy));
    PSPS_CUDA(cudaMemcpyAsync(q.p, spec->hQ, sizeof(double) * q.n, cudaMemcpyHostToDevice, s));
    PSPS_CUDA(cudaMemcpyAsync(sbuf.p, spec->hS, sizeof(double) * sbuf.n, cudaMemcpyHostToDevice, s));
    fisher_kernel<<<(unsigned)cdiv(n_rays, 128), 128, 0, s>>>(spec->n_mat, spec->n_energy, spec->n_chan, q.p, sbuf.p,
                                                            n_rays, y, F);
    PSPS_LAUNCH_CHECK();
    PSPS_CUDA(cudaStreamSynchronize(s));  // q, sbuf are freed on return
    return MBIR_OK;
}

__global__ void model_fill_ones_kernel(float *p, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = 1.f;
}

mbir_status fill_ones(float *p, int64_t n, cudaStream_t s) {
    const int64_t b = cdiv(n, 256);
    model_fill_ones_kernel<<<(unsigned)(b < 4096 ? (b < 1 ? 1 : b) : 4096), 256, 0, s>>>(p, n);
    PSPS_LAUNCH_CHECK();
    return MBIR_OK;
}

}  // namespace psps

using namespace psps;

extern "C" mbir_status mbmd_spectrum_create(int n_mat, int n_energy, int n_chan, const double *Q, const double *S,
                                            mbmd_spectrum **out) {
    if (!out || !Q || !S) return fail(MBIR_ERR_ARG, "mbmd_spectrum_create: null argument");
    *out = nullptr;
    if (n_mat < 1 || n_mat > 4 || n_energy < 1 || n_energy > kMaxE || n_chan < 1 || n_chan > kMaxC)
        return fail(MBIR_ERR_ARG, "mbmd_spectrum_create: sizes n_mat=%d n_energy=%d n_chan=%d out of range", n_mat,
                    n_energy, n_chan);
    for (int i = 0; i < n_energy * n_mat; ++i)
        if (!std::isfinite(Q[i]) || Q[i] < 0) return fail(MBIR_ERR_ARG, "mbmd_spectrum_create: Q must be finite and >= 0");
    for (int i = 0; i < n_chan * n_energy; ++i)
        if (!std::isfinite(S[i]) || S[i] < 0) return fail(MBIR_ERR_ARG, "mbmd_spectrum_create: S must be finite and >= 0");
    mbmd_spectrum *sp = new mbmd_spectrum();
    sp->n_mat = n_mat;
    sp->n_energy = n_energy;
    sp->n_chan = n_chan;
    sp->hQ = new double[n_energy * n_mat];
    sp->hS = new double[n_chan * n_energy];
    std::vector<float> h(n_energy * n_mat + n_chan * n_energy + n_chan);
    for (int i = 0; i < n_energy * n_mat; ++i) {
        sp->hQ[i] = Q[i];
        h[i] = (float)Q[i];
    }
    for (int c = 0; c < n_chan; ++c) {
        double sig = 0.0;
        for (int e = 0; e < n_energy; ++e) {
            sp->hS[c * n_energy + e] = S[c * n_energy + e];
            h[n_energy * n_mat + c * n_energy + e] = (float)S[c * n_energy + e];
            sig += S[c * n_energy + e];
        }
        h[n_energy * n_mat + n_chan * n_energy + c] = (float)sig;
    }
    mbir_status st = sp->qs.alloc(h.size());
    if (st != MBIR_OK) {
        delete sp;
        return st;
    }
    cudaError_t e = cudaMemcpy(sp->qs.p, h.data(), sizeof(float) * h.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        delete sp;
        return fail(MBIR_ERR_CUDA, "mbmd_spectrum_create: %s", cudaGetErrorString(e));
    }
    *out = sp;
    return MBIR_OK;
}

extern "C" mbir_status mbmd_spectrum_destroy(mbmd_spectrum *s) {
    delete s;
    return MBIR_OK;
}

extern "C" mbir_status mbmd_forward_model(const mbmd_spectrum *spec, const float *l, float *ybar, int64_t n_rays,
                                          mbir_stream s) {
    if (!spec || !l || !ybar || n_rays < 0) return fail(MBIR_ERR_ARG, "mbmd_forward_model: bad argument");
    if (n_rays == 0) return MBIR_OK;
    if (spec->blur_r == 0) return launch_forward_model(spec_dev(spec), n_rays, l, ybar, (cudaStream_t)s);
    if (n_rays % spec->blur_row) return fail(MBIR_ERR_ARG, "mbmd_forward_model: n_rays is not a multiple of the blur row");
    DBuf<float> y0;
    PSPS_TRY(y0.alloc((size_t)spec->n_chan * n_rays));
    PSPS_TRY(launch_forward_model(spec_dev(spec), n_rays, l, ybar, (cudaStream_t)s, y0.p));
    PSPS_CUDA(cudaStreamSynchronize((cudaStream_t)s));  // y0 is released on return
    return MBIR_OK;
}

extern "C" mbir_status mbmd_spectrum_set_blur(mbmd_spectrum *spec, int radius, int row, const double *taps) {
    if (!spec) return fail(MBIR_ERR_ARG, "mbmd_spectrum_set_blur: spec is null");
    if (radius < 0 || radius > 3) return fail(MBIR_ERR_ARG, "mbmd_spectrum_set_blur: radius %d outside 0..3", radius);
    if (radius > 0 && (!taps || row < 1))
        return fail(MBIR_ERR_ARG, "mbmd_spectrum_set_blur: taps must be given and row must be >= 1");
    float b[7] = {};
    for (int k = 0; radius > 0 && k < 2 * radius + 1; ++k) {
        if (!std::isfinite(taps[k]) || taps[k] < 0)
            return fail(MBIR_ERR_ARG, "mbmd_spectrum_set_blur: taps must be finite and >= 0");
        b[k] = (float)taps[k];
    }
    if (radius > 0 && spec->noise_a > 0.f && row != spec->noise_row)
        return fail(MBIR_ERR_ARG, "mbmd_spectrum_set_blur: row differs from the correlated noise's row");
    spec->blur_r = radius;
    spec->blur_row = radius > 0 ? row : 1;
    for (int k = 0; k < 7; ++k) spec->blur_b[k] = b[k];
    return MBIR_OK;
}

extern "C" mbir_status mbmd_spectrum_set_noise(mbmd_spectrum *spec, double a, int row) {
    if (!spec) return fail(MBIR_ERR_ARG, "mbmd_spectrum_set_noise: spec is null");
    if (!std::isfinite(a) || a < 0.0 || a >= 0.99)
        return fail(MBIR_ERR_ARG, "mbmd_spectrum_set_noise: correlation %g outside [0, 0.99)", a);
    if (a > 0.0 && row < 2) return fail(MBIR_ERR_ARG, "mbmd_spectrum_set_noise: row must be >= 2");
    if (a > 0.0 && spec->blur_r > 0 && row != spec->blur_row)
        return fail(MBIR_ERR_ARG, "mbmd_spectrum_set_noise: row differs from the blur's row");
    spec->noise_a = (float)a;
    spec->noise_row = a > 0.0 ? row : 1;
    return MBIR_OK;
}

namespace {
// Scratch for the stateless model calls: l, g and kappa sinograms, gamma and
// partials.
struct ModelScratch {
    DBuf<float> l, g, kap, gam, ones;
    DBuf<dfloat> part;
};


mbir_status data_term(mbir_plan *plan, const mbmd_spectrum *spec, const float *x_or_l, const float *y, int64_t n_rays,
                      float *grad, double *objective, cudaStream_t s, float *curv = nullptr) {
    if (!spec || !x_or_l || !y || n_rays < 1) return fail(MBIR_ERR_ARG, "mbmd: bad argument");
    if (plan && n_rays != plan->n_rays)
        return fail(MBIR_ERR_ARG, "mbmd: n_rays %lld does not match the plan (%lld)", (long long)n_rays,
                    (long long)plan->n_rays);
    if (plan && spec->n_mat > plan->n_mat_max) return fail(MBIR_ERR_ARG, "mbmd: n_mat exceeds the plan's n_mat_max");
    if (n_rays % spec->blur_row || n_rays % spec->noise_row)
        return fail(MBIR_ERR_ARG, "mbmd: n_rays is not a multiple of the blur / noise row");
    ModelScratch sc;
    const int nm = spec->n_mat;
    const float *l = x_or_l;
    if (plan) {
        PSPS_TRY(sc.l.alloc((size_t)nm * n_rays));
        PSPS_TRY(project(plan, x_or_l, sc.l.p, nm, s));
        l = sc.l.p;
    }
    const int nb = model_blocks(n_rays);
    PSPS_TRY(sc.part.alloc(nb));
    float *g = nullptr;
    if (grad) {
        if (plan) {
            PSPS_TRY(sc.g.alloc((size_t)nm * n_rays));
            g = sc.g.p;
        } else {
            g = grad;
        }
    }
    // plain-SPS curvature numerators: gamma_m = [A 1]_m (projection domain: 1)
    float *kap = nullptr;
    if (curv) {
        PSPS_TRY(sc.gam.alloc((size_t)nm * n_rays));
        if (plan) {
            PSPS_TRY(sc.ones.alloc((size_t)nm * plan->n_pix));
            PSPS_TRY(fill_ones(sc.ones.p, (int64_t)nm * plan->n_pix, s));
            PSPS_TRY(project(plan, sc.ones.p, sc.gam.p, nm, s));
            PSPS_TRY(sc.kap.alloc((size_t)nm * n_rays));
            kap = sc.kap.p;
        } else {
            PSPS_TRY(fill_ones(sc.gam.p, (int64_t)nm * n_rays, s));
            kap = curv;
        }
    }
    PSPS_TRY(launch_model_grad(spec_dev(spec), n_rays, l, y, curv ? sc.gam.p : nullptr, g, kap, sc.part.p, nb, s));
    if (objective) PSPS_TRY(reduce_partials(sc.part.p, nb, 1, objective, 0, s));
    if (grad && plan) PSPS_TRY(backproject(plan, g, grad, nm, 0, s));
    if (curv && plan) PSPS_TRY(backproject(plan, kap, curv, nm, 0, s));
    PSPS_CUDA(cudaStreamSynchronize(s));  // scratch is released on return
    return MBIR_OK;
}
}  // namespace

extern "C" mbir_status mbmd_objective(mbir_plan *plan, const mbmd_spectrum *spec, const float *x_or_l, const float *y,
                                      int64_t n_rays, double *objective, mbir_stream s) {
    if (!objective) return fail(MBIR_ERR_ARG, "mbmd_objective: objective is null");
    return data_term(plan, spec, x_or_l, y, n_rays, nullptr, objective, (cudaStream_t)s);
}

extern "C" mbir_status mbmd_gradient(mbir_plan *plan, const mbmd_spectrum *spec, const float *x_or_l, const float *y,
                                     int64_t n_rays, float *grad, double *objective, mbir_stream s) {
    if (!grad) return fail(MBIR_ERR_ARG, "mbmd_gradient: grad is null");
    return data_term(plan, spec, x_or_l, y, n_rays, grad, objective, (cudaStream_t)s);
}

extern "C" mbir_status mbmd_curvature(mbir_plan *plan, const mbmd_spectrum *spec, const float *x_or_l, const float *y,
                                      int64_t n_rays, float *curv, mbir_stream s) {
    if (!curv) return fail(MBIR_ERR_ARG, "mbmd_curvature: curv is null");
    return data_term(plan, spec, x_or_l, y, n_rays, nullptr, nullptr, (cudaStream_t)s, curv);
}
