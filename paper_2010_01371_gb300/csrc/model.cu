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
// Exponentials and per-ray sums run in FP32 (expf); the objective and
// line-search sums over rays are double-float reductions.
#include <cmath>
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
            const float t = expf(-z);
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
                const float t = expf(-z);
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
                const float t = expf(-z);
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
                    const float t = expf(-z);
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
            const float t = expf(-z);
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

mbir_status launch_model_grad(SpecDev sp, int64_t n_rays, const float *l, const float *y, const float *gamma,
                              float *g, float *kappa, dfloat *partials, int nblocks, cudaStream_t s) {
    const size_t smem = spec_smem(sp);
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

mbir_status launch_ls_fused(SpecDev sp, int64_t n_rays, const float *l, const float *q, const float *y, DevLS *ls,
                            LsCfg cfg, int mode, int last, dfloat *partials, int nblocks, cudaStream_t s) {
    const size_t smem = spec_smem(sp);
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

mbir_status launch_forward_model(SpecDev sp, int64_t n_rays, const float *l, float *ybar, cudaStream_t s) {
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
    return launch_forward_model(spec_dev(spec), n_rays, l, ybar, (cudaStream_t)s);
}

namespace {
// Scratch for the stateless model calls: l and g sinograms plus partials.
struct ModelScratch {
    DBuf<float> l, g;
    DBuf<dfloat> part;
};

mbir_status data_term(mbir_plan *plan, const mbmd_spectrum *spec, const float *x_or_l, const float *y, int64_t n_rays,
                      float *grad, double *objective, cudaStream_t s) {
    if (!spec || !x_or_l || !y || n_rays < 1) return fail(MBIR_ERR_ARG, "mbmd: bad argument");
    if (plan && n_rays != plan->n_rays)
        return fail(MBIR_ERR_ARG, "mbmd: n_rays %lld does not match the plan (%lld)", (long long)n_rays,
                    (long long)plan->n_rays);
    if (plan && spec->n_mat > plan->n_mat_max) return fail(MBIR_ERR_ARG, "mbmd: n_mat exceeds the plan's n_mat_max");
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
    PSPS_TRY(launch_model_grad(spec_dev(spec), n_rays, l, y, nullptr, g, nullptr, sc.part.p, nb, s));
    if (objective) PSPS_TRY(reduce_partials(sc.part.p, nb, 1, objective, 0, s));
    if (grad && plan) PSPS_TRY(backproject(plan, g, grad, nm, 0, s));
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
