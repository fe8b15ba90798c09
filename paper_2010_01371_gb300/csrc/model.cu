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

#include "model_inst.cuh"
#include "model_kernels.cuh"

namespace psps {
namespace {

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

mbir_status launch_model_grad(SpecDev sp, int64_t n_rays, const float *l, const float *y, const float *gamma,
                              float *g, float *kappa, dfloat *partials, int nblocks, cudaStream_t s) {
    const size_t smem = spec_smem(sp);
    auto run = [&](auto fn) { fn(sp, n_rays, l, y, gamma, g, kappa, partials, nblocks, smem, s); };
    const bool rows = row_coupled(sp);
    switch (sp.nm) {
        case 1: rows ? run(model_rows_nm<1>) : run(model_grad_nm<1>); break;
        case 2: rows ? run(model_rows_nm<2>) : run(model_grad_nm<2>); break;
        case 3: rows ? run(model_rows_nm<3>) : run(model_grad_nm<3>); break;
        case 4: rows ? run(model_rows_nm<4>) : run(model_grad_nm<4>); break;
        default: return fail(MBIR_ERR_ARG, "n_mat %d unsupported", sp.nm);
    }
    PSPS_LAUNCH_CHECK();
    return MBIR_OK;
}

mbir_status launch_ls_fused(SpecDev sp, int64_t n_rays, const float *l, const float *q, const float *y, DevLS *ls,
                            LsCfg cfg, int mode, int last, dfloat *partials, int nblocks, cudaStream_t s) {
    const size_t smem = spec_smem(sp);
    auto run = [&](auto fn) { fn(sp, n_rays, l, q, y, ls, cfg, mode, last, partials, nblocks, smem, s); };
    const bool rows = row_coupled(sp);
    switch (sp.nm) {
        case 1: rows ? run(ls_rows_nm<1>) : run(ls_fused_nm<1>); break;
        case 2: rows ? run(ls_rows_nm<2>) : run(ls_fused_nm<2>); break;
        case 3: rows ? run(ls_rows_nm<3>) : run(ls_fused_nm<3>); break;
        case 4: rows ? run(ls_rows_nm<4>) : run(ls_fused_nm<4>); break;
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
    if (grad && plan) {
        plan->tile_fine = nm;   // gradient numerators: terms to 2^-12 of the tile transpose's unit
        const mbir_status r = backproject(plan, g, grad, nm, 0, s);
        plan->tile_fine = 0;
        PSPS_TRY(r);
    }
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
