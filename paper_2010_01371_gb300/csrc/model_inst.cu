// Explicit instantiation of the model-kernel launchers for one material count
// (PSPS_MODEL_NM) and one family (PSPS_MODEL_ROWS: 0 rays independent, 1 rays
// coupled along detector rows).  The build compiles this file once per
// (count, family) pair so that the kernel variants compile in parallel;
// compiled without the macros it instantiates nothing.
#include "model_inst.cuh"
#include "model_kernels.cuh"

#if defined(PSPS_MODEL_NM) && defined(PSPS_MODEL_ROWS)

namespace psps {

#if PSPS_MODEL_ROWS == 0

template <int NM>
void model_grad_nm(SpecDev sp, int64_t n_rays, const float *l, const float *y, const float *gamma, float *g,
                   float *kappa, dfloat *partials, int nblocks, size_t smem, cudaStream_t s) {
    switch (channel_bound(sp.nc)) {
        case 1: model_grad_kernel<NM, 1><<<nblocks, kModelThreads, smem, s>>>(sp, n_rays, l, y, gamma, g, kappa, partials); break;
        case 2: model_grad_kernel<NM, 2><<<nblocks, kModelThreads, smem, s>>>(sp, n_rays, l, y, gamma, g, kappa, partials); break;
        case 4: model_grad_kernel<NM, 4><<<nblocks, kModelThreads, smem, s>>>(sp, n_rays, l, y, gamma, g, kappa, partials); break;
        default: model_grad_kernel<NM, 8><<<nblocks, kModelThreads, smem, s>>>(sp, n_rays, l, y, gamma, g, kappa, partials); break;
    }
}

template <int NM, int CM>
static void ls_fused_cm(SpecDev sp, int64_t n_rays, const float *l, const float *q, const float *y, DevLS *ls,
                        LsCfg cfg, int mode, int last, dfloat *partials, int nblocks, size_t smem, cudaStream_t s) {
    if (mode == 0)
        ls_fused_kernel<NM, CM, 0><<<nblocks, kModelThreads, smem, s>>>(sp, n_rays, l, q, y, ls, cfg, last, partials);
    else
        ls_fused_kernel<NM, CM, 1><<<nblocks, kModelThreads, smem, s>>>(sp, n_rays, l, q, y, ls, cfg, last, partials);
}

template <int NM>
void ls_fused_nm(SpecDev sp, int64_t n_rays, const float *l, const float *q, const float *y, DevLS *ls, LsCfg cfg,
                 int mode, int last, dfloat *partials, int nblocks, size_t smem, cudaStream_t s) {
    switch (channel_bound(sp.nc)) {
        case 1: ls_fused_cm<NM, 1>(sp, n_rays, l, q, y, ls, cfg, mode, last, partials, nblocks, smem, s); break;
        case 2: ls_fused_cm<NM, 2>(sp, n_rays, l, q, y, ls, cfg, mode, last, partials, nblocks, smem, s); break;
        case 4: ls_fused_cm<NM, 4>(sp, n_rays, l, q, y, ls, cfg, mode, last, partials, nblocks, smem, s); break;
        default: ls_fused_cm<NM, 8>(sp, n_rays, l, q, y, ls, cfg, mode, last, partials, nblocks, smem, s); break;
    }
}

template void model_grad_nm<PSPS_MODEL_NM>(SpecDev, int64_t, const float *, const float *, const float *, float *,
                                           float *, dfloat *, int, size_t, cudaStream_t);
template void ls_fused_nm<PSPS_MODEL_NM>(SpecDev, int64_t, const float *, const float *, const float *, DevLS *,
                                         LsCfg, int, int, dfloat *, int, size_t, cudaStream_t);

#else

// Shared memory of the row kernels: the spectrum plus per-thread staging
// (counts, weighted residuals and, with correlated noise, one more column).
template <int NM, int CM>
static void model_rows_cm(SpecDev sp, int64_t n, const float *l, const float *y, const float *gamma, float *g,
                          float *kappa, dfloat *partials, int nblocks, size_t smem, cudaStream_t s) {
    const size_t sm = smem + sizeof(float) * (sp.noise.a > 0.f ? 3 : 2) * CM * kModelThreads;
    model_grad_rows_kernel<NM, CM><<<nblocks, kModelThreads, sm, s>>>(sp, n, l, y, gamma, g, kappa, partials);
}

template <int NM>
void model_rows_nm(SpecDev sp, int64_t n_rays, const float *l, const float *y, const float *gamma, float *g,
                   float *kappa, dfloat *partials, int nblocks, size_t smem, cudaStream_t s) {
    switch (channel_bound(sp.nc)) {
        case 1: model_rows_cm<NM, 1>(sp, n_rays, l, y, gamma, g, kappa, partials, nblocks, smem, s); break;
        case 2: model_rows_cm<NM, 2>(sp, n_rays, l, y, gamma, g, kappa, partials, nblocks, smem, s); break;
        case 4: model_rows_cm<NM, 4>(sp, n_rays, l, y, gamma, g, kappa, partials, nblocks, smem, s); break;
        default: model_rows_cm<NM, 8>(sp, n_rays, l, y, gamma, g, kappa, partials, nblocks, smem, s); break;
    }
}

template <int NM, int CM>
static void ls_rows_cm(SpecDev sp, int64_t n, const float *l, const float *q, const float *y, DevLS *ls, LsCfg cfg,
                       int mode, int last, dfloat *partials, int nblocks, size_t smem, cudaStream_t s) {
    const size_t sm = smem + sizeof(float) * (mode == 0 ? 3 : 1) * CM * kModelThreads;
    if (mode == 0)
        ls_rows_kernel<NM, CM, 0><<<nblocks, kModelThreads, sm, s>>>(sp, n, l, q, y, ls, cfg, last, partials);
    else
        ls_rows_kernel<NM, CM, 1><<<nblocks, kModelThreads, sm, s>>>(sp, n, l, q, y, ls, cfg, last, partials);
}

template <int NM>
void ls_rows_nm(SpecDev sp, int64_t n_rays, const float *l, const float *q, const float *y, DevLS *ls, LsCfg cfg,
                int mode, int last, dfloat *partials, int nblocks, size_t smem, cudaStream_t s) {
    switch (channel_bound(sp.nc)) {
        case 1: ls_rows_cm<NM, 1>(sp, n_rays, l, q, y, ls, cfg, mode, last, partials, nblocks, smem, s); break;
        case 2: ls_rows_cm<NM, 2>(sp, n_rays, l, q, y, ls, cfg, mode, last, partials, nblocks, smem, s); break;
        case 4: ls_rows_cm<NM, 4>(sp, n_rays, l, q, y, ls, cfg, mode, last, partials, nblocks, smem, s); break;
        default: ls_rows_cm<NM, 8>(sp, n_rays, l, q, y, ls, cfg, mode, last, partials, nblocks, smem, s); break;
    }
}

template void model_rows_nm<PSPS_MODEL_NM>(SpecDev, int64_t, const float *, const float *, const float *, float *,
                                           float *, dfloat *, int, size_t, cudaStream_t);
template void ls_rows_nm<PSPS_MODEL_NM>(SpecDev, int64_t, const float *, const float *, const float *, DevLS *,
                                        LsCfg, int, int, dfloat *, int, size_t, cudaStream_t);

#endif

}  // namespace psps

#endif
