// Launchers of the templated model kernels for one material count NM; each is
// explicitly instantiated in its own translation unit (model_inst.cu built
// with PSPS_MODEL_NM = 1..4 and PSPS_MODEL_ROWS = 0 / 1), the channel bound
// CM in {1, 2, 4, 8} is chosen inside.
#pragma once
#include "model.cuh"

namespace psps {

// Smallest channel bound CM in {1, 2, 4, 8} with nc <= CM.
inline int channel_bound(int nc) { return nc <= 1 ? 1 : nc <= 2 ? 2 : nc <= 4 ? 4 : 8; }

// Data term and SPS numerators, rays independent (model_grad_kernel).
template <int NM>
void model_grad_nm(SpecDev sp, int64_t n_rays, const float *l, const float *y, const float *gamma, float *g,
                   float *kappa, dfloat *partials, int nblocks, size_t smem, cudaStream_t s);
// The same with rays coupled along detector rows (model_grad_rows_kernel).
template <int NM>
void model_rows_nm(SpecDev sp, int64_t n_rays, const float *l, const float *y, const float *gamma, float *g,
                   float *kappa, dfloat *partials, int nblocks, size_t smem, cudaStream_t s);
// One fused line-search evaluation (ls_fused_kernel, mode 0 or 1).
template <int NM>
void ls_fused_nm(SpecDev sp, int64_t n_rays, const float *l, const float *q, const float *y, DevLS *ls, LsCfg cfg,
                 int mode, int last, dfloat *partials, int nblocks, size_t smem, cudaStream_t s);
// The same with rays coupled along detector rows (ls_rows_kernel).
template <int NM>
void ls_rows_nm(SpecDev sp, int64_t n_rays, const float *l, const float *q, const float *y, DevLS *ls, LsCfg cfg,
                int mode, int last, dfloat *partials, int nblocks, size_t smem, cudaStream_t s);

#define PSPS_MODEL_EXTERN(NM)                                                                                     \
    extern template void model_grad_nm<NM>(SpecDev, int64_t, const float *, const float *, const float *, float *, \
                                           float *, dfloat *, int, size_t, cudaStream_t);                         \
    extern template void model_rows_nm<NM>(SpecDev, int64_t, const float *, const float *, const float *, float *, \
                                           float *, dfloat *, int, size_t, cudaStream_t);                         \
    extern template void ls_fused_nm<NM>(SpecDev, int64_t, const float *, const float *, const float *, DevLS *,   \
                                         LsCfg, int, int, dfloat *, int, size_t, cudaStream_t);                    \
    extern template void ls_rows_nm<NM>(SpecDev, int64_t, const float *, const float *, const float *, DevLS *,    \
                                        LsCfg, int, int, dfloat *, int, size_t, cudaStream_t);
PSPS_MODEL_EXTERN(1)
PSPS_MODEL_EXTERN(2)
PSPS_MODEL_EXTERN(3)
PSPS_MODEL_EXTERN(4)
#undef PSPS_MODEL_EXTERN

}  // namespace psps
