#pragma once
#include "common.cuh"

namespace psps {

bool haar_supported(int nx, int ny);
// coef = U (pre .* in) with detail / low-pass coefficients multiplied by
// scale (if given); channel c uses |U| when bit c of abs_mask is set.
mbir_status haar_forward(int n, int channels, const float *in, float *coef, const float *pre, const float *scale,
                         unsigned abs_mask, cudaStream_t s);
// out = post .* (U^T coef); coef is used as scratch (its low-pass block is
// overwritten).
mbir_status haar_inverse(int n, int channels, float *coef, float *out, const float *post, unsigned abs_mask,
                         cudaStream_t s);
// out = m0 .* U^T (scale .* U (m0 .* in)); tmp is an n*n*channels scratch.
mbir_status haar_apply(int n, int channels, const float *in, float *tmp, float *out, const float *m0,
                       const float *scale, unsigned abs_mask, cudaStream_t s);

}  // namespace psps
