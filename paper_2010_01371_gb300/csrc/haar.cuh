#pragma once
#include "common.cuh"

namespace psps {

// n x n images (nz = 1; n a power of two <= 2048) or n^3 volumes (nz = n,
// a power of two <= 256).
bool haar_supported(int nx, int ny, int nz = 1);
// coef = U (pre .* in) with detail / low-pass coefficients multiplied by
// scale (if given); channel c uses |U| when bit c of abs_mask is set.
// nz > 1 selects the 3-D transform of n^3 volumes.
mbir_status haar_forward(int n, int channels, const float *in, float *coef, const float *pre, const float *scale,
                         unsigned abs_mask, cudaStream_t s, int nz = 1);
// out = post .* (U^T coef); coef is used as scratch (its low-pass block is
// overwritten).
mbir_status haar_inverse(int n, int channels, float *coef, float *out, const float *post, unsigned abs_mask,
                         cudaStream_t s, int nz = 1);
// out = post .* U^T (scale .* U (pre .* in)) (pre, post nullable); tmp is a
// (image size) * channels scratch.
mbir_status haar_apply(int n, int channels, const float *in, float *tmp, float *out, const float *pre,
                       const float *post, const float *scale, unsigned abs_mask, cudaStream_t s, int nz = 1);

}  // namespace psps
