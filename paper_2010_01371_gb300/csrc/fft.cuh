#pragma once
#include "common.cuh"

namespace psps {

bool fft_supported(int n);

// 2-D / 3-D FFT filter for images [channels][nz][ny][nx] (nz = 1: 2-D):
//   out = post .* Re( IDFT( spec .* DFT(pre .* in) ) )
// with a real spectrum spec[kz][ky][kx] (pre, post nullable).  Z is an
// nx*ny*nz*channels complex scratch buffer.
struct FftPlan {
    int nx = 0, ny = 0, nz = 1;
    DBuf<float2> twx, twy, twz;
    mbir_status init(int nx, int ny, int nz = 1);
    mbir_status run(int axis, int mode, int channels, const float *rin, float2 *Z, float *rout, const float *pre_post,
                    const float *spec, cudaStream_t s) const;
    // Z = DFT(in) (unnormalised, complex [channels][nz][ny][nx]).
    mbir_status forward(int channels, const float *in, float2 *Z, cudaStream_t s) const;
    // out = post .* Re(IDFT(Z)) (normalised by 1/(nx ny nz)); Z is overwritten.
    mbir_status inverse(int channels, float2 *Z, float *out, const float *post, cudaStream_t s) const;
    mbir_status filter(int channels, const float *in, float2 *Z, float *out, const float *pre, const float *post,
                       const float *spec, cudaStream_t s) const;
};

}  // namespace psps
