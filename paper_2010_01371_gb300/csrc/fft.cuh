#pragma once
#include "common.cuh"

namespace psps {

bool fft_supported(int n);

// 2-D FFT filter for images [channels][ny][nx]:
//   out = m0 .* Re( IDFT( spec .* DFT(m0 .* in) ) )
// with a real spectrum spec[ky][kx] (m0 nullable).  Z is an
// nx*ny*channels complex scratch buffer.
struct FftPlan {
    int nx = 0, ny = 0;
    DBuf<float2> twx, twy;
    mbir_status init(int nx, int ny);
    // Z = DFT(in) (unnormalised, complex [channels][ny][nx]).
    mbir_status forward(int channels, const float *in, float2 *Z, cudaStream_t s) const;
    // out = post .* Re(IDFT(Z)) (normalised by 1/(nx ny)); Z is overwritten.
    mbir_status inverse(int channels, float2 *Z, float *out, const float *post, cudaStream_t s) const;
    mbir_status filter(int channels, const float *in, float2 *Z, float *out, const float *m0, const float *spec,
                       cudaStream_t s) const;
};

}  // namespace psps
