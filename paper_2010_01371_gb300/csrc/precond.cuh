#pragma once
#include "common.cuh"
#include "fft.cuh"
#include "penalty.cuh"

struct psps_precond {
    int kind = PSPS_PRECOND_NONE;
    int nm = 1;
    bool image = true;       // false: projection-domain unknowns [nm][n_rays]
    int nx = 1, ny = 1, nz = 1;  // image grid (nz = 1: 2-D)
    int64_t n = 0;           // unknowns per material
    int sides = 2;           // Fourier / wavelet kinds: M = M0^T C (1) or M0^T C M0 (2); set per kind
    psps::DBuf<float> m0;    // diagonal zero-frequency normalisation (one material)
    psps::DBuf<float> s, s_abs;  // spectra / wavelet-domain scales
    psps::DBuf<float> B, Babs;   // blocks [nm][nm][n]
    psps::DBuf<float> Li, Li_abs;  // cross-material Fourier: per-frequency blocks [nm][nm][n]
    psps::DBuf<float> Hblk;      // built: the (F+R)1_k blocks of Eqs. 30, 53-54, [nm][nm][n]
    psps::DBuf<float> est;       // built: Eq. 18 estimates before the floor ([n] or [nm][nm][n])
    psps::DBuf<float> tmp;       // scratch (n * nm * 2)
    psps::DBuf<float2> Z;        // FFT scratch (n * nm * 2 complex)
    psps::FftPlan fft;
};

namespace psps {
// op(M) for two inputs at once (channels 0: in0 -> out0 with op0, 1: in1 ->
// out1 with op1), used by the iteration for M^T grad and |M|^T curvature.
mbir_status precond_apply(psps_precond *pc, int op, const float *in, float *out, cudaStream_t s);
mbir_status precond_apply2(psps_precond *pc, int op0, const float *in0, float *out0, int op1, const float *in1,
                           float *out1, cudaStream_t s);
}  // namespace psps
