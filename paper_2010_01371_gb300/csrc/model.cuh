// Per-ray spectral forward model, PWLS data term, SPS numerators and
// line-search terms (model.cu).
#pragma once
#include "common.cuh"
#include "ls.cuh"

namespace psps {

// Detector blur of the outer operator (B S): [B v]_i = sum_k b[k + r] v_{i+k},
// k = -r..r, within rows of `row` consecutive rays (zero past the row ends).
struct BlurDev {
    int r = 0, row = 1;
    float b[7] = {};
};

// Correlated noise: W = Sigma_y^-1 = D^-1/2 C^-1 D^-1/2 with the tridiagonal
// inverse of the row correlation C[j][k] = a^|j-k| (a = 0: diagonal).
struct NoiseDev {
    float a = 0.f;
    int row = 1;
};

struct SpecDev {
    int nm, ne, nc;
    const float *qs;  // Q[ne][nm], S[nc][ne], sigma[nc] (sigma_c = sum_E S[c][E])
    BlurDev blur;     // r = 0: no blur (b[0] = 1, the identity)
    NoiseDev noise;
};

inline SpecDev spec_dev(const mbmd_spectrum *s) {
    SpecDev d{s->n_mat, s->n_energy, s->n_chan, s->qs.p, {}, {}};
    d.blur.r = s->blur_r;
    d.blur.row = s->blur_row;
    for (int k = 0; k < 7; ++k) d.blur.b[k] = s->blur_b[k];
    if (d.blur.r == 0) d.blur.b[0] = 1.f;
    d.noise.a = s->noise_a;
    d.noise.row = s->noise_row;
    return d;
}

// Rays couple along detector rows (a blur or correlated noise): the model
// and line-search kernels then work on row segments with halo rays.
inline bool row_coupled(const SpecDev &sp) { return sp.blur.r > 0 || sp.noise.a > 0.f; }

constexpr int kModelThreads = 256;
constexpr int kModelMaxBlocks = 2048;  // grid-stride; partial sums per block

// About two rays per thread, at most kModelMaxBlocks blocks.
inline int model_blocks(int64_t n) {
    int64_t b = cdiv(n, 2 * kModelThreads);
    return (int)(b < kModelMaxBlocks ? (b < 1 ? 1 : b) : kModelMaxBlocks);
}

// data term partials (1 per block); g, kappa optional ([nm][n_rays]).
// gamma: per-ray gamma_m = [A |M| 1]_m ([nm][n_rays]) for kappa.  With a
// detector blur or correlated noise the same quantities come from row
// segments with halos (one kernel, no scratch).
mbir_status launch_model_grad(SpecDev sp, int64_t n_rays, const float *l, const float *y, const float *gamma,
                              float *g, float *kappa, dfloat *partials, int nblocks, cudaStream_t s);
// Fused line-search evaluation: mode 0 evaluates phi, phi', phi'' at
// ls->alpha and its last block runs the Newton control; mode 1 (skipped when
// the search is done) evaluates the n_halve halving candidates at once and
// its last block picks the step.  partials: 2 kMaxHalve per block.  With a
// detector blur or correlated noise the same evaluation runs on row segments
// with halos (one kernel, no scratch).
mbir_status launch_ls_fused(SpecDev sp, int64_t n_rays, const float *l, const float *q, const float *y, DevLS *ls,
                            LsCfg cfg, int mode, int last, dfloat *partials, int nblocks, cudaStream_t s);
// ybar = B S exp(-Q l); with a blur, y0 ([n_chan][n_rays]) holds the unblurred
// counts.
mbir_status launch_forward_model(SpecDev sp, int64_t n_rays, const float *l, float *ybar, cudaStream_t s,
                                 float *y0 = nullptr);
// Per-ray Fisher blocks F_i = Q^T D S^T W S D Q (upper triangle, packed
// [nm(nm+1)/2][n_rays]) with D = y / I0 (one energy/channel) or the water fit.
mbir_status launch_fisher_blocks(const mbmd_spectrum *spec, int64_t n_rays, const float *y, float *F,
                                 cudaStream_t s);

}  // namespace psps
