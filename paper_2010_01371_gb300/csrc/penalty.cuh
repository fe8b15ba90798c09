#pragma once
#include "common.cuh"

namespace psps {

struct PenaltyDev {
    int nm;
    float beta[16];  // beta[k * 4 + k']
};

int penalty_blocks(int64_t npix);
// rx_out (+)= R x (or |R| x with abs_mode); partials (3 per block, nullable):
// sum x.Rx, sum p.Rx, sum p.Rp.  x or p may be null (their terms are zero).
mbir_status launch_penalty(const PenaltyDev &pd, int nx, int ny, int nz, const float *x, const float *p, float *rx_out,
                           int accumulate, int abs_mode, dfloat *partials, int nblocks, cudaStream_t s);

}  // namespace psps
