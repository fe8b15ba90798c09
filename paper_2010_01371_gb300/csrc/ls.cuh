// Device-side state and control of the line search (see psps.cu), shared by
// the fused evaluation kernels in model.cu.
#pragma once
#include "common.cuh"

namespace psps {

struct DevLS {
    double phi0, R0, pRx, pRp;  // phi(0) and the penalty's quadratic in alpha
    double alpha;               // point to evaluate / accepted step
    double best_a, best_f;      // last Newton point (halving starts below it)
    double a_prev;              // step accepted in the previous iteration
    int done, nonfinite, it;
    unsigned ticket;            // arrival counter of the last-block reductions
};

struct LsCfg {
    int n_ls, n_halve;
    double alpha_max, trust;
    float z_min;
};

constexpr int kMaxHalve = 8;

// Last-block arrival: thread 0 of every block makes its partial sums visible
// and takes a ticket; the block that draws the last ticket gets true (no
// waiting anywhere).
__device__ inline bool last_block_arrive(unsigned *ticket) {
    __shared__ bool last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned t = atomicAdd(ticket, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (last) __threadfence();
    return last;
}

// One Newton evaluation (phi, phi', phi'' data sums; bad = rays outside the
// domain) at ls->alpha; the last one decides acceptance.
__device__ inline void ls_newton_control(DevLS *ls, double fd, double f1d, double f2d, double bad, int last,
                                         const LsCfg &cfg) {
    const double a = ls->alpha;
    const double f = bad > 0 ? INFINITY : fd + ls->R0 + a * ls->pRx + 0.5 * a * a * ls->pRp;
    const double f1 = f1d + ls->pRx + a * ls->pRp;
    const double f2 = f2d + ls->pRp;
    const bool finite = isfinite(f) && isfinite(f1) && isfinite(f2);
    if (!last) {
        double an;
        if (!finite) {
            an = a / cfg.trust;
        } else if (f2 > 0) {
            an = a - f1 / f2;
            if (an < a / cfg.trust) an = a / cfg.trust;
            if (an > a * cfg.trust) an = a * cfg.trust;
        } else {
            an = a;
        }
        if (an > cfg.alpha_max) an = cfg.alpha_max;
        ls->alpha = an;
    } else {
        // accept the last evaluated alpha unless phi rose above phi(0)
        ls->best_a = a;
        ls->best_f = f;
        if (isfinite(f) && f <= ls->phi0) {
            ls->done = 1;
        } else if (cfg.n_halve == 0) {
            ls->alpha = 0.0;
            ls->done = 1;
        }
    }
}

// Halving candidates alpha_k = best_a / 2^k, k = 1..nh, evaluated together:
// the first with phi <= phi(0) is taken, else alpha = 0.
__device__ inline void ls_halve_control(DevLS *ls, const double *fk, const double *badk, int nh) {
    double a = ls->best_a;
    for (int k = 0; k < nh; ++k) {
        a *= 0.5;
        const double f = badk[k] > 0 ? INFINITY : fk[k] + ls->R0 + a * ls->pRx + 0.5 * a * a * ls->pRp;
        if (isfinite(f) && f <= ls->phi0) {
            ls->alpha = a;
            ls->done = 1;
            return;
        }
    }
    ls->alpha = 0.0;
    ls->done = 1;
}

}  // namespace psps
