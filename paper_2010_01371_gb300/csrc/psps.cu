// The (preconditioned) SPS iteration (Sec. II-B, II-C) on the GPU.
//
// One iteration, all on the device (optionally replayed as a CUDA graph):
//   [every `reproject_every` iterations: l = A x exactly]
//   per ray:   g = dL/dl, kappa = sum_E Q gamma~_E c_E, data term    (model.cu)
//   G = A^T [g; kappa]  (2 n_mat channels in one backprojection)
//   grad = G_g + R x,   Phi(x) = data + 1/2 x^T R x                    (FP64)
//   grad' = M^T grad,   d' = |M|^T G_kappa + |M|^T |R| |M| 1
//   p' = -grad'/d' (0 where d' = 0),  p = M p',  q = A p
//   step length: 1 (classic SPS), or safeguarded Newton on
//     phi(alpha) = Phi(x + alpha p) from the previous iteration's step length
//     (steps kept within a factor 8; n_ls evaluations; the last evaluated
//     alpha, halved up to n_halve times until phi <= phi(0), else 0), with
//     per-ray exact phi, phi', phi'' and the penalty's exact
//     quadratic in alpha; scalar control runs in one-thread kernels that read
//     the FP64 partial sums, so nothing returns to the host
//   x += alpha p,  l += alpha q
// gamma~ = A |M| 1 generalises gamma = A 1 (Eq. 9) to the operator A M; with
// M = I this is the paper's SPS update (Eq. 7) with the surrogate gradient
// equal to the true gradient at x^n.
#include <cmath>
#include <vector>

#include "model.cuh"
#include "penalty.cuh"
#include "precond.cuh"

namespace psps {
namespace {

constexpr int kThreads = 256;

// phi0 = data + 1/2 x.Rx; records the objective history.
__global__ void ctrl_begin_kernel(DevLS *ls, const dfloat *pobj, int nobj, const dfloat *ppen, int npen,
                                  double *history) {
    const double d = block_sum_partials(pobj, nobj);
    const double xRx = ppen ? block_sum_partials(ppen, npen) : 0.0;
    if (threadIdx.x == 0) {
        ls->R0 = 0.5 * xRx;
        ls->phi0 = d + 0.5 * xRx;
        if (!isfinite(ls->phi0)) ls->nonfinite = 1;
        history[ls->it] = ls->phi0;
    }
}

// penalty terms along p: partials are (x.Rx, p.Rx, p.Rp) blocks
__global__ void ctrl_ls_init_kernel(DevLS *ls, const dfloat *ppen, int npen) {
    double pen[2] = {0.0, 0.0};
    if (ppen) block_sum_partials_k<2>(ppen + npen, npen, pen);
    if (threadIdx.x == 0) {
        ls->pRx = pen[0];
        ls->pRp = pen[1];
        ls->alpha = ls->a_prev > 0 ? ls->a_prev : 1.0;
        ls->best_a = 0.0;
        ls->best_f = INFINITY;
        ls->done = 0;
    }
}

__global__ void set_alpha_one_kernel(DevLS *ls) { ls->alpha = 1.0; }

// p' = -grad'/(d' + dR) where positive, else 0
__global__ void direction_kernel(const float *__restrict__ gp, const float *__restrict__ dp,
                                 const float *__restrict__ dR, float *__restrict__ pp, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float d = dp[i] + (dR ? dR[i] : 0.f);
        pp[i] = d > 0.f ? -gp[i] / d : 0.f;
    }
}

// x += alpha p (clamped at 0 when nonneg), l += alpha q; records alpha
__global__ void update_kernel(DevLS *ls, float *__restrict__ x, const float *__restrict__ p, int64_t nx_tot,
                              float *__restrict__ l, const float *__restrict__ q, int64_t nl_tot, int nonneg,
                              double *alphas) {
    const float a = (float)ls->alpha;
    const int64_t tot = nx_tot > nl_tot ? nx_tot : nl_tot;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += (int64_t)gridDim.x * blockDim.x) {
        if (i < nx_tot) {
            float v = fmaf(a, p[i], x[i]);
            if (nonneg) v = fmaxf(v, 0.f);
            x[i] = v;
        }
        if (l && i < nl_tot) l[i] = fmaf(a, q[i], l[i]);
    }
}

// Records alpha; the next line search starts from it, or below the last
// halving after a failed search.
__global__ void finish_iter_kernel(DevLS *ls, double *alphas, int n_halve) {
    alphas[ls->it] = ls->alpha;
    ls->a_prev = ls->alpha > 0 ? ls->alpha : ls->best_a / (double)(2 << n_halve);
    ls->it += 1;
}

__global__ void reset_counter_kernel(DevLS *ls) {
    ls->it = 0;
    ls->nonfinite = 0;
}

unsigned grid_for(int64_t n) {
    int64_t b = cdiv(n, kThreads);
    return (unsigned)(b > 8192 ? 8192 : (b < 1 ? 1 : b));
}

}  // namespace
}  // namespace psps

using namespace psps;

struct psps_state {
    mbir_plan *plan = nullptr;      // NULL: projection domain
    const mbmd_spectrum *spec = nullptr;
    psps_precond *pc = nullptr;     // NULL: plain SPS
    int nm = 1, nc = 1, flags = 0, reproject_every = 10;
    int64_t n = 0, n_rays = 0;
    bool has_pen = false;
    PenaltyDev pd{};
    LsCfg cfg{3, 8, 1e12, 8.0, -20.0f};
    DBuf<float> x, l, y, gamma, dR, gk, G, gp, dp, pp, p, q;
    SpecDev sd;  // the spectrum (and its blur) as it was at creation
    DBuf<dfloat> part_obj, part_pen, part_ls;
    DBuf<double> history, alphas;
    DBuf<DevLS> ls;
    int nb_model = 1, nb_pen = 1;
    int hist_cap = 0;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};  // [0] plain, [1] with re-projection
    // optional stage timers (events around contiguous regions of one iteration)
    int64_t graph_kernels[2] = {0, 0};  // kernel nodes per captured iteration
    bool graph_marks[2][PSPS_PROF_STAGES] = {};  // stages timed inside each graph
    int64_t launches = 0;                // kernels launched through graph replays
    bool prof = false;
    cudaEvent_t ev[PSPS_PROF_STAGES][2] = {};
    bool recorded[PSPS_PROF_STAGES] = {};
    double prof_ms[PSPS_PROF_STAGES] = {};
    int64_t prof_cnt[PSPS_PROF_STAGES] = {};
    void drop_graphs() {
        for (auto &g : graph)
            if (g) {
                cudaGraphExecDestroy(g);
                g = nullptr;
            }
    }
    ~psps_state() {
        drop_graphs();
        for (auto &e : ev)
            for (auto &x : e)
                if (x) cudaEventDestroy(x);
    }
};

namespace {

// Stage timer: during graph capture the record must be an external event
// node (a plain record in a capturing stream only expresses a dependency).
inline void mark(psps_state *st, int stage, int end, cudaStream_t s) {
    if (!st->prof) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s, &cs);
    if (cs == cudaStreamCaptureStatusActive)
        cudaEventRecordWithFlags(st->ev[stage][end], s, cudaEventRecordExternal);
    else
        cudaEventRecord(st->ev[stage][end], s);
    if (end) st->recorded[stage] = true;
}

mbir_status project_or_copy(psps_state *st, const float *x, float *l, cudaStream_t s) {
    if (st->plan) return project(st->plan, x, l, st->nm, s);
    if (x != l) PSPS_CUDA(cudaMemcpyAsync(l, x, sizeof(float) * st->nm * st->n_rays, cudaMemcpyDeviceToDevice, s));
    return MBIR_OK;
}

// fine: leading channels whose terms the 3-D tile transpose keeps to 2^-12
// of its fixed-point unit
mbir_status backproject_or_copy(psps_state *st, const float *s_, float *x, int ch, cudaStream_t s, int fine = 0) {
    if (st->plan) {
        st->plan->tile_fine = fine;
        const mbir_status r = backproject(st->plan, s_, x, ch, 0, s);
        st->plan->tile_fine = 0;
        return r;
    }
    PSPS_CUDA(cudaMemcpyAsync(x, s_, sizeof(float) * ch * st->n_rays, cudaMemcpyDeviceToDevice, s));
    return MBIR_OK;
}

mbir_status apply_M(psps_state *st, int op, const float *in, float *out, cudaStream_t s) {
    if (!st->pc) {
        if (in != out)
            PSPS_CUDA(cudaMemcpyAsync(out, in, sizeof(float) * st->nm * st->n, cudaMemcpyDeviceToDevice, s));
        return MBIR_OK;
    }
    return precond_apply(st->pc, op, in, out, s);
}

mbir_status penalty_call(psps_state *st, const float *x, const float *p, float *rx_out, int acc, int abs_mode,
                         dfloat *part, cudaStream_t s) {
    const mbir_geometry &g = st->plan->g;
    return launch_penalty(st->pd, g.nx, g.ny, g.kind == MBIR_CONE3D ? g.nz : 1, x, p, rx_out, acc, abs_mode, part,
                          st->nb_pen, s);
}

// One iteration (no host synchronisation).
mbir_status iterate(psps_state *st, bool reproject, cudaStream_t s) {
    const int nm = st->nm;
    const int64_t n = st->n, nr = st->n_rays;
    const SpecDev sp = st->sd;
    if (reproject) {
        mark(st, PSPS_PROF_REPROJECT, 0, s);
        PSPS_TRY(project_or_copy(st, st->x.p, st->l.p, s));
        mark(st, PSPS_PROF_REPROJECT, 1, s);
    }
    // per-ray numerators and the data term
    mark(st, PSPS_PROF_MODEL, 0, s);
    PSPS_TRY(launch_model_grad(sp, nr, st->l.p, st->y.p, st->gamma.p, st->gk.p, st->gk.p + (int64_t)nm * nr,
                               st->part_obj.p, st->nb_model, s));
    mark(st, PSPS_PROF_MODEL, 1, s);
    mark(st, PSPS_PROF_BACKPROJECT, 0, s);
    // the cross-material Fourier and wavelet preconditioners difference the
    // materials' gradient numerators after a spatial filter, which shows a
    // fixed-point grid of M 2^-22 in the step: keep those to 2^-12 of it
    const bool fine = st->pc && (st->pc->kind == PSPS_PRECOND_BLOCK_FOURIER || st->pc->kind == PSPS_PRECOND_BLOCK_HAAR);
    PSPS_TRY(backproject_or_copy(st, st->gk.p, st->G.p, 2 * nm, s, fine ? nm : 0));
    mark(st, PSPS_PROF_BACKPROJECT, 1, s);
    mark(st, PSPS_PROF_PRECOND, 0, s);
    if (st->has_pen) PSPS_TRY(penalty_call(st, st->x.p, nullptr, st->G.p, 1, 0, st->part_pen.p, s));
    ctrl_begin_kernel<<<1, kThreads, 0, s>>>(st->ls.p, st->part_obj.p, st->nb_model,
                                             st->has_pen ? st->part_pen.p : nullptr, st->nb_pen, st->history.p);
    PSPS_LAUNCH_CHECK();
    // preconditioned gradient, curvature and direction
    PSPS_TRY(apply_M(st, PSPS_APPLY_MT, st->G.p, st->gp.p, s));
    PSPS_TRY(apply_M(st, PSPS_APPLY_ABS_MT, st->G.p + (int64_t)nm * n, st->dp.p, s));
    direction_kernel<<<grid_for(nm * n), kThreads, 0, s>>>(st->gp.p, st->dp.p, st->has_pen ? st->dR.p : nullptr,
                                                           st->pp.p, nm * n);
    PSPS_LAUNCH_CHECK();
    PSPS_TRY(apply_M(st, PSPS_APPLY_M, st->pp.p, st->p.p, s));
    mark(st, PSPS_PROF_PRECOND, 1, s);
    const bool nonneg = (st->flags & PSPS_FLAG_NONNEG) != 0;
    mark(st, PSPS_PROF_PROJECT, 0, s);
    PSPS_TRY(project_or_copy(st, st->p.p, st->q.p, s));
    mark(st, PSPS_PROF_PROJECT, 1, s);
    // step length
    mark(st, PSPS_PROF_LINESEARCH, 0, s);
    if (st->flags & PSPS_FLAG_LINESEARCH) {
        if (st->has_pen) PSPS_TRY(penalty_call(st, st->x.p, st->p.p, nullptr, 0, 0, st->part_pen.p, s));
        ctrl_ls_init_kernel<<<1, kThreads, 0, s>>>(st->ls.p, st->has_pen ? st->part_pen.p : nullptr, st->nb_pen);
        PSPS_LAUNCH_CHECK();
        const int nb = st->nb_model;
        for (int k = 0; k < st->cfg.n_ls; ++k)
            PSPS_TRY(launch_ls_fused(sp, nr, st->l.p, st->q.p, st->y.p, st->ls.p, st->cfg, 0, k + 1 == st->cfg.n_ls,
                                     st->part_ls.p, nb, s));
        if (st->cfg.n_halve > 0)
            PSPS_TRY(
                launch_ls_fused(sp, nr, st->l.p, st->q.p, st->y.p, st->ls.p, st->cfg, 1, 1, st->part_ls.p, nb, s));
    } else {
        set_alpha_one_kernel<<<1, 1, 0, s>>>(st->ls.p);
        PSPS_LAUNCH_CHECK();
    }
    mark(st, PSPS_PROF_LINESEARCH, 1, s);
    mark(st, PSPS_PROF_UPDATE, 0, s);
    update_kernel<<<grid_for(nm * (n > nr ? n : nr)), kThreads, 0, s>>>(
        st->ls.p, st->x.p, st->p.p, nm * n, nonneg ? nullptr : st->l.p, st->q.p, nm * nr, nonneg ? 1 : 0,
        st->alphas.p);
    PSPS_LAUNCH_CHECK();
    finish_iter_kernel<<<1, 1, 0, s>>>(st->ls.p, st->alphas.p, st->cfg.n_halve);
    PSPS_LAUNCH_CHECK();
    if (nonneg) PSPS_TRY(project_or_copy(st, st->x.p, st->l.p, s));
    mark(st, PSPS_PROF_UPDATE, 1, s);
    return MBIR_OK;
}

mbir_status final_objective(psps_state *st, cudaStream_t s) {
    PSPS_TRY(project_or_copy(st, st->x.p, st->l.p, s));
    PSPS_TRY(launch_model_grad(st->sd, st->n_rays, st->l.p, st->y.p, nullptr, nullptr, nullptr,
                               st->part_obj.p, st->nb_model, s));
    if (st->has_pen) PSPS_TRY(penalty_call(st, st->x.p, nullptr, nullptr, 0, 0, st->part_pen.p, s));
    ctrl_begin_kernel<<<1, kThreads, 0, s>>>(st->ls.p, st->part_obj.p, st->nb_model,
                                             st->has_pen ? st->part_pen.p : nullptr, st->nb_pen, st->history.p);
    PSPS_LAUNCH_CHECK();
    return MBIR_OK;
}

// Kernel nodes of a captured graph (the launches one replay makes).
int64_t count_kernel_nodes(cudaGraph_t g) {
    size_t nn = 0;
    cudaGraphGetNodes(g, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    int64_t nk = 0;
    if (nn && cudaGraphGetNodes(g, nodes.data(), &nn) == cudaSuccess)
        for (auto nd : nodes) {
            cudaGraphNodeType t;
            if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++nk;
        }
    return nk;
}

mbir_status ensure_graph(psps_state *st, int which, cudaStream_t s) {
    if (st->graph[which]) return MBIR_OK;
    cudaStream_t cs;
    PSPS_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t g;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cudaStreamDestroy(cs);
        return fail(MBIR_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
    }
    for (int k = 0; k < PSPS_PROF_STAGES; ++k) st->recorded[k] = false;
    mbir_status st_ = iterate(st, which == 1, cs);
    for (int k = 0; k < PSPS_PROF_STAGES; ++k) {
        st->graph_marks[which][k] = st->recorded[k];
        st->recorded[k] = false;
    }
    e = cudaStreamEndCapture(cs, &g);
    cudaStreamDestroy(cs);
    if (st_ != MBIR_OK) return st_;
    if (e != cudaSuccess) return fail(MBIR_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
    st->graph_kernels[which] = count_kernel_nodes(g);
    e = cudaGraphInstantiate(&st->graph[which], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(MBIR_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
    (void)s;
    return MBIR_OK;
}

}  // namespace

extern "C" mbir_status psps_state_create(mbir_plan *plan, const mbmd_spectrum *spec, psps_precond *pc, const float *y,
                                         int64_t n_rays, const double *beta, const float *x0, int flags,
                                         int reproject_every, mbir_stream stream, psps_state **out) {
    if (!spec || !y || !out) return fail(MBIR_ERR_ARG, "psps_state_create: null argument");
    *out = nullptr;
    if (plan && n_rays != plan->n_rays) return fail(MBIR_ERR_ARG, "psps_state_create: n_rays does not match plan");
    if (n_rays < 1) return fail(MBIR_ERR_ARG, "psps_state_create: n_rays must be >= 1");
    if (n_rays % spec->blur_row || n_rays % spec->noise_row)
        return fail(MBIR_ERR_ARG, "psps_state_create: n_rays is not a multiple of the spectrum's blur / noise row");
    if (plan && 2 * spec->n_mat > plan->n_mat_max)
        return fail(MBIR_ERR_ARG, "psps_state_create: plan n_mat_max must be >= 2 n_mat");
    if ((flags & PSPS_FLAG_NONNEG) && pc && pc->kind != PSPS_PRECOND_NONE)
        return fail(MBIR_ERR_ARG, "psps_state_create: NONNEG is for plain SPS only");
    if (pc && (pc->nm != spec->n_mat || pc->image != (plan != nullptr) ||
               pc->n != (plan ? plan->n_pix : n_rays)))
        return fail(MBIR_ERR_ARG, "psps_state_create: preconditioner does not match the problem");
    if (reproject_every < 0) return fail(MBIR_ERR_ARG, "psps_state_create: reproject_every must be >= 0");
    cudaStream_t s = (cudaStream_t)stream;
    psps_state *st = new psps_state();
    st->plan = plan;
    st->spec = spec;
    st->sd = spec_dev(spec);
    st->pc = (pc && pc->kind != PSPS_PRECOND_NONE) ? pc : nullptr;
    st->nm = spec->n_mat;
    st->nc = spec->n_chan;
    st->flags = flags;
    st->reproject_every = reproject_every;
    st->n_rays = n_rays;
    st->n = plan ? plan->n_pix : n_rays;
    st->pd.nm = st->nm;
    if (beta && plan)
        for (int a = 0; a < st->nm; ++a)
            for (int b = 0; b < st->nm; ++b) {
                st->pd.beta[a * 4 + b] = (float)beta[a * st->nm + b];
                if (beta[a * st->nm + b] != 0.0) st->has_pen = true;
            }
    const int nm = st->nm;
    const int64_t n = st->n, nr = n_rays;
    st->nb_model = model_blocks(nr);
    st->nb_pen = penalty_blocks(n);
    mbir_status e = MBIR_OK;
    auto A = [&](DBuf<float> &b, size_t cnt) {
        if (e == MBIR_OK) e = b.alloc(cnt);
    };
    A(st->x, nm * n);
    A(st->l, nm * nr);
    A(st->y, st->nc * nr);
    A(st->gamma, nm * nr);
    A(st->dR, nm * n);
    A(st->gk, 2 * nm * nr);
    A(st->G, 2 * nm * n);
    A(st->gp, nm * n);
    A(st->dp, nm * n);
    A(st->pp, nm * n);
    A(st->p, nm * n);
    A(st->q, nm * nr);
    if (e == MBIR_OK) e = st->part_obj.alloc(st->nb_model);
    if (e == MBIR_OK) e = st->part_pen.alloc(3 * st->nb_pen);
    if (e == MBIR_OK) e = st->part_ls.alloc(2 * kMaxHalve * st->nb_model);
    if (e == MBIR_OK) e = st->ls.alloc(1);
    if (e != MBIR_OK) {
        delete st;
        return e;
    }
    auto setup = [&]() -> mbir_status {
        PSPS_CUDA(cudaMemcpyAsync(st->y.p, y, sizeof(float) * st->nc * nr, cudaMemcpyDeviceToDevice, s));
        if (x0) PSPS_CUDA(cudaMemcpyAsync(st->x.p, x0, sizeof(float) * nm * n, cudaMemcpyDeviceToDevice, s));
        else PSPS_CUDA(cudaMemsetAsync(st->x.p, 0, sizeof(float) * nm * n, s));
        PSPS_CUDA(cudaMemsetAsync(st->ls.p, 0, sizeof(DevLS), s));
        // gamma~ = A |M| 1 ;  dR = |M|^T |R| |M| 1
        float *ones = st->pp.p, *absM1 = st->p.p;
        {
            std::vector<float> h1((size_t)nm * n, 1.f);
            PSPS_CUDA(cudaMemcpyAsync(ones, h1.data(), sizeof(float) * h1.size(), cudaMemcpyHostToDevice, s));
            PSPS_CUDA(cudaStreamSynchronize(s));
        }
        PSPS_TRY(apply_M(st, PSPS_APPLY_ABS_M, ones, absM1, s));
        PSPS_TRY(project_or_copy(st, absM1, st->gamma.p, s));
        PSPS_CUDA(cudaMemsetAsync(st->dR.p, 0, sizeof(float) * nm * n, s));
        if (st->has_pen) {
            PSPS_TRY(penalty_call(st, absM1, nullptr, st->gp.p, 0, 1, nullptr, s));
            PSPS_TRY(apply_M(st, PSPS_APPLY_ABS_MT, st->gp.p, st->dR.p, s));
        }
        PSPS_TRY(project_or_copy(st, st->x.p, st->l.p, s));
        PSPS_CUDA(cudaStreamSynchronize(s));
        return MBIR_OK;
    };
    e = setup();
    if (e != MBIR_OK) {
        delete st;
        return e;
    }
    *out = st;
    return MBIR_OK;
}

extern "C" mbir_status psps_state_destroy(psps_state *st) {
    delete st;
    return MBIR_OK;
}

extern "C" mbir_status psps_step(psps_state *st, int n_iter, double *objective_history, mbir_stream stream) {
    if (!st || n_iter < 0) return fail(MBIR_ERR_ARG, "psps_step: bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    if (st->hist_cap < n_iter + 1) {
        PSPS_TRY(st->history.alloc(n_iter + 1));
        PSPS_TRY(st->alphas.alloc(n_iter + 1));
        st->hist_cap = n_iter + 1;
        for (auto &g : st->graph)
            if (g) {
                cudaGraphExecDestroy(g);
                g = nullptr;
            }
    }
    reset_counter_kernel<<<1, 1, 0, s>>>(st->ls.p);
    PSPS_LAUNCH_CHECK();
    const bool use_graph = (st->flags & PSPS_FLAG_GRAPH) != 0;
    for (int it = 0; it < n_iter; ++it) {
        const bool rp = it > 0 && st->reproject_every > 0 && it % st->reproject_every == 0;
        if (use_graph) {
            PSPS_TRY(ensure_graph(st, rp ? 1 : 0, s));
            PSPS_CUDA(cudaGraphLaunch(st->graph[rp ? 1 : 0], s));
            st->launches += st->graph_kernels[rp ? 1 : 0];
            if (st->prof)
                for (int k = 0; k < PSPS_PROF_STAGES; ++k) st->recorded[k] = st->graph_marks[rp ? 1 : 0][k];
        } else {
            PSPS_TRY(iterate(st, rp, s));
        }
    }
    if (st->prof && n_iter > 0) {
        PSPS_CUDA(cudaStreamSynchronize(s));
        for (int k = 0; k < PSPS_PROF_STAGES; ++k) {
            if (!st->recorded[k]) continue;
            float ms = 0.f;
            PSPS_CUDA(cudaEventElapsedTime(&ms, st->ev[k][0], st->ev[k][1]));
            st->prof_ms[k] += ms;
            st->prof_cnt[k] += 1;
            st->recorded[k] = false;
        }
    }
    if (objective_history) {
        PSPS_TRY(final_objective(st, s));
        PSPS_CUDA(cudaMemcpyAsync(objective_history, st->history.p, sizeof(double) * (n_iter + 1),
                                  cudaMemcpyDeviceToHost, s));
        DevLS h;
        PSPS_CUDA(cudaMemcpyAsync(&h, st->ls.p, sizeof(DevLS), cudaMemcpyDeviceToHost, s));
        PSPS_CUDA(cudaStreamSynchronize(s));
        if (h.nonfinite) return fail(MBIR_ERR_NONFINITE, "psps_step: non-finite objective or line-search value");
    }
    return MBIR_OK;
}

extern "C" mbir_status psps_state_set_data(psps_state *st, const float *y, int64_t n, mbir_stream stream) {
    if (!st || !y) return fail(MBIR_ERR_ARG, "psps_state_set_data: null argument");
    if (n != (int64_t)st->nc * st->n_rays)
        return fail(MBIR_ERR_ARG, "psps_state_set_data: %lld values given, the state holds %lld", (long long)n,
                    (long long)st->nc * st->n_rays);
    PSPS_CUDA(cudaMemcpyAsync(st->y.p, y, sizeof(float) * n, cudaMemcpyDefault, (cudaStream_t)stream));
    return MBIR_OK;
}

extern "C" mbir_status psps_get_image(psps_state *st, float *x, mbir_stream s) {
    if (!st || !x) return fail(MBIR_ERR_ARG, "psps_get_image: null argument");
    PSPS_CUDA(cudaMemcpyAsync(x, st->x.p, sizeof(float) * st->nm * st->n, cudaMemcpyDeviceToDevice, (cudaStream_t)s));
    return MBIR_OK;
}

extern "C" mbir_status psps_get_alphas(psps_state *st, double *alphas, int n, mbir_stream s) {
    if (!st || !alphas || n < 0 || n > st->hist_cap) return fail(MBIR_ERR_ARG, "psps_get_alphas: bad argument");
    PSPS_CUDA(cudaMemcpyAsync(alphas, st->alphas.p, sizeof(double) * n, cudaMemcpyDeviceToHost, (cudaStream_t)s));
    PSPS_CUDA(cudaStreamSynchronize((cudaStream_t)s));
    return MBIR_OK;
}

extern "C" mbir_status psps_profile(psps_state *st, int enable) {
    if (!st) return fail(MBIR_ERR_ARG, "psps_profile: null state");
    for (int k = 0; k < PSPS_PROF_STAGES; ++k) {
        for (int b = 0; b < 2; ++b)
            if (!st->ev[k][b]) PSPS_CUDA(cudaEventCreate(&st->ev[k][b]));
        st->prof_ms[k] = 0.0;
        st->prof_cnt[k] = 0;
        st->recorded[k] = false;
    }
    if (st->prof != (enable != 0)) st->drop_graphs();
    st->prof = enable != 0;
    return MBIR_OK;
}

extern "C" mbir_status psps_profile_read(psps_state *st, double *ms, int64_t *count) {
    if (!st || !ms || !count) return fail(MBIR_ERR_ARG, "psps_profile_read: null argument");
    for (int k = 0; k < PSPS_PROF_STAGES; ++k) {
        ms[k] = st->prof_ms[k];
        count[k] = st->prof_cnt[k];
    }
    return MBIR_OK;
}

// ----------------------------------------------------------------- batches
// Independent reconstructions (the slices of a batched workload) advanced
// together: one CUDA graph per iteration holds every state's iteration as a
// parallel branch (fork/join through events during capture), so the small
// kernels of different slices run concurrently and the whole batch costs one
// graph launch per iteration.
struct psps_batch {
    std::vector<psps_state *> st;
    int reproject_every = 10;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int64_t graph_kernels[2] = {0, 0};
    int64_t launches = 0;
    int hist_cap = 0;
    void drop_graphs() {
        for (auto &g : graph)
            if (g) {
                cudaGraphExecDestroy(g);
                g = nullptr;
            }
    }
    ~psps_batch() { drop_graphs(); }
};

namespace {

mbir_status batch_graph(psps_batch *b, int which) {
    if (b->graph[which]) return MBIR_OK;
    const size_t n = b->st.size();
    std::vector<cudaStream_t> side(n, nullptr);
    std::vector<cudaEvent_t> join(n, nullptr);
    cudaStream_t cs = nullptr;
    cudaEvent_t fork = nullptr;
    mbir_status res = MBIR_OK;
    cudaGraph_t g = nullptr;
    auto cuda = [&](cudaError_t e, const char *what) {
        if (e != cudaSuccess && res == MBIR_OK) res = fail(MBIR_ERR_CUDA, "batch graph: %s: %s", what, cudaGetErrorString(e));
        return e == cudaSuccess;
    };
    bool ok = cuda(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "stream") &&
              cuda(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming), "event");
    for (size_t i = 0; ok && i < n; ++i)
        ok = cuda(cudaStreamCreateWithFlags(&side[i], cudaStreamNonBlocking), "stream") &&
             cuda(cudaEventCreateWithFlags(&join[i], cudaEventDisableTiming), "event");
    if (ok && cuda(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal), "begin capture")) {
        bool cap = cuda(cudaEventRecord(fork, cs), "fork");
        for (size_t i = 0; cap && i < n; ++i) {
            cap = cuda(cudaStreamWaitEvent(side[i], fork, 0), "fork wait");
            if (cap) {
                const mbir_status r = iterate(b->st[i], which == 1, side[i]);
                if (r != MBIR_OK) {
                    if (res == MBIR_OK) res = r;
                    cap = false;
                }
            }
            if (cap) cap = cuda(cudaEventRecord(join[i], side[i]), "join") && cuda(cudaStreamWaitEvent(cs, join[i], 0), "join wait");
        }
        const cudaError_t e = cudaStreamEndCapture(cs, &g);
        if (res == MBIR_OK) cuda(e, "end capture");
    }
    if (res == MBIR_OK) {
        b->graph_kernels[which] = count_kernel_nodes(g);
        cuda(cudaGraphInstantiate(&b->graph[which], g, 0), "instantiate");
    }
    if (g) cudaGraphDestroy(g);
    for (size_t i = 0; i < n; ++i) {
        if (side[i]) cudaStreamDestroy(side[i]);
        if (join[i]) cudaEventDestroy(join[i]);
    }
    if (fork) cudaEventDestroy(fork);
    if (cs) cudaStreamDestroy(cs);
    return res;
}

}  // namespace

extern "C" mbir_status psps_batch_create(psps_state *const *states, int n, psps_batch **out) {
    if (!states || !out || n < 1) return fail(MBIR_ERR_ARG, "psps_batch_create: bad argument");
    *out = nullptr;
    for (int i = 0; i < n; ++i) {
        if (!states[i]) return fail(MBIR_ERR_ARG, "psps_batch_create: state %d is NULL", i);
        if (states[i]->reproject_every != states[0]->reproject_every)
            return fail(MBIR_ERR_ARG, "psps_batch_create: the states must share reproject_every");
        for (int j = 0; j < i; ++j) {
            if (states[j] == states[i]) return fail(MBIR_ERR_ARG, "psps_batch_create: state %d appears twice", i);
            // plans and preconditioners hold per-call scratch: concurrent
            // branches may not share them
            if (states[i]->plan && states[j]->plan == states[i]->plan)
                return fail(MBIR_ERR_ARG, "psps_batch_create: states %d and %d share a plan", j, i);
            if (states[i]->pc && states[j]->pc == states[i]->pc)
                return fail(MBIR_ERR_ARG, "psps_batch_create: states %d and %d share a preconditioner", j, i);
        }
    }
    psps_batch *b = new psps_batch();
    b->st.assign(states, states + n);
    b->reproject_every = states[0]->reproject_every;
    *out = b;
    return MBIR_OK;
}

extern "C" mbir_status psps_batch_destroy(psps_batch *b) {
    delete b;
    return MBIR_OK;
}

extern "C" mbir_status psps_batch_step(psps_batch *b, int n_iter, double *objective_history, mbir_stream stream) {
    if (!b || n_iter < 0) return fail(MBIR_ERR_ARG, "psps_batch_step: bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    if (b->hist_cap < n_iter + 1) {
        for (psps_state *st : b->st)
            if (st->hist_cap < n_iter + 1) {
                PSPS_TRY(st->history.alloc(n_iter + 1));
                PSPS_TRY(st->alphas.alloc(n_iter + 1));
                st->hist_cap = n_iter + 1;
                st->drop_graphs();
            }
        b->hist_cap = n_iter + 1;
        b->drop_graphs();
    }
    for (psps_state *st : b->st) {
        reset_counter_kernel<<<1, 1, 0, s>>>(st->ls.p);
        PSPS_LAUNCH_CHECK();
    }
    for (int it = 0; it < n_iter; ++it) {
        const int rp = (it > 0 && b->reproject_every > 0 && it % b->reproject_every == 0) ? 1 : 0;
        PSPS_TRY(batch_graph(b, rp));
        PSPS_CUDA(cudaGraphLaunch(b->graph[rp], s));
        b->launches += b->graph_kernels[rp];
    }
    if (objective_history) {
        const size_t n = b->st.size();
        std::vector<DevLS> h(n);
        for (size_t i = 0; i < n; ++i) {
            psps_state *st = b->st[i];
            PSPS_TRY(final_objective(st, s));
            PSPS_CUDA(cudaMemcpyAsync(objective_history + i * (size_t)(n_iter + 1), st->history.p,
                                      sizeof(double) * (n_iter + 1), cudaMemcpyDeviceToHost, s));
            PSPS_CUDA(cudaMemcpyAsync(&h[i], st->ls.p, sizeof(DevLS), cudaMemcpyDeviceToHost, s));
        }
        PSPS_CUDA(cudaStreamSynchronize(s));
        for (size_t i = 0; i < n; ++i)
            if (h[i].nonfinite)
                return fail(MBIR_ERR_NONFINITE, "psps_batch_step: state %zu went non-finite", i);
    }
    return MBIR_OK;
}

extern "C" mbir_status psps_batch_launch_count(psps_batch *b, int64_t *count) {
    if (!b || !count) return fail(MBIR_ERR_ARG, "psps_batch_launch_count: null argument");
    *count = b->launches;
    return MBIR_OK;
}

extern "C" mbir_status psps_launch_count(psps_state *st, int64_t *count) {
    if (!st || !count) return fail(MBIR_ERR_ARG, "psps_launch_count: null argument");
    *count = st->launches;
    return MBIR_OK;
}
