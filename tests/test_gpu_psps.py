"""GPU (preconditioned) SPS iterations against the FP64 oracle run of the
same algorithm on the same seeded inputs.

* Without the line search (the paper's update, Eq. 7, on the operator A M)
  the iteration is a majorise-minimise contraction and whole 50-iteration
  runs are compared: objective history to 1e-5, image to 1e-4.
* With the line search the iterates of a descent method with a
  data-dependent step amplify rounding differences from one iteration to the
  next (measured: relative differences grow 2-3x per iteration on the plain
  Fourier preconditioner), so FP32 and FP64 runs part after a few dozen
  iterations.  There the check is per step: from oracle iterates x_k the GPU
  runs one iteration (line search from alpha = 1) and x_{k+1}, Phi and alpha
  are compared with the oracle's one step from the same x_k; whole runs are
  checked for monotone descent.
"""
import numpy as np
import pytest

import synth
from _helpers import gpu_precond_from, oracle_haar_parallel, oracle_precond, rel_l2, to_dev, to_host

pytestmark = pytest.mark.gpu

IMG_TOL = 1e-4      # relative L2 of the image after the run
OBJ_TOL = 1e-5      # relative objective history


@pytest.fixture(scope="module")
def psps():
    import paper_2010_01371_gb300 as p
    p.lib()
    return p


def gpu_state(psps, prob, kind, data, proj=True, line_search=True, nonneg=False, graph=False, x0=None,
              gpu_build=False):
    plan = psps.Plan(prob.geom) if proj else None
    spec = psps.Spectrum(prob.Q, prob.S)
    yd = to_dev(prob.y)
    beta = prob.beta if proj else None
    if gpu_build:
        pc = psps.Precond(plan, spec, kind, yd, beta) if kind != "none" else None
    else:
        pc = gpu_precond_from(psps, plan, spec, kind, data)
    return psps.State(plan, spec, pc, yd, beta, x0=to_dev(x0) if x0 is not None else None,
                      line_search=line_search, nonneg=nonneg, graph=graph), (plan, spec, pc)


def run_both(psps, oracle_lib, prob, kind, n_iter, line_search=True, nonneg=False, graph=False, proj=True,
             gpu_build=False):
    """Oracle and GPU runs of the same iteration.  The GPU preconditioner is
    created from the oracle's eigenvalues/blocks (so the comparison isolates
    the iteration), or built on the GPU when gpu_build is set."""
    from oracle import psps as opsps
    st, P, data = oracle_precond(oracle_lib, prob, kind, proj=proj)
    xo, ho, ao = opsps.run(st, P, n_iter, opsps.LineSearch() if line_search else None, nonneg=nonneg,
                           return_alphas=True)
    state, keep = gpu_state(psps, prob, kind, data, proj, line_search, nonneg, graph, gpu_build=gpu_build)
    hg = psps.psps_step(state, n_iter)
    xg = to_host(psps.psps_get_image(state))
    ag = psps.psps_get_alphas(state, n_iter)
    return xo, ho, ao, xg, hg, ag


# Plain Fourier (Eqs. 27-29) applies M through FP32 FFTs: a 64^2 transform
# (12 radix-2 passes) carries about log2(N) * eps ~ 7e-7 of the largest
# spectral component, and the clamped spectrum spans about 3 decades, so the
# components at its small end carry up to ~7e-4 relative error; measured
# ~2.0e-4 on the image after one step.
FOURIER_IMG_TOL = 4e-4


@pytest.mark.parametrize("kind", ["none", "fourier", "mod_fourier", "haar", "block"])
def test_config1_50_iterations(psps, oracle_lib, kind):
    prob = synth.config1()
    xo, ho, ao, xg, hg, ag = run_both(psps, oracle_lib, prob, kind, 50, line_search=False)
    assert np.all(np.isfinite(hg))
    assert np.max(np.abs(hg - ho) / np.abs(ho)) < OBJ_TOL, np.max(np.abs(hg - ho) / np.abs(ho))
    # plain Fourier without the line search moves x by ~1e-6 in 50 steps
    # (the separable curvature of its dense |M| is far too large); the FP32
    # FFT of the preconditioned gradient then carries ~1e-4 relative error
    assert rel_l2(xg, xo) < (FOURIER_IMG_TOL if kind == "fourier" else IMG_TOL), rel_l2(xg, xo)


def test_config2_reduced_haar_no_ls(psps, oracle_lib):
    prob = synth.config2(nx=128, n_views=180, n_u=222)
    xo, ho, ao, xg, hg, ag = run_both(psps, oracle_lib, prob, "haar", 20, line_search=False)
    assert np.max(np.abs(hg - ho) / np.abs(ho)) < OBJ_TOL
    assert rel_l2(xg, xo) < IMG_TOL, rel_l2(xg, xo)


@pytest.mark.parametrize("kind", ["none", "block", "block_fourier"])
def test_config4_slice_no_ls(psps, oracle_lib, kind):
    """One-step MBMD, 3 materials x 4 photon-counting channels (101 energies)."""
    prob = synth.config4_slice(nx=64, n_views=90, n_u=111)
    xo, ho, ao, xg, hg, ag = run_both(psps, oracle_lib, prob, kind, 30, line_search=False)
    assert np.max(np.abs(hg - ho) / np.abs(ho)) < OBJ_TOL, np.max(np.abs(hg - ho) / np.abs(ho))
    assert rel_l2(xg, xo) < IMG_TOL, rel_l2(xg, xo)


def test_config5_16_block_haar_no_ls(psps, oracle_lib):
    """3-D cross-material wavelet (Eq. 61 over the voxel grid), 16^3."""
    prob = synth.config5(n=16, n_views=12, n_u=32, n_v=24)
    xo, ho, ao, xg, hg, ag = run_both(psps, oracle_lib, prob, "block_haar", 20, line_search=False)
    assert np.max(np.abs(hg - ho) / np.abs(ho)) < OBJ_TOL, np.max(np.abs(hg - ho) / np.abs(ho))
    assert rel_l2(xg, xo) < IMG_TOL, rel_l2(xg, xo)


@pytest.mark.parametrize("kind", ["none", "block"])
def test_config5_reduced_no_ls(psps, oracle_lib, kind):
    """3-D cone-beam one-step MBMD (2 materials, dual energy), 32^3 reduction."""
    prob = synth.config5(n=32, n_views=24, n_u=64, n_v=48)
    xo, ho, ao, xg, hg, ag = run_both(psps, oracle_lib, prob, kind, 20, line_search=False)
    assert np.max(np.abs(hg - ho) / np.abs(ho)) < OBJ_TOL, np.max(np.abs(hg - ho) / np.abs(ho))
    assert rel_l2(xg, xo) < IMG_TOL, rel_l2(xg, xo)


def step_cases():
    c1 = synth.config1
    c2 = lambda: synth.config2(nx=128, n_views=180, n_u=222)   # noqa: E731
    c3 = lambda: synth.config3(n_views=12, n_u=301)            # noqa: E731
    c4 = lambda: synth.config4_slice(nx=64, n_views=90, n_u=111)   # noqa: E731
    c5 = lambda: synth.config5(n=32, n_views=24, n_u=64, n_v=48)   # noqa: E731
    c5s = lambda: synth.config5(n=16, n_views=12, n_u=32, n_v=24)  # noqa: E731
    return {"c5_16-block_haar": (c5s, "block_haar", True), "c1-none": (c1, "none", True), "c1-fourier": (c1, "fourier", True),
            "c1-mod_fourier": (c1, "mod_fourier", True), "c1-haar": (c1, "haar", True),
            "c1-block": (c1, "block", True), "c2-haar": (c2, "haar", True), "c2-none": (c2, "none", True),
            "c3-block": (c3, "block", False),
            "c4-block": (c4, "block", True), "c4-block_fourier": (c4, "block_fourier", True),
            "c4-block_haar": (c4, "block_haar", True),
            "c5-block": (c5, "block", True), "c5-block_fourier": (c5, "block_fourier", True)}


@pytest.mark.parametrize("case", list(step_cases()))
def test_line_search_step_parity(psps, oracle_lib, case):
    from oracle import psps as opsps
    mk, kind, proj = step_cases()[case]
    prob = mk()
    st, P, data = oracle_precond(oracle_lib, prob, kind, proj=proj)
    for k in [0, 4, 15]:
        xk, _ = opsps.run(st, P, k, opsps.LineSearch()) if k else (st.zeros(), None)
        x1o, h1o, a1o = opsps.run(st, P, 1, opsps.LineSearch(), x0=xk, return_alphas=True)
        state, keep = gpu_state(psps, prob, kind, data, proj, x0=xk)
        h1g = psps.psps_step(state, 1)
        a1g = psps.psps_get_alphas(state, 1)
        x1g = to_host(psps.psps_get_image(state))
        assert abs(h1g[0] - h1o[0]) <= OBJ_TOL * abs(h1o[0]), (k, h1g, h1o)
        assert abs(h1g[1] - h1o[1]) <= OBJ_TOL * abs(h1o[1]), (k, h1g, h1o)
        assert abs(a1g[0] - a1o[0]) <= 1e-4 * abs(a1o[0]), (k, a1g, a1o)
        tol = FOURIER_IMG_TOL if kind == "fourier" else IMG_TOL
        assert rel_l2(x1g, x1o) < tol, (k, rel_l2(x1g, x1o))


@pytest.mark.parametrize("case", ["c1-haar", "c1-mod_fourier", "c2-haar", "c3-block"])
def test_line_search_runs_descend(psps, oracle_lib, case):
    mk, kind, proj = step_cases()[case]
    prob = mk()
    st, P, data = oracle_precond(oracle_lib, prob, kind, proj=proj)
    state, keep = gpu_state(psps, prob, kind, data, proj)
    h = psps.psps_step(state, 40)
    assert np.all(np.isfinite(h))
    assert np.all(np.diff(h) <= 1e-7 * h[0])
    assert h[-1] < 0.05 * h[0]


@pytest.mark.parametrize("kind", ["mod_fourier", "haar"])
def test_config1_gpu_built(psps, oracle_lib, error_log, kind):
    """Whole pipeline without the line search: GPU-built preconditioner (its
    element-wise error against the FP64 build is bounded in
    test_gpu_build.py) and 50 iterations against the oracle's FP64 build and
    run: objective history to 1e-5, image to 1e-4."""
    prob = synth.config1()
    xo, ho, ao, xg, hg, ag = run_both(psps, oracle_lib, prob, kind, 50, line_search=False, gpu_build=True)
    eo, ex = np.max(np.abs(hg - ho) / np.abs(ho)), rel_l2(xg, xo)
    error_log.add(f"c1 GPU-built {kind} 50 iterations", "objective history", eo, OBJ_TOL)
    error_log.add(f"c1 GPU-built {kind} 50 iterations", "image", ex, IMG_TOL)
    assert eo < OBJ_TOL, eo
    assert ex < IMG_TOL, ex


def test_projection_domain_block_no_ls(psps, oracle_lib):
    prob = synth.config3(n_views=12, n_u=301)
    xo, ho, ao, xg, hg, ag = run_both(psps, oracle_lib, prob, "block", 50, proj=False, line_search=False)
    assert np.max(np.abs(hg - ho) / np.abs(ho)) < OBJ_TOL
    assert rel_l2(xg, xo) < IMG_TOL, rel_l2(xg, xo)


def test_nonneg_plain_sps_monotone(psps, oracle_lib):
    prob = synth.config1()
    xo, ho, ao, xg, hg, ag = run_both(psps, oracle_lib, prob, "none", 30, line_search=False, nonneg=True)
    assert np.all(np.diff(hg) <= 1e-7 * hg[0])
    assert (xg >= 0).all()
    assert rel_l2(xg, xo) < IMG_TOL


def test_graph_replay_matches(psps):
    prob = synth.config1()
    plan, spec = psps.Plan(prob.geom), psps.Spectrum(prob.Q, prob.S)
    yd = to_dev(prob.y)
    pc = psps.Precond(plan, spec, "mod_fourier", yd, prob.beta)
    a = psps.State(plan, spec, pc, yd, prob.beta, line_search=False)
    b = psps.State(plan, spec, pc, yd, prob.beta, line_search=False, graph=True)
    ha, hb = psps.psps_step(a, 25), psps.psps_step(b, 25)
    assert np.allclose(ha, hb, rtol=1e-6)
    assert rel_l2(to_host(psps.psps_get_image(b)), to_host(psps.psps_get_image(a))) < 1e-5
    c = psps.State(plan, spec, pc, yd, prob.beta, graph=True)
    hc = psps.psps_step(c, 10)
    assert np.all(np.diff(hc) <= 1e-7 * hc[0])
    assert psps.psps_launch_count(c) > 0


def test_set_data_replaces_counts(psps):
    """psps_state_set_data from a pinned host tensor: a state that starts on
    other counts and receives the real ones before its first step runs the
    same iterations as a state created on the real counts (graph replay
    included, since the graph reads the state's own buffer); with the other
    counts kept, the run differs."""
    import torch
    prob = synth.config1()
    plan, spec = psps.Plan(prob.geom), psps.Spectrum(prob.Q, prob.S)
    yd = to_dev(prob.y)
    pc = psps.Precond(plan, spec, "haar", yd, prob.beta)
    a = psps.State(plan, spec, pc, yd, prob.beta, graph=True)
    b = psps.State(plan, spec, pc, yd * 0.5 + 3.0, prob.beta, graph=True)
    psps.psps_state_set_data(b, torch.as_tensor(prob.y.astype(np.float32)).reshape(-1).pin_memory())
    ha, hb = psps.psps_step(a, 8), psps.psps_step(b, 8)
    # equal up to the summation order of the transpose's FP32 atomics
    assert np.allclose(ha, hb, rtol=1e-6)
    assert rel_l2(to_host(psps.psps_get_image(b)), to_host(psps.psps_get_image(a))) < 1e-5
    c = psps.State(plan, spec, pc, yd * 0.5 + 3.0, prob.beta, graph=True)
    assert not np.allclose(psps.psps_step(c, 8), ha, rtol=1e-3)
    with pytest.raises(RuntimeError):
        psps.psps_state_set_data(b, torch.zeros(5, dtype=torch.float32))


def test_batch_matches_single_states(psps):
    """Four uneven slices of the batched MBMD workload (shrunk by 8: 32..64
    pixels, mixed-radix cross-material Fourier) advanced together by one
    graph per iteration give each slice's own run: same objective histories
    and images as the states stepped one by one, and the same kernel count."""
    probs = synth.config4(n_slices=4, n_views=90, shrink=8)
    setups = []
    for p in probs:
        plan, spec, yd = psps.Plan(p.geom), psps.Spectrum(p.Q, p.S), to_dev(p.y)
        setups.append((p, plan, spec, yd, psps.Precond(plan, spec, "block_fourier", yd, p.beta)))
    n_iter = 12   # crosses one exact re-projection (every 10)
    single, h_single = [], []
    for p, plan, spec, yd, pc in setups:
        s = psps.State(plan, spec, pc, yd, p.beta, graph=True)
        h_single.append(psps.psps_step(s, n_iter))
        single.append(s)
    states = [psps.State(plan, spec, pc, yd, p.beta, graph=True) for p, plan, spec, yd, pc in setups]
    batch = psps.Batch(states)
    hb = psps.psps_batch_step(batch, n_iter)
    assert hb.shape == (4, n_iter + 1)
    # every kernel of the 2-D iteration is deterministic (the tile transpose
    # sums in fixed point), so the batch reproduces the single runs bit for bit
    for i in range(4):
        assert np.array_equal(hb[i], h_single[i]), i
        assert np.array_equal(to_host(psps.psps_get_image(states[i])), to_host(psps.psps_get_image(single[i]))), i
    assert psps.psps_batch_launch_count(batch) == sum(psps.psps_launch_count(s) for s in single)
    # states may not repeat or share a plan / preconditioner
    with pytest.raises(RuntimeError):
        psps.Batch([states[0], states[0]])
    p, plan, spec, yd, pc = setups[0]
    other = psps.State(plan, spec, None, yd, p.beta)
    with pytest.raises(RuntimeError):
        psps.Batch([states[0], other])


def test_full_size_step(psps, oracle_lib):
    """The full 512^2 / 720 x 888 fan-beam workload in the launch
    configuration the benchmark times (CUDA graph, line search): two
    iterations from x = 0 with the per-pixel M0 preconditioner created from
    the oracle's blocks, against the oracle's two iterations."""
    from oracle import psps as opsps
    prob = synth.config2()
    st, P, data = oracle_precond(oracle_lib, prob, "block")
    xo, ho, ao = opsps.run(st, P, 2, opsps.LineSearch(), return_alphas=True)
    state, keep = gpu_state(psps, prob, "block", data, graph=True)
    hg = psps.psps_step(state, 2)
    ag = psps.psps_get_alphas(state, 2)
    assert np.max(np.abs(hg - ho) / np.abs(ho)) < OBJ_TOL, (hg, ho)
    assert np.allclose(ag, ao, rtol=1e-4), (ag, ao)
    assert rel_l2(to_host(psps.psps_get_image(state)), xo) < IMG_TOL


def test_zero_iterations(psps):
    """psps_step with n_iter = 0 returns the objective at x0 only."""
    prob = synth.config1()
    plan, spec = psps.Plan(prob.geom), psps.Spectrum(prob.Q, prob.S)
    st = psps.State(plan, spec, None, to_dev(prob.y), prob.beta)
    h = psps.psps_step(st, 0)
    assert h.shape == (1,) and np.isfinite(h[0]) and h[0] > 0
    assert np.array_equal(psps.psps_step(st, 0), h)


FULL_SIZE = {
    # the benchmark's workloads at their own sizes, preconditioners built on
    # the GPU the way bench.py builds them: (synth builder, keywords, kind)
    "c2_512-haar": ("config2", {}, "haar"),
    "c4_512-block_fourier": ("config4_slice", {}, "block_fourier"),
    "c5_64-block": ("config5", {"n": 64, "n_views": 90, "n_u": 128, "n_v": 96}, "block"),
}


@pytest.mark.parametrize("case", list(FULL_SIZE))
def test_full_size_gpu_built_step(psps, oracle_lib, error_log, case):
    """Line-searched step parity at the workload's own size with the GPU-built
    preconditioner (autotuned plan, as timed by the benchmark): from the
    oracle's iterates x_0 = 0 and x_4, one GPU iteration against one oracle
    iteration with the oracle's FP64-built preconditioner.  Objective before
    and after to 1e-5, alpha and the image to 1e-4."""
    from oracle import psps as opsps
    builder, kw, kind = FULL_SIZE[case]
    prob = getattr(synth, builder)(**kw)
    if kind == "haar":       # 205 Hessian applications at 512^2: split among host cores
        st, P = oracle_haar_parallel(oracle_lib, builder, kw)
    else:
        st, P, data = oracle_precond(oracle_lib, prob, kind)
    plan, spec = psps.Plan(prob.geom), psps.Spectrum(prob.Q, prob.S)
    plan.autotune(2 * st.nm)
    yd = to_dev(prob.y)
    pc = psps.Precond(plan, spec, kind, yd, prob.beta)
    xk = st.zeros()
    done = 0
    for k in [0, 4]:
        if k > done:
            xk, _ = opsps.run(st, P, k - done, opsps.LineSearch(), x0=xk)
            done = k
        x1o, h1o, a1o = opsps.run(st, P, 1, opsps.LineSearch(), x0=xk, return_alphas=True)
        state = psps.State(plan, spec, pc, yd, prob.beta, x0=to_dev(xk), line_search=True, graph=True)
        h1g = psps.psps_step(state, 1)
        a1g = psps.psps_get_alphas(state, 1)
        x1g = to_host(psps.psps_get_image(state))
        eo = [abs(h1g[i] - h1o[i]) / abs(h1o[i]) for i in (0, 1)]
        ea = abs(a1g[0] - a1o[0]) / abs(a1o[0])
        ex = rel_l2(x1g, x1o)
        error_log.add(f"full-size step {case} k={k}", "objective before/after", max(eo), OBJ_TOL)
        error_log.add(f"full-size step {case} k={k}", "alpha", ea, 1e-4)
        error_log.add(f"full-size step {case} k={k}", "image", ex, IMG_TOL)
        assert max(eo) <= OBJ_TOL, (k, eo)
        assert ea <= 1e-4, (k, a1g, a1o)
        assert ex < IMG_TOL, (k, ex)
