"""Correlated detector noise (non-diagonal Sigma_y: a first-order
autoregressive correlation along detector rows, Sec. II-A) on the GPU: data
term, gradient, curvature and (P)SPS iterations against the FP64 oracle,
alone and together with a detector blur."""
import numpy as np
import pytest

import synth
from _helpers import gpu_precond_from, oracle_precond, phantom, rel_l2, small_geoms, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def psps():
    import paper_2010_01371_gb300 as p
    p.lib()
    return p


def spectral():
    E = np.arange(20.0, 141.0)
    Q = synth.material_Q(E, ["water", "bone"], np.random.default_rng(11))
    S = np.stack([1e5 * synth.kramers(E, 80.0), 1e5 * synth.kramers(E, 140.0)])
    return Q, S


@pytest.mark.parametrize("case", ["image-noise", "image-blur-noise", "projdomain-noise"])
def test_noise_data_term(psps, oracle_lib, case):
    from oracle import model
    Q, S = spectral()
    if case.startswith("image"):
        g = small_geoms()["fan2d_ragged"]
        A = oracle_lib.Projector(g)
        x_true = 20 * phantom(g, seed=3, nm=2)
        x = 0.6 * x_true
        n_u, lt, lx = g.n_u, A.project(x_true), A.project(x)
        plan = psps.Plan(g)
        gamma = A.project(np.ones((2,) + g.image_shape))
    else:
        rng = np.random.default_rng(6)
        n_u = 101
        lt = np.stack([rng.uniform(0, 300, 41 * n_u), rng.uniform(0, 30, 41 * n_u)])
        x = lx = 0.8 * lt
        plan, A = None, None
        gamma = np.ones_like(lx)
    blur = model.Blur(synth.BLUR_TAPS["r1"], n_u) if "blur" in case else None
    noise = model.RowCorrelation(0.5, n_u)
    y = np.random.default_rng(4).poisson(model.forward_model(Q, S, lt, blur)).astype(float)
    spec = psps.Spectrum(Q, S)
    if blur is not None:
        spec.set_blur(blur.b, n_u)
    spec.set_noise(0.5, n_u)
    want_obj = model.data_objective(Q, S, lx, y, blur, noise)
    obj = float(psps.mbmd_objective(plan, spec, to_dev(x), to_dev(y)).item())
    assert abs(obj - want_obj) <= 1e-5 * abs(want_obj), (obj, want_obj)
    grad, _ = psps.mbmd_gradient(plan, spec, to_dev(x), to_dev(y))
    gl = model.data_grad_l(Q, S, lx, y, blur, noise)
    want = A.backproject(gl) if A is not None else gl
    assert rel_l2(to_host(grad), want) < 1e-5, rel_l2(to_host(grad), want)
    kap = model.curvature_numerator(Q, S, lx, y, gamma, blur, noise)
    want = A.backproject(kap) if A is not None else kap
    got = to_host(psps.mbmd_curvature(plan, spec, to_dev(x), to_dev(y)))
    assert rel_l2(got, want) < 1e-5, rel_l2(got, want)
    # the correlation matters at this size
    assert abs(model.data_objective(Q, S, lx, y, blur) - want_obj) > 1e-3 * abs(want_obj)


def noisy_case(oracle_lib, name):
    from oracle import model
    cases = {"c1-none": (synth.config1, "none", None), "c4-block-r1": (
        lambda: synth.config4_slice(nx=64, n_views=90, n_u=111), "block", "r1")}
    mk, kind, taps = cases[name]
    prob = mk()
    n_u = prob.geom.n_u
    if taps:
        prob = synth.with_detector_blur(prob, synth.BLUR_TAPS[taps], n_u)
    blur = model.Blur(synth.BLUR_TAPS[taps], n_u) if taps else None
    noise = model.RowCorrelation(0.4, n_u)
    st, P, data = oracle_precond(oracle_lib, prob, kind, blur=blur)
    st.noise = noise
    return prob, kind, taps, n_u, st, P, data


def noisy_state(psps, prob, kind, data, taps, n_u, line_search=True, x0=None):
    plan = psps.Plan(prob.geom)
    spec = psps.Spectrum(prob.Q, prob.S)
    if taps:
        spec.set_blur(synth.BLUR_TAPS[taps], n_u)
    spec.set_noise(0.4, n_u)
    pc = gpu_precond_from(psps, plan, spec, kind, data)
    st = psps.State(plan, spec, pc, to_dev(prob.y), prob.beta, x0=to_dev(x0) if x0 is not None else None,
                    line_search=line_search)
    return st, (plan, spec, pc)


@pytest.mark.parametrize("name", ["c1-none", "c4-block-r1"])
def test_noise_runs_and_steps(psps, oracle_lib, name):
    """20 iterations of the paper's update (Eq. 7) and one line-searched
    step from an oracle iterate, with correlated noise (and a blur)."""
    from oracle import psps as opsps
    prob, kind, taps, n_u, st, P, data = noisy_case(oracle_lib, name)
    xo, ho = opsps.run(st, P, 20, None)
    state, keep = noisy_state(psps, prob, kind, data, taps, n_u, line_search=False)
    hg = psps.psps_step(state, 20)
    xg = to_host(psps.psps_get_image(state))
    assert np.max(np.abs(hg - ho) / np.abs(ho)) < 1e-5, np.max(np.abs(hg - ho) / np.abs(ho))
    assert rel_l2(xg, xo) < 1e-4, rel_l2(xg, xo)
    assert np.all(np.diff(hg) <= 1e-7 * hg[0])
    xk, _ = opsps.run(st, P, 4, opsps.LineSearch())
    x1o, h1o, a1o = opsps.run(st, P, 1, opsps.LineSearch(), x0=xk, return_alphas=True)
    state, keep = noisy_state(psps, prob, kind, data, taps, n_u, x0=xk)
    h1g = psps.psps_step(state, 1)
    a1g = psps.psps_get_alphas(state, 1)
    assert abs(h1g[1] - h1o[1]) <= 1e-5 * abs(h1o[1]), (h1g, h1o)
    assert abs(a1g[0] - a1o[0]) <= 1e-4 * abs(a1o[0]), (a1g, a1o)
    assert rel_l2(to_host(psps.psps_get_image(state)), x1o) < 1e-4


def test_noise_arguments(psps):
    from paper_2010_01371_gb300._abi import MbirError
    Q, S = spectral()
    spec = psps.Spectrum(Q, S)
    with pytest.raises(MbirError):
        spec.set_noise(0.995, 10)
    with pytest.raises(MbirError):
        spec.set_noise(0.5, 1)
    spec.set_blur([0.2, 0.6, 0.2], 10)
    with pytest.raises(MbirError):
        spec.set_noise(0.5, 12)               # rows of blur and noise differ
    spec.set_blur(None, 1)
    spec.set_noise(0.5, 10)
    with pytest.raises(MbirError):
        spec.set_blur([0.2, 0.6, 0.2], 12)
    y = to_dev(np.full((2, 25), 100.0))
    with pytest.raises(MbirError):
        psps.mbmd_objective(None, spec, to_dev(np.ones((2, 25))), y)   # 25 rays are not whole rows
    spec.set_noise(0.0)
    psps.mbmd_objective(None, spec, to_dev(np.ones((2, 25))), y)
