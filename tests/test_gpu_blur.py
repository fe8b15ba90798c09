"""Detector blur in the outer operator (B S, Eq. 1): GPU forward model, PWLS
objective and gradient, and (P)SPS iterations with the blurred numerators of
Eqs. 8 and 10, against the FP64 oracle with the same blur."""
import numpy as np
import pytest

import synth
from _helpers import gpu_precond_from, oracle_precond, rel_l2, small_geoms, to_dev, to_host

pytestmark = pytest.mark.gpu

IMG_TOL = 1e-4
OBJ_TOL = 1e-5


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


@pytest.mark.parametrize("taps", ["r1", "r3"])
def test_blurred_forward_model(psps, oracle_lib, taps):
    from oracle import model
    Q, S = spectral()
    n_u, n_rows = 97, 53          # ragged rows, several model blocks
    rng = np.random.default_rng(2)
    l = np.stack([rng.uniform(0, 300, n_u * n_rows), rng.uniform(0, 30, n_u * n_rows)])
    spec = psps.Spectrum(Q, S)
    spec.set_blur(synth.BLUR_TAPS[taps], n_u)
    got = to_host(psps.mbmd_forward_model(spec, to_dev(l)))
    want = model.forward_model(Q, S, l, model.Blur(synth.BLUR_TAPS[taps], n_u))
    assert rel_l2(got, want) < 1e-5, rel_l2(got, want)
    spec.set_blur(None, 1)       # removing the blur gives the plain model back
    got = to_host(psps.mbmd_forward_model(spec, to_dev(l)))
    assert rel_l2(got, model.forward_model(Q, S, l)) < 1e-5


@pytest.mark.parametrize("case", ["image-r1", "image-r3", "projdomain-r3"])
def test_blurred_objective_and_gradient(psps, oracle_lib, case):
    from oracle import model
    from _helpers import phantom
    kind, taps = case.split("-")
    Q, S = spectral()
    blur_taps = synth.BLUR_TAPS[taps]
    if kind == "image":
        g = small_geoms()["fan2d_ragged"]
        A = oracle_lib.Projector(g)
        x_true = 20 * phantom(g, seed=3, nm=2)
        x = 0.6 * x_true
        n_u, lt, lx = g.n_u, A.project(x_true), A.project(x)
        plan = psps.Plan(g)
    else:
        rng = np.random.default_rng(6)
        n_u = 101
        lt = np.stack([rng.uniform(0, 300, 41 * n_u), rng.uniform(0, 30, 41 * n_u)])
        x = lx = 0.8 * lt
        plan = None
    blur = model.Blur(blur_taps, n_u)
    y = np.random.default_rng(4).poisson(model.forward_model(Q, S, lt, blur)).astype(float)
    spec = psps.Spectrum(Q, S)
    spec.set_blur(blur_taps, n_u)
    want_obj = model.data_objective(Q, S, lx, y, blur)
    obj = float(psps.mbmd_objective(plan, spec, to_dev(x), to_dev(y)).item())
    assert abs(obj - want_obj) <= 1e-5 * abs(want_obj), (obj, want_obj)
    grad, obj2 = psps.mbmd_gradient(plan, spec, to_dev(x), to_dev(y))
    gl = model.data_grad_l(Q, S, lx, y, blur)
    want = A.backproject(gl) if plan is not None else gl
    assert rel_l2(to_host(grad), want) < 1e-5, rel_l2(to_host(grad), want)
    assert abs(float(obj2.item()) - want_obj) <= 1e-5 * abs(want_obj)
    # the blur matters at this size: the unblurred model is far off
    assert abs(model.data_objective(Q, S, lx, y) - want_obj) > 1e-3 * abs(want_obj)


def blurred_state(psps, prob, kind, data, taps, n_u, proj=True, line_search=True, x0=None, graph=False):
    plan = psps.Plan(prob.geom) if proj else None
    spec = psps.Spectrum(prob.Q, prob.S)
    spec.set_blur(taps, n_u)
    beta = prob.beta if proj else None
    pc = gpu_precond_from(psps, plan, spec, kind, data)
    st = psps.State(plan, spec, pc, to_dev(prob.y), beta, x0=to_dev(x0) if x0 is not None else None,
                    line_search=line_search, graph=graph)
    return st, (plan, spec, pc)


def blur_cases():
    c1 = synth.config1
    c3 = lambda: synth.config3(n_views=12, n_u=301)                # noqa: E731
    c4 = lambda: synth.config4_slice(nx=64, n_views=90, n_u=111)   # noqa: E731
    c5 = lambda: synth.config5(n=32, n_views=24, n_u=64, n_v=48)   # noqa: E731
    return {"c1-none-r1": (c1, "none", "r1", None, True), "c1-block-r3": (c1, "block", "r3", None, True),
            "c3-block-r3": (c3, "block", "r3", 301, False), "c4-block-r1": (c4, "block", "r1", None, True),
            "c4-block_fourier-r3": (c4, "block_fourier", "r3", None, True),
            "c5-block-r1": (c5, "block", "r1", None, True)}


def make_case(oracle_lib, case):
    from oracle import model
    mk, kind, taps, n_u, proj = blur_cases()[case]
    prob = mk()
    n_u = n_u or prob.geom.n_u
    prob = synth.with_detector_blur(prob, synth.BLUR_TAPS[taps], n_u)
    blur = model.Blur(synth.BLUR_TAPS[taps], n_u)
    st, P, data = oracle_precond(oracle_lib, prob, kind, proj=proj, blur=blur)
    return prob, kind, synth.BLUR_TAPS[taps], n_u, proj, st, P, data


@pytest.mark.parametrize("case", ["c1-none-r1", "c1-block-r3", "c4-block-r1", "c5-block-r1"])
def test_blurred_runs_no_ls(psps, oracle_lib, case):
    """The paper's update (Eq. 7) with the blurred SPS curvature: whole runs."""
    from oracle import psps as opsps
    prob, kind, taps, n_u, proj, st, P, data = make_case(oracle_lib, case)
    n_iter = 20
    xo, ho = opsps.run(st, P, n_iter, None)
    state, keep = blurred_state(psps, prob, kind, data, taps, n_u, proj, line_search=False)
    hg = psps.psps_step(state, n_iter)
    xg = to_host(psps.psps_get_image(state))
    assert np.max(np.abs(hg - ho) / np.abs(ho)) < OBJ_TOL, np.max(np.abs(hg - ho) / np.abs(ho))
    assert rel_l2(xg, xo) < IMG_TOL, rel_l2(xg, xo)
    # majorise-minimise: monotone on both sides
    assert np.all(np.diff(ho) <= 0) and np.all(np.diff(hg) <= 1e-7 * hg[0])


@pytest.mark.parametrize("case", list(blur_cases()))
def test_blurred_line_search_step(psps, oracle_lib, case):
    """One iteration with the line search from oracle iterates x_k."""
    from oracle import psps as opsps
    prob, kind, taps, n_u, proj, st, P, data = make_case(oracle_lib, case)
    for k in [0, 4]:
        xk, _ = opsps.run(st, P, k, opsps.LineSearch()) if k else (st.zeros(), None)
        x1o, h1o, a1o = opsps.run(st, P, 1, opsps.LineSearch(), x0=xk, return_alphas=True)
        state, keep = blurred_state(psps, prob, kind, data, taps, n_u, proj, x0=xk)
        h1g = psps.psps_step(state, 1)
        a1g = psps.psps_get_alphas(state, 1)
        x1g = to_host(psps.psps_get_image(state))
        assert abs(h1g[0] - h1o[0]) <= OBJ_TOL * abs(h1o[0]), (k, h1g, h1o)
        assert abs(h1g[1] - h1o[1]) <= OBJ_TOL * abs(h1o[1]), (k, h1g, h1o)
        assert abs(a1g[0] - a1o[0]) <= 1e-4 * abs(a1o[0]), (k, a1g, a1o)
        assert rel_l2(x1g, x1o) < IMG_TOL, (k, rel_l2(x1g, x1o))


def test_blurred_graph_replay(psps, oracle_lib):
    prob, kind, taps, n_u, proj, st, P, data = make_case(oracle_lib, "c4-block-r1")
    a, ka = blurred_state(psps, prob, kind, data, taps, n_u, proj)
    b, kb = blurred_state(psps, prob, kind, data, taps, n_u, proj, graph=True)
    ha, hb = psps.psps_step(a, 8), psps.psps_step(b, 8)
    assert np.allclose(ha, hb, rtol=1e-6)
    assert np.all(np.diff(hb) <= 1e-7 * hb[0])


def test_blur_arguments(psps):
    from paper_2010_01371_gb300._abi import MbirError
    Q, S = spectral()
    spec = psps.Spectrum(Q, S)
    with pytest.raises(MbirError):
        spec.set_blur([0.1] * 9, 10)                # radius 4 > 3
    with pytest.raises(MbirError):
        spec.set_blur([0.2, -0.1, 0.9], 10)         # negative tap
    with pytest.raises(MbirError):
        spec.set_blur([0.2, 0.6, 0.2], 0)           # row < 1
    spec.set_blur([0.2, 0.6, 0.2], 10)
    l = to_dev(np.ones((2, 25)))
    with pytest.raises(MbirError):
        psps.mbmd_forward_model(spec, l)            # 25 rays are not whole rows of 10
    y = to_dev(np.full((2, 25), 100.0))
    with pytest.raises(MbirError):
        psps.State(None, spec, None, y)
    # a state keeps the blur it was created with
    l = np.random.default_rng(1).uniform(0, 20, (2, 30))
    y = to_dev(np.full((2, 30), 1e4))
    st = psps.State(None, spec, None, y, x0=to_dev(l), line_search=False)
    spec.set_blur(None, 1)
    h = psps.psps_step(st, 1)
    from oracle import model
    want = model.data_objective(Q, S, l, np.full((2, 30), 1e4), model.Blur([0.2, 0.6, 0.2], 10))
    assert abs(h[0] - want) <= 1e-5 * abs(want)
