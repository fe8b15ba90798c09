"""GPU forward model, PWLS objective and adjoint gradient parity with the
FP64 oracle (standard CT and spectral)."""
import math

import numpy as np
import pytest

import synth
from _helpers import phantom, rel_l2, small_geoms, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def psps():
    import paper_2010_01371_gb300 as p
    p.lib()
    return p


def spectral(nm=2):
    E = np.arange(20.0, 141.0)
    names = ["water", "bone", "iodine"][:nm]
    Q = synth.material_Q(E, names, np.random.default_rng(11))
    S = np.stack([1e5 * synth.kramers(E, 80.0), 1e5 * synth.kramers(E, 140.0)])
    return Q, S


def test_forward_model_parity(psps, oracle_lib):
    from oracle import model
    Q, S = spectral(2)
    rng = np.random.default_rng(1)
    l = np.stack([rng.uniform(0, 300, 5003), rng.uniform(0, 30, 5003)])
    spec = psps.Spectrum(Q, S)
    got = to_host(psps.mbmd_forward_model(spec, to_dev(l)))
    want = model.forward_model(Q, S, l)
    assert rel_l2(got, want) < 1e-5


@pytest.mark.parametrize("case", ["mbir", "spectral"])
def test_objective_and_gradient_parity(psps, oracle_lib, case):
    from oracle import model
    g = small_geoms()["fan2d_ragged"]
    A = oracle_lib.Projector(g)
    if case == "mbir":
        Q, S = np.ones((1, 1)), np.full((1, 1), 1e5)
        x_true = phantom(g, seed=2, nm=1)
        x = 0.5 * x_true
    else:
        Q, S = spectral(2)
        x_true = 20 * phantom(g, seed=3, nm=2)
        x = 0.6 * x_true
    y = np.random.default_rng(4).poisson(model.forward_model(Q, S, A.project(x_true))).astype(float)
    plan = psps.Plan(g)
    spec = psps.Spectrum(Q, S)
    obj = float(psps.mbmd_objective(plan, spec, to_dev(x), to_dev(y)).item())
    want_obj = model.data_objective(Q, S, A.project(x), y)
    assert abs(obj - want_obj) <= 1e-5 * abs(want_obj)
    grad, obj2 = psps.mbmd_gradient(plan, spec, to_dev(x), to_dev(y))
    want = A.backproject(model.data_grad_l(Q, S, A.project(x), y))
    assert rel_l2(to_host(grad), want) < 1e-5, rel_l2(to_host(grad), want)
    assert abs(float(obj2.item()) - want_obj) <= 1e-5 * abs(want_obj)


def test_projection_domain_gradient(psps, oracle_lib):
    from oracle import model
    Q, S = spectral(2)
    rng = np.random.default_rng(6)
    lt = np.stack([rng.uniform(0, 300, 4099), rng.uniform(0, 30, 4099)])
    y = rng.poisson(model.forward_model(Q, S, lt)).astype(float)
    l = 0.8 * lt
    spec = psps.Spectrum(Q, S)
    grad, obj = psps.mbmd_gradient(None, spec, to_dev(l), to_dev(y))
    assert rel_l2(to_host(grad), model.data_grad_l(Q, S, l, y)) < 1e-5
    want = model.data_objective(Q, S, l, y)
    assert abs(float(obj.item()) - want) <= 1e-5 * abs(want)


def test_autograd_adjoint(psps, oracle_lib):
    """MBMDData: backward (hand-written adjoint) equals the oracle gradient and
    a central finite difference of the forward along a random direction."""
    import torch
    from oracle import model
    g = small_geoms()["par2d_ragged"]
    A = oracle_lib.Projector(g)
    Q, S = np.ones((1, 1)), np.full((1, 1), 1e4)
    xt = phantom(g, seed=7)
    y = np.random.default_rng(8).poisson(1e4 * np.exp(-A.project(xt))).astype(float)
    plan, spec = psps.Plan(g), psps.Spectrum(Q, S)
    x = to_dev(0.5 * xt).requires_grad_(True)
    yd = to_dev(y)
    L = psps.MBMDData.apply(x, plan, spec, yd)
    L.backward()
    want = A.backproject(model.data_grad_l(Q, S, A.project(0.5 * xt), y))
    assert rel_l2(to_host(x.grad), want) < 1e-5
    v = np.random.default_rng(9).standard_normal(xt.shape)
    h = 1e-3 * np.abs(xt).max()
    with torch.no_grad():
        fp = float(psps.MBMDData.apply(to_dev(0.5 * xt + h * v), plan, spec, yd))
        fm = float(psps.MBMDData.apply(to_dev(0.5 * xt - h * v), plan, spec, yd))
    fd = (fp - fm) / (2 * h)
    an = float(np.sum(want * v))
    assert abs(fd - an) <= 1e-3 * abs(an)


AUTOGRAD_CASES = {
    # one-step MBMD, 3 materials x 4 photon-counting channels (101 energies)
    "c4_64_3mat": lambda: synth.config4_slice(nx=64, n_views=90, n_u=111),
    # cone-beam one-step MBMD, 2 materials x 2 kVp, 32^3 (the scan scaled down)
    "c5_32_cone": lambda: synth.config5(n=32, n_views=24, n_u=64, n_v=48),
}


@pytest.mark.parametrize("case", list(AUTOGRAD_CASES))
def test_autograd_basis_images(psps, oracle_lib, error_log, case):
    """MBMDData over several basis images (Sec. II-F, Eqs. 43-48): the
    backward (mbmd_gradient) against the oracle gradient (1e-5), its
    directional derivative against a central finite difference of the FP64
    oracle objective (1e-5) and of the GPU forward (1e-3: FP32 objective),
    and the graph saves only x and y -- l = A x and exp(-Q l) are recomputed
    in backward, never stored."""
    import torch
    from oracle import model
    prob = AUTOGRAD_CASES[case]()
    A = oracle_lib.Projector(prob.geom)
    Q, S, y = prob.Q, prob.S, prob.y
    x0 = 0.8 * prob.truth
    plan, spec = psps.Plan(prob.geom), psps.Spectrum(Q, S)
    yd = to_dev(y)
    x = to_dev(x0).requires_grad_(True)
    saved = []
    with torch.autograd.graph.saved_tensors_hooks(lambda t: saved.append(t.numel()) or t, lambda t: t):
        L = psps.MBMDData.apply(x, plan, spec, yd)
    assert sum(saved) <= x.numel() + yd.numel(), saved
    want_L = model.data_objective(Q, S, A.project(x0), y)
    assert abs(float(L) - want_L) <= 1e-5 * abs(want_L)
    L.backward()
    want = A.backproject(model.data_grad_l(Q, S, A.project(x0), y))
    e = rel_l2(to_host(x.grad), want)
    error_log.add(f"autograd {case}", "gradient vs oracle", e, 1e-5)
    assert e < 1e-5, e
    # direction: the oracle gradient, each material scaled to that
    # material's norm (a random direction makes g . v a sum with
    # cancellation, whose relative error is the gradient's times
    # ||g|| ||v|| / |g . v|; one scale for all materials would step far
    # along the strongly attenuating iodine-like one, where the central
    # difference's truncation error grows)
    ax = tuple(range(1, x0.ndim))
    v = want * (np.sqrt((x0 ** 2).sum(axis=ax, keepdims=True)) / np.sqrt((want ** 2).sum(axis=ax, keepdims=True)))
    dg = float(np.sum(to_host(x.grad) * v))
    h = 1e-5      # FP64 central difference: truncation ~1e-8 relative here
    fd_o = (model.data_objective(Q, S, A.project(x0 + h * v), y)
            - model.data_objective(Q, S, A.project(x0 - h * v), y)) / (2 * h)
    error_log.add(f"autograd {case}", "directional derivative vs oracle central difference",
                  abs(dg - fd_o) / abs(fd_o), 1e-5)
    assert abs(dg - fd_o) <= 1e-5 * abs(fd_o), (dg, fd_o)
    # central difference of the GPU forward itself (FP32 data term, double-
    # float sum): checks the autograd plumbing, not the precision
    h = 1e-3
    with torch.no_grad():
        fp = float(psps.MBMDData.apply(to_dev(x0 + h * v), plan, spec, yd))
        fm = float(psps.MBMDData.apply(to_dev(x0 - h * v), plan, spec, yd))
    fd_g = (fp - fm) / (2 * h)
    error_log.add(f"autograd {case}", "directional derivative vs GPU central difference", abs(dg - fd_g) / abs(dg),
                  1e-3)
    assert abs(dg - fd_g) <= 1e-3 * abs(dg), (dg, fd_g)


def test_full_size_projection_domain(psps, oracle_lib):
    """Full projection-domain workload (720 x 888 rays, 2 materials x 2 kVp,
    121 energies): the per-ray gradient numerators of every ray and the data
    term over all rays against the oracle."""
    from oracle import model
    prob = synth.config3()
    l = 0.7 * prob.truth
    spec = psps.Spectrum(prob.Q, prob.S)
    grad, obj = psps.mbmd_gradient(None, spec, to_dev(l), to_dev(prob.y))
    want = model.data_grad_l(prob.Q, prob.S, l, prob.y)
    assert rel_l2(to_host(grad), want) < 1e-5, rel_l2(to_host(grad), want)
    want_obj = model.data_objective(prob.Q, prob.S, l, prob.y)
    assert abs(float(obj.item()) - want_obj) <= 1e-5 * abs(want_obj)


def test_full_size_mbmd_slice(psps, oracle_lib):
    """Full 512^2 one-step MBMD slice (3 materials, 4 photon-counting
    channels, 101 energies, 720 x 888 fan beam): data term and image gradient
    A^T g against the oracle."""
    from oracle import model
    prob = synth.config4_slice()
    A = oracle_lib.Projector(prob.geom)
    x = 0.8 * prob.truth
    plan, spec = psps.Plan(prob.geom), psps.Spectrum(prob.Q, prob.S)
    grad, obj = psps.mbmd_gradient(plan, spec, to_dev(x), to_dev(prob.y))
    lx = A.project(x)
    want = A.backproject(model.data_grad_l(prob.Q, prob.S, lx, prob.y))
    assert rel_l2(to_host(grad), want) < 1e-5, rel_l2(to_host(grad), want)
    want_obj = model.data_objective(prob.Q, prob.S, lx, prob.y)
    assert abs(float(obj.item()) - want_obj) <= 1e-5 * abs(want_obj)


def test_size_limits_and_degenerate_counts(psps, oracle_lib):
    """Largest spectral sizes the library takes (4 materials, 256 energies, 8
    channels), counts that are all zero (w = 1) and a single ray; sizes past
    the limits are rejected."""
    from oracle import model
    rng = np.random.default_rng(21)
    E = np.linspace(15.0, 150.0, 256)
    Q = synth.material_Q(E, ["water", "bone", "iodine", "water"], rng)
    edges = np.linspace(15.0, 151.0, 9)
    S = np.stack([1e4 * synth.kramers(E, 150.0) * ((E >= a) & (E < b)) for a, b in zip(edges[:-1], edges[1:])])
    l = np.stack([rng.uniform(0, 100, 777), rng.uniform(0, 10, 777), rng.uniform(0, 0.5, 777),
                  rng.uniform(0, 50, 777)])
    spec = psps.Spectrum(Q, S)
    got = to_host(psps.mbmd_forward_model(spec, to_dev(l)))
    assert rel_l2(got, model.forward_model(Q, S, l)) < 1e-5
    for y in [np.zeros((8, 777)), rng.poisson(model.forward_model(Q, S, 1.1 * l)).astype(float)]:
        grad, obj = psps.mbmd_gradient(None, spec, to_dev(l), to_dev(y))
        assert rel_l2(to_host(grad), model.data_grad_l(Q, S, l, y)) < 1e-5
        want = model.data_objective(Q, S, l, y)
        assert abs(float(obj.item()) - want) <= 1e-5 * abs(want)
    one = l[:, :1]
    grad, obj = psps.mbmd_gradient(None, spec, to_dev(one), to_dev(np.ones((8, 1))))
    assert rel_l2(to_host(grad), model.data_grad_l(Q, S, one, np.ones((8, 1)))) < 1e-5
    with pytest.raises(RuntimeError):
        psps.Spectrum(np.ones((257, 1)), np.ones((1, 257)))
    with pytest.raises(RuntimeError):
        psps.Spectrum(np.ones((4, 5)), np.ones((1, 4)))


@pytest.mark.parametrize("case", ["mbir", "spectral", "projdomain", "spectral-blur"])
def test_curvature_parity(psps, oracle_lib, case):
    """Plain-SPS separable curvature A^T kappa (Eqs. 6, 8-11 with M = I)
    against the oracle's numerators with gamma = A 1 (projection domain:
    gamma = 1), on image and line-integral inputs, with and without a
    detector blur."""
    from oracle import model
    if case == "projdomain":
        Q, S = spectral(2)
        rng = np.random.default_rng(8)
        lt = np.stack([rng.uniform(0, 300, 4099), rng.uniform(0, 30, 4099)])
        y = rng.poisson(model.forward_model(Q, S, lt)).astype(float)
        l = 0.8 * lt
        spec = psps.Spectrum(Q, S)
        got = to_host(psps.mbmd_curvature(None, spec, to_dev(l), to_dev(y)))
        want = model.curvature_numerator(Q, S, l, y, np.ones_like(l))
        assert rel_l2(got, want) < 1e-5, rel_l2(got, want)
        return
    g = small_geoms()["fan2d_ragged"]
    A = oracle_lib.Projector(g)
    blur = None
    if case == "mbir":
        Q, S = np.ones((1, 1)), np.full((1, 1), 1e5)
        x_true = phantom(g, seed=2, nm=1)
        x = 0.5 * x_true
    else:
        Q, S = spectral(2)
        x_true = 20 * phantom(g, seed=3, nm=2)
        x = 0.6 * x_true
        if case == "spectral-blur":
            blur = model.Blur([0.1, 0.2, 0.5, 0.15, 0.05], g.n_u)
    nm = Q.shape[1]
    y = np.random.default_rng(4).poisson(model.forward_model(Q, S, A.project(x_true), blur)).astype(float)
    plan = psps.Plan(g)
    spec = psps.Spectrum(Q, S)
    if blur is not None:
        spec.set_blur(blur.b, g.n_u)
    got = to_host(psps.mbmd_curvature(plan, spec, to_dev(x), to_dev(y)))
    gamma = A.project(np.ones((nm,) + g.image_shape))
    want = A.backproject(model.curvature_numerator(Q, S, A.project(x), y, gamma, blur))
    assert rel_l2(got, want) < 1e-5, rel_l2(got, want)
    assert np.all(got >= -1e-6 * np.abs(want).max())
