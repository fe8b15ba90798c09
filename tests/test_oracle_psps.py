"""Pins for the oracle SPS / preconditioned-SPS iteration (CPU): monotone
descent, majorisation by the separable surrogate, and convergence to the
minimiser found by brute force (dense FP64 Newton) on tiny problems."""
import math

import numpy as np
import pytest

import synth
from synth import FAN2D, PAR2D, Geometry


def tiny_mbir(oracle_lib, n=8, views=12, bins=13, beta=20.0, I0=1e4, seed=0):
    from oracle import psps
    g = Geometry(PAR2D, n, n, 1, 1.0, 1.0, 1.0, views, 0.0, math.pi, bins, 1, 1.0 * n / 8, 1.0)
    A = oracle_lib.Projector(g)
    rng = np.random.default_rng(seed)
    img = synth.render(g, [synth.Ellipse(0.4, -0.3, 0.3 * n, 0.25 * n, 0.3, 0.05),
                           synth.Ellipse(-0.8, 0.5, 0.1 * n, 0.12 * n, 0.0, 0.03)])
    y = rng.poisson(I0 * np.exp(-A.project(img[None]))).astype(float)
    return psps.Setup(A, np.ones((1, 1)), np.full((1, 1), I0), y, np.array([[beta]])), img


def tiny_mbmd(oracle_lib, n=8, seed=1):
    from oracle import model, psps
    g = Geometry(FAN2D, n, n, 1, 1.0, 1.0, 1.0, 14, 0.0, 2 * math.pi, 15, 1, 1.5, 1.0, 30.0, 60.0)
    A = oracle_lib.Projector(g)
    rng = np.random.default_rng(seed)
    E = np.arange(20.0, 81.0)
    Q = synth.material_Q(E, ["water", "bone"], rng)
    S = np.stack([1e4 * synth.kramers(E, 60.0), 1e4 * synth.kramers(E, 80.0)])
    x = np.stack([synth.render(g, [synth.Ellipse(0, 0, 3.0, 2.5, 0.0, 1.0)]),
                  synth.render(g, [synth.Ellipse(0.5, 0.2, 1.0, 1.2, 0.0, 1.5)])])
    y = rng.poisson(model.forward_model(Q, S, A.project(x))).astype(float)
    beta = np.array([[30.0, 3.0], [3.0, 40.0]])
    return psps.Setup(A, Q, S, y, beta), x


def newton_minimiser(st, x0=None, iters=60):
    """Dense FP64 damped Newton (Hessian by central differences of the exact
    gradient) to a gradient norm near machine precision."""
    x = st.zeros() if x0 is None else x0.copy()
    n = x.size
    for _ in range(iters):
        g = st.gradient(x).ravel()
        if np.linalg.norm(g) < 1e-11 * max(1.0, abs(st.objective(x))):
            break
        H = np.zeros((n, n))
        h = 1e-6
        for j in range(n):
            e = np.zeros(n)
            e[j] = h
            H[:, j] = (st.gradient(x + e.reshape(x.shape)).ravel() - st.gradient(x - e.reshape(x.shape)).ravel()) / (2 * h)
        H = 0.5 * (H + H.T)
        w, V = np.linalg.eigh(H)
        step = -(V @ ((V.T @ g) / np.maximum(w, 1e-12 * w.max()))).reshape(x.shape)
        f0 = st.objective(x)
        a = 1.0
        while st.objective(x + a * step) > f0 and a > 1e-8:
            a *= 0.5
        x = x + a * step
    return x


def test_plain_sps_nonneg_monotone(oracle_lib):
    """With x >= 0 (so l >= 0) and A, S, Q >= 0 the maximum-curvature SPS
    surrogate majorises Phi and plain SPS decreases it monotonically."""
    from oracle import precond, psps
    st, _ = tiny_mbir(oracle_lib, n=16, views=20, bins=23)
    _, h = psps.run(st, precond.Identity(), 40, None, nonneg=True)
    assert np.all(np.diff(h) <= 1e-12 * h[0])
    assert h[-1] < 0.2 * h[0]


@pytest.mark.parametrize("kind", ["none", "fourier", "mod_fourier", "haar", "block"])
def test_psps_linesearch_monotone(oracle_lib, kind):
    from oracle import build, psps
    st, _ = tiny_mbir(oracle_lib, n=16, views=20, bins=23)
    P = build.build(st, kind)
    _, h = psps.run(st, P, 25, psps.LineSearch())
    assert np.all(np.diff(h) <= 1e-12 * h[0])


def test_mbmd_linesearch_monotone(oracle_lib):
    from oracle import build, psps
    st, _ = tiny_mbmd(oracle_lib)
    for kind in ["none", "block", "block_fourier"]:
        _, h = psps.run(st, build.build(st, kind), 15, psps.LineSearch())
        assert np.all(np.diff(h) <= 1e-12 * h[0]), kind


def test_surrogate_majorises_preconditioned(oracle_lib):
    """Phi(x + M d) <= Phi(x) + grad'.d + 1/2 sum d'_j d_j^2 for small random
    d around a strictly positive x (so that l stays inside the range where the
    maximum curvature holds)."""
    from oracle import build, model, psps
    st, img = tiny_mbir(oracle_lib, n=8)
    x = img[None] + 0.01
    l = st.proj.project(x)
    Q, S, y = st.Q, st.S, st.y
    for kind in ["none", "mod_fourier", "haar"]:
        P = build.build(st, kind)
        absM1 = P.absM(np.ones_like(x))
        gm = st.proj.project(absM1)
        dR = P.absMT(st.pen.abs_apply(absM1))
        kappa = model.curvature_numerator(Q, S, l, y, gm)
        dp = P.absMT(st.proj.backproject(kappa)) + dR
        gp = P.MT(st.gradient(x))
        f0 = st.objective(x)
        rng = np.random.default_rng(7)
        for _ in range(30):
            d = rng.standard_normal(x.shape)
            d *= 0.005 / np.abs(P.M(d)).max()
            surr = f0 + np.sum(gp * d) + 0.5 * np.sum(dp * d * d)
            assert st.objective(x + P.M(d)) <= surr + 1e-10 * abs(f0), kind


def test_converges_to_bruteforce_minimiser(oracle_lib):
    from oracle import build, psps
    st, img = tiny_mbir(oracle_lib, n=8, views=24, beta=1000.0)
    xs = newton_minimiser(st, x0=img[None].copy())
    fs = st.objective(xs)
    # plain and preconditioned SPS are diagonally / basis-scaled descent
    # methods: the tolerances follow their (measured) rates on this problem
    for kind, tol in [("none", 1e-2), ("mod_fourier", 1e-3), ("haar", 1e-6)]:
        x, h = psps.run(st, build.build(st, kind), 300, psps.LineSearch())
        assert h.min() >= fs - 1e-9 * abs(fs), kind
        err = np.linalg.norm(x - xs) / np.linalg.norm(xs)
        assert err <= tol, (kind, err)


def test_ideal_preconditioner_is_fast(oracle_lib):
    """With the ideal M = H^-1/2 (dense eigendecomposition at the minimiser,
    Eq. 17) PSPS closes the objective gap far faster than plain SPS.  (It is
    not a one-step Newton method: the separable curvature of the surrogate
    for the signed operator A M is not uniform across x'.)"""
    from oracle import psps
    st, img = tiny_mbir(oracle_lib, n=8, views=24, beta=1000.0)
    xs = newton_minimiser(st, x0=img[None].copy())
    fs = st.objective(xs)
    n = xs.size
    H = np.zeros((n, n))
    h = 1e-6
    for j in range(n):
        e = np.zeros(n)
        e[j] = h
        H[:, j] = (st.gradient(xs + e.reshape(xs.shape)).ravel() - st.gradient(xs - e.reshape(xs.shape)).ravel()) / (2 * h)
    w, V = np.linalg.eigh(0.5 * (H + H.T))
    Mh = V @ np.diag(w ** -0.5) @ V.T

    class Dense:
        def M(self, v):
            return (Mh @ v.ravel()).reshape(v.shape)
        MT = M

        def absM(self, v):
            return (np.abs(Mh) @ v.ravel()).reshape(v.shape)
        absMT = absM
    from oracle import precond
    _, hi = psps.run(st, Dense(), 10, psps.LineSearch())
    _, hs = psps.run(st, precond.Identity(), 10, psps.LineSearch())
    gap_i = (hi[-1] - fs) / (hi[0] - fs)
    gap_s = (hs[-1] - fs) / (hs[0] - fs)
    assert gap_i < 1e-4, gap_i
    assert gap_i < 0.1 * gap_s


def test_blurred_model_sps_monotone(oracle_lib):
    """With a detector blur in the model (B S outside the exponential) the
    SPS surrogate still majorises: plain SPS with x >= 0 and the
    preconditioned iterations with the line search decrease Phi every
    iteration, and the converged objective beats the blur-free model's fit to
    the same blurred data."""
    from oracle import build, model, psps
    st0, img = tiny_mbir(oracle_lib, n=16, views=20, bins=23)
    blur = model.Blur([0.25, 0.5, 0.25], 23)
    rng = np.random.default_rng(3)
    y = rng.poisson(model.forward_model(st0.Q, st0.S, st0.proj.project(img[None]), blur)).astype(float)
    st = psps.Setup(st0.proj, st0.Q, st0.S, y, np.array([[20.0]]), blur=blur)
    _, h = psps.run(st, build.build(st, "none"), 40, None, nonneg=True)
    assert np.all(np.diff(h) <= 1e-12 * h[0])
    for kind in ["none", "mod_fourier"]:
        xb, hb = psps.run(st, build.build(st, kind), 25, psps.LineSearch())
        assert np.all(np.diff(hb) <= 1e-12 * hb[0]), kind
    st_nb = psps.Setup(st0.proj, st0.Q, st0.S, y, np.array([[20.0]]))
    x_nb, _ = psps.run(st_nb, build.build(st_nb, "mod_fourier"), 25, psps.LineSearch())
    assert st.objective(xb) < st.objective(x_nb)


def test_correlated_noise_sps_monotone(oracle_lib):
    """Correlated detector noise (Sigma_y with a first-order autoregressive
    correlation along detector rows, negative entries in Sigma^-1): with the
    |P| 1 curvature the SPS surrogate still majorises, so plain SPS with
    x >= 0 and the preconditioned iterations with the line search decrease
    Phi every iteration, also together with a detector blur."""
    from oracle import build, model, psps
    st0, img = tiny_mbir(oracle_lib, n=16, views=20, bins=23)
    rng = np.random.default_rng(4)
    noise = model.RowCorrelation(0.6, 23)
    for blur in (None, model.Blur([0.25, 0.5, 0.25], 23)):
        y = rng.poisson(model.forward_model(st0.Q, st0.S, st0.proj.project(img[None]), blur)).astype(float)
        st = psps.Setup(st0.proj, st0.Q, st0.S, y, np.array([[20.0]]), blur=blur, noise=noise)
        _, h = psps.run(st, build.build(st, "none"), 40, None, nonneg=True)
        assert np.all(np.diff(h) <= 1e-12 * h[0])
        for kind in ["none", "haar"]:
            _, hb = psps.run(st, build.build(st, kind), 25, psps.LineSearch())
            assert np.all(np.diff(hb) <= 1e-12 * hb[0]), kind
            assert hb[-1] < 0.2 * hb[0]
