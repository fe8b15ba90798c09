"""Pins for the oracle forward model, objective, gradient, SPS curvature,
penalty and water fit (CPU)."""
import math

import numpy as np
import pytest

import synth
from synth import FAN2D, PAR2D, Geometry


def small_spectral(nm=2, ne=7, nc=3, seed=0):
    rng = np.random.default_rng(seed)
    Q = rng.uniform(0.01, 0.05, (ne, nm))
    S = rng.uniform(10.0, 200.0, (nc, ne))
    return Q, S


def test_monoenergetic_reduces_to_beer_lambert(oracle_lib):
    """One energy, one channel, Q = 1, S = I0: y_bar = I0 exp(-l)."""
    from oracle import model
    l = np.array([[0.0, 0.5, 2.0, -0.3]])
    got = model.forward_model(np.ones((1, 1)), np.full((1, 1), 1e4), l)
    assert np.allclose(got[0], 1e4 * np.array([1.0, math.exp(-0.5), math.exp(-2.0), math.exp(0.3)]),
                       rtol=1e-15)


def test_energy_independent_attenuation(oracle_lib):
    """Q with identical rows: every channel sees exp(-q.l) times its total
    sensitivity sum_E S[c,E] (non-square shapes catch transposes)."""
    from oracle import model
    rng = np.random.default_rng(1)
    q = np.array([0.02, 0.07])
    Q = np.tile(q, (5, 1))
    S = rng.uniform(1, 10, (3, 5))
    l = rng.uniform(0, 30, (2, 11))
    got = model.forward_model(Q, S, l)
    want = S.sum(1)[:, None] * np.exp(-(q @ l))[None, :]
    assert np.allclose(got, want, rtol=1e-14)


def _fd_check(f, grad, x, h_rel=1e-6, n_dir=6, seed=0):
    rng = np.random.default_rng(seed)
    for _ in range(n_dir):
        v = rng.standard_normal(x.shape)
        h = h_rel * max(1.0, np.abs(x).max())
        fd = (f(x + h * v) - f(x - h * v)) / (2 * h)
        an = float(np.sum(grad * v))
        assert abs(fd - an) <= 1e-7 * max(abs(an), abs(fd), 1e-30) + 1e-9 * abs(f(x)), (fd, an)


@pytest.mark.parametrize("spectral", [False, True])
def test_gradient_finite_differences(oracle_lib, spectral):
    from oracle import psps
    g = Geometry(FAN2D, 10, 9, 1, 1.0, 1.0, 1.0, 15, 0.0, 2 * math.pi, 17, 1, 1.2, 1.0, 40.0, 80.0)
    A = oracle_lib.Projector(g)
    rng = np.random.default_rng(2)
    if spectral:
        Q, S = small_spectral()
        beta = np.array([[3.0, 0.4], [0.4, 2.0]])
        x = rng.uniform(0, 2.0, (2, 9, 10))
    else:
        Q, S = np.ones((1, 1)), np.full((1, 1), 1e3)
        beta = np.array([[5.0]])
        x = rng.uniform(0, 0.05, (1, 9, 10))
    l = A.project(x)
    from oracle import model
    y = np.round(model.forward_model(Q, S, l) * rng.uniform(0.9, 1.1, (S.shape[0], g.n_rays)))
    st = psps.Setup(A, Q, S, y, beta)
    _fd_check(lambda z: st.objective(z), st.gradient(x), x)


def test_sps_curvature_majorises():
    """The parabola with curvature c touching h(z) = 1/2 eta e^{-2z} + rho
    e^{-z} at z^n lies above h on z >= min(0, z^n) for every ray/energy; the
    construction is exercised with eta, rho from random spectra and data."""
    from oracle import model
    rng = np.random.default_rng(4)
    Q, S = small_spectral(nm=2, ne=6, nc=3, seed=5)
    l = rng.uniform(-0.5, 40.0, (2, 400))
    y = rng.poisson(model.forward_model(Q, S, rng.uniform(0, 40, (2, 400)))).astype(float)
    w = model.weights(y)
    t = model.transmission(Q, l)
    r = S @ t - y
    eta = S.T @ (w * S.sum(1)[:, None])
    rho = S.T @ (w * r) - eta * t
    c = model.sps_curvature(Q, S, l, y)
    zn = Q @ l

    def h(z):
        return 0.5 * eta * np.exp(-2 * z) + rho * np.exp(-z)

    def dh(z):
        return -eta * np.exp(-2 * z) - rho * np.exp(-z)
    for s in np.linspace(0, 1, 41):
        lo = np.minimum(0.0, zn)
        z = lo + s * (zn + 3.0 - lo)
        surr = h(zn) + dh(zn) * (z - zn) + 0.5 * c * (z - zn) ** 2
        assert np.all(surr >= h(z) - 1e-9 * (np.abs(h(z)) + 1))
    # the surrogate's gradient at z^n is the true data gradient (paper's rho
    # with t^n): -Q^T (eta t^2 + rho t) == dL/dl
    gs = -(Q.T @ (eta * t * t + rho * t))
    assert np.allclose(gs, model.data_grad_l(Q, S, l, y), rtol=1e-12, atol=1e-12 * np.abs(gs).max())


def test_fisher_blocks_are_gauss_newton_hessian():
    """At noiseless data the Hessian of L in l is J^T W J = F_i (FD check)."""
    from oracle import model
    rng = np.random.default_rng(6)
    Q, S = small_spectral(nm=3, ne=8, nc=4, seed=7)
    l = rng.uniform(0, 20, (3, 5))
    y = model.forward_model(Q, S, l)
    F = model.fisher_blocks(Q, S, y, model.transmission(Q, l))
    h = 1e-5
    for i in range(5):
        H = np.zeros((3, 3))
        for a in range(3):
            e = np.zeros((3, 5))
            e[a, i] = h
            H[:, a] = (model.data_grad_l(Q, S, l + e, y)[:, i] - model.data_grad_l(Q, S, l - e, y)[:, i]) / (2 * h)
        assert np.allclose(H, F[i], rtol=1e-6, atol=1e-8 * np.abs(F[i]).max())


def test_water_fit_recovers_water():
    from oracle import model
    E = np.arange(20.0, 121.0)
    Q = synth.material_Q(E, ["water", "bone"], np.random.default_rng(0))
    S = np.stack([1e5 * synth.kramers(E, 80.0), 1e5 * synth.kramers(E, 120.0)])
    lw = np.array([0.0, 10.0, 100.0, 250.0])
    y = model.forward_model(Q, S, np.stack([lw, np.zeros(4)]))
    assert np.allclose(model.water_fit(Q, S, y), lw, rtol=1e-7, atol=1e-7)


# ---------------------------------------------------------------------------
# penalty
# ---------------------------------------------------------------------------

def _pairs(shape):
    idx = np.arange(int(np.prod(shape))).reshape(shape)
    out = []
    for ax in range(len(shape)):
        a = np.moveaxis(idx, ax, 0)
        out += list(zip(a[:-1].ravel(), a[1:].ravel()))
    return out


@pytest.mark.parametrize("shape", [(5, 7), (3, 4, 5)])
def test_penalty_pairs_and_gradient(shape):
    from oracle.penalty import Penalty, gamma_apply
    rng = np.random.default_rng(8)
    beta = np.array([[2.0, 0.3], [0.3, 1.5]])
    x = rng.standard_normal((2,) + shape)
    pen = Penalty(beta)
    xf = x.reshape(2, -1)
    want = 0.0
    for j, k in _pairs(shape):
        dj = xf[:, j] - xf[:, k]
        want += 0.5 * float(dj @ beta @ dj)
    assert abs(pen.value(x) - want) <= 1e-12 * abs(want)
    assert np.allclose(gamma_apply(np.ones(shape)), 0.0)
    _fd_check(pen.value, pen.apply(x), x)
    # |Gamma| 1 = 2 |N_j|
    nb = np.zeros(int(np.prod(shape)))
    for j, k in _pairs(shape):
        nb[j] += 1
        nb[k] += 1
    assert np.allclose(pen.abs_apply(np.ones((2,) + shape))[0].ravel(), 2 * nb * np.abs(beta[0]).sum())


# ---------------------------------------------------------------------------
# detector blur B (the operator outside the exponential is B S)

def _blur_case(seed=8, nm=2, ne=5, nc=2, n_rows=3, n_u=7):
    from oracle import model
    rng = np.random.default_rng(seed)
    Q, S = small_spectral(nm=nm, ne=ne, nc=nc, seed=seed)
    blur = model.Blur([0.2, 0.5, 0.3], n_u)          # deliberately not symmetric
    n = n_rows * n_u
    l = rng.uniform(0.0, 30.0, (nm, n))
    y = rng.poisson(model.forward_model(Q, S, rng.uniform(0, 30, (nm, n)), blur)).astype(float)
    return Q, S, blur, l, y, n


def _dense_blur(blur, n):
    """B as a dense n x n matrix, built from its definition cell by cell."""
    Bd = np.zeros((n, n))
    for i in range(n):
        row, j = divmod(i, blur.n_u)
        for k in range(-blur.R, blur.R + 1):
            if 0 <= j + k < blur.n_u:
                Bd[i, row * blur.n_u + j + k] = blur.b[k + blur.R]
    return Bd


def test_blur_definition_and_transpose():
    """B applied to unit vectors gives the taps clipped at the row ends; B^T is
    its transpose (<B u, v> = <u, B^T v>)."""
    from oracle import model
    blur = model.Blur([0.1, 0.2, 0.4, 0.2, 0.1], 6)
    n = 18
    Bd = _dense_blur(blur, n)
    eye = np.eye(n)
    got = np.stack([blur.apply(eye[j][None])[0] for j in range(n)], 1)
    assert np.allclose(got, Bd, atol=1e-15)
    gotT = np.stack([blur.applyT(eye[j][None])[0] for j in range(n)], 1)
    assert np.allclose(gotT, Bd.T, atol=1e-15)


def test_identity_blur_is_no_blur():
    from oracle import model
    Q, S, _, l, y, n = _blur_case()
    one = model.Blur([1.0], 7)
    assert np.allclose(model.forward_model(Q, S, l, one), model.forward_model(Q, S, l), rtol=1e-15)
    assert np.allclose(model.data_grad_l(Q, S, l, y, one), model.data_grad_l(Q, S, l, y), rtol=1e-14)
    assert np.allclose(model.sps_curvature(Q, S, l, y, one), model.sps_curvature(Q, S, l, y), rtol=1e-14)


def test_blur_eta_rho_dense():
    """eta and rho of Eqs. 8 and 10 with the dense operator (B S) over the
    (energy, ray) unknowns: eta = P 1, rho = P t - eta t - (BS)^T W y,
    P = (BS)^T W (BS)."""
    from oracle import model
    Q, S, blur, l, y, n = _blur_case()
    ne, nc = S.shape[1], S.shape[0]
    Bd = _dense_blur(blur, n)
    # (B S) maps t[E, i] (flattened E-major) to y_bar[c, i] (c-major)
    BS = np.einsum("ce,ij->ciej", S, Bd).reshape(nc * n, ne * n)
    W = np.diag(model.weights(y).ravel())
    P = BS.T @ W @ BS
    t = model.transmission(Q, l).ravel()
    eta_d = P @ np.ones(ne * n)
    rho_d = P @ t - eta_d * t - BS.T @ W @ y.ravel()
    eta, rho, _ = model.sps_eta_rho(Q, S, l, y, blur)
    assert np.allclose(eta.ravel(), eta_d, rtol=1e-12)
    assert np.allclose(rho.ravel(), rho_d, rtol=1e-10, atol=1e-10 * np.abs(rho_d).max())


def test_blur_gradient_finite_differences():
    from oracle import model
    Q, S, blur, l, y, n = _blur_case(seed=9)
    _fd_check(lambda z: model.data_objective(Q, S, z, y, blur), model.data_grad_l(Q, S, l, y, blur), l)


def test_blur_surrogate_majorises():
    """With eta = P 1 (P = (BS)^T W (BS) has nonnegative entries) the separable
    sum of h(z) = 1/2 eta e^{-2z} + rho e^{-z} over every (energy, ray)
    majorises the data term as a function of the exponents z, touching it at
    the current point: L(z) - L(z^n) <= sum h(z) - h(z^n) for any z."""
    from oracle import model
    Q, S, blur, l, y, n = _blur_case(seed=10)
    eta, rho, t0 = model.sps_eta_rho(Q, S, l, y, blur)
    z0 = Q @ l
    w = model.weights(y)

    def L(z):
        r = blur.apply(S @ np.exp(-z)) - y
        return 0.5 * float(np.sum(w * r * r))

    def H(z):
        return float(np.sum(0.5 * eta * np.exp(-2 * z) + rho * np.exp(-z)))
    rng = np.random.default_rng(11)
    for _ in range(50):
        z = z0 + rng.normal(0.0, 0.5, z0.shape)
        assert L(z) - L(z0) <= H(z) - H(z0) + 1e-9 * (abs(L(z0)) + 1)


# ---------------------------------------------------------------------------
# Correlated detector noise (non-diagonal Sigma_y)
# ---------------------------------------------------------------------------

def _dense_sigma(noise, y_c):
    """Sigma_y of one channel as a dense matrix, from its definition:
    D^1/2 C D^1/2, C[j, k] = a^|j-k| within each row of n_u cells."""
    n = y_c.size
    C = np.zeros((n, n))
    for i in range(n):
        ri, ji = divmod(i, noise.n_u)
        for k in range(n):
            rk, jk = divmod(k, noise.n_u)
            if ri == rk:
                C[i, k] = noise.a ** abs(ji - jk)
    d = np.sqrt(np.maximum(y_c, 1.0))
    return d[:, None] * C * d[None, :]


def test_row_correlation_inverse():
    """The tridiagonal W of RowCorrelation is the inverse of the dense
    covariance built from the definition, and |W| its elementwise modulus."""
    from oracle import model
    rng = np.random.default_rng(21)
    noise = model.RowCorrelation(0.6, 5)
    y = rng.uniform(0.5, 400.0, (2, 15))
    eye = np.eye(15)
    for c in range(2):
        Wd = np.linalg.inv(_dense_sigma(noise, y[c]))
        cols = []
        for j in range(15):
            v = np.zeros((2, 15))
            v[c] = eye[j]
            cols.append(noise.W(v, y)[c])
        got = np.stack(cols, 1)
        assert np.allclose(got, Wd, rtol=1e-11, atol=1e-13 * np.abs(Wd).max())
        cols = []
        for j in range(15):
            v = np.zeros((2, 15))
            v[c] = eye[j]
            cols.append(noise.absW(v, y)[c])
        assert np.allclose(np.stack(cols, 1), np.abs(Wd), rtol=1e-11, atol=1e-13 * np.abs(Wd).max())


def test_zero_correlation_is_diagonal():
    from oracle import model
    Q, S, blur, l, y, n = _blur_case(seed=22)
    none = model.RowCorrelation(0.0, 7)
    for b in (None, blur):
        assert np.isclose(model.data_objective(Q, S, l, y, b, none), model.data_objective(Q, S, l, y, b), rtol=1e-14)
        assert np.allclose(model.data_grad_l(Q, S, l, y, b, none), model.data_grad_l(Q, S, l, y, b), rtol=1e-13)
        assert np.allclose(model.sps_curvature(Q, S, l, y, b, none), model.sps_curvature(Q, S, l, y, b),
                           rtol=1e-13)


def test_correlated_objective_dense_and_gradient():
    """L = 1/2 r^T Sigma^-1 r with the dense covariance, and the gradient
    against central finite differences (blur and correlation together)."""
    from oracle import model
    Q, S, blur, l, y, n = _blur_case(seed=23)
    noise = model.RowCorrelation(0.45, 7)
    r = model.forward_model(Q, S, l, blur) - y
    want = 0.5 * sum(float(r[c] @ np.linalg.solve(_dense_sigma(noise, y[c]), r[c])) for c in range(y.shape[0]))
    got = model.data_objective(Q, S, l, y, blur, noise)
    assert abs(got - want) <= 1e-11 * abs(want)
    _fd_check(lambda z: model.data_objective(Q, S, z, y, blur, noise), model.data_grad_l(Q, S, l, y, blur, noise), l)


def test_correlated_line_terms():
    """phi, phi', phi'' of the correlated data term along a direction equal
    the objective and its finite-difference derivatives."""
    from oracle import model
    Q, S, blur, l, y, n = _blur_case(seed=24)
    noise = model.RowCorrelation(0.3, 7)
    q = np.random.default_rng(25).normal(0.0, 1.0, l.shape)
    a, h = 0.2, 1e-4
    f, f1, f2 = model.line_terms(Q, S, l, q, y, a, blur, noise)
    phi = lambda t: model.data_objective(Q, S, l + t * q, y, blur, noise)  # noqa: E731
    assert abs(f - phi(a)) <= 1e-12 * abs(f)
    assert abs(f1 - (phi(a + h) - phi(a - h)) / (2 * h)) <= 1e-6 * abs(f1) + 1e-9 * abs(f)
    assert abs(f2 - (phi(a + h) - 2 * phi(a) + phi(a - h)) / h ** 2) <= 1e-4 * abs(f2) + 1e-7 * abs(f)


def test_correlated_surrogate_majorises():
    """With negative off-diagonal entries in Sigma^-1 the separable bound of
    Eqs. 8 and 10 uses eta = |P| 1 (P = (BS)^T Sigma^-1 (BS)); the sum of
    h(z) over every (energy, ray) still majorises the data term and touches
    it at the current point."""
    from oracle import model
    Q, S, blur, l, y, n = _blur_case(seed=26)
    noise = model.RowCorrelation(0.7, 7)
    eta, rho, t0 = model.sps_eta_rho(Q, S, l, y, blur, noise)
    z0 = Q @ l

    def L(z):
        r = blur.apply(S @ np.exp(-z)) - y
        return 0.5 * float(np.sum(r * noise.W(r, y)))

    def H(z):
        return float(np.sum(0.5 * eta * np.exp(-2 * z) + rho * np.exp(-z)))
    rng = np.random.default_rng(27)
    for _ in range(50):
        z = z0 + rng.normal(0.0, 0.5, z0.shape)
        assert L(z) - L(z0) <= H(z) - H(z0) + 1e-9 * (abs(L(z0)) + 1)
    # negative control: one energy, one channel, no blur, strong correlation
    # (P = Sigma^-1 itself): eta = P 1 instead of |P| 1 fails to majorise
    # along a direction that moves neighbouring cells in opposite ways, while
    # |P| 1 holds there
    Q1, S1 = np.ones((1, 1)), np.full((1, 1), 1e4)
    noise1 = model.RowCorrelation(0.9, 8)
    l1 = np.full((1, 16), 1.0)
    y1 = np.full((1, 16), 1e4 * np.exp(-1.2))
    eta1, rho1, t1 = model.sps_eta_rho(Q1, S1, l1, y1, None, noise1)
    eta_w = S1.T @ noise1.W(np.full((1, 16), S1.sum()), y1)
    rho_w = rho1 + (eta1 - eta_w) * t1
    z0 = Q1 @ l1
    z = z0 + 0.3 * np.where(np.arange(16) % 2 == 0, 1.0, -1.0)[None, :]

    def L1(zz):
        r = S1 @ np.exp(-zz) - y1
        return 0.5 * float(np.sum(r * noise1.W(r, y1)))

    def Hs(e, rh, zz):
        return float(np.sum(0.5 * e * np.exp(-2 * zz) + rh * np.exp(-zz)))
    assert L1(z) - L1(z0) <= Hs(eta1, rho1, z) - Hs(eta1, rho1, z0) + 1e-9 * abs(L1(z0))
    assert L1(z) - L1(z0) > Hs(eta_w, rho_w, z) - Hs(eta_w, rho_w, z0) + 1e-6 * abs(L1(z) - L1(z0))


@pytest.mark.parametrize("with_blur", [False, True])
def test_line_terms_derivatives(with_blur):
    """phi, phi', phi'' of the data term along a direction (diagonal
    Sigma_y, with and without a detector blur) equal the objective and its
    central differences."""
    from oracle import model
    Q, S, blur, l, y, n = _blur_case(seed=31)
    blur = blur if with_blur else None
    q = np.random.default_rng(32).normal(0.0, 1.0, l.shape)
    a, h = 0.3, 1e-4
    f, f1, f2 = model.line_terms(Q, S, l, q, y, a, blur)
    phi = lambda t: model.data_objective(Q, S, l + t * q, y, blur)  # noqa: E731
    assert abs(f - phi(a)) <= 1e-12 * abs(f)
    assert abs(f1 - (phi(a + h) - phi(a - h)) / (2 * h)) <= 1e-6 * abs(f1) + 1e-9 * abs(f)
    assert abs(f2 - (phi(a + h) - 2 * phi(a) + phi(a - h)) / h ** 2) <= 1e-4 * abs(f2) + 1e-7 * abs(f)


def test_line_terms_one_ray_closed_form():
    """One ray, one energy (Beer-Lambert): phi(a) = 1/2 w (I0 e^-(l + a q) - y)^2
    with w = 1 / y, so phi' = -w r I0 q e^-z and
    phi'' = w I0^2 q^2 e^-2z + w r I0 q^2 e^-z (r = I0 e^-z - y, z = l + a q)."""
    from oracle import model
    I0, l0, q, y, a = 1.0e4, 0.7, 0.013, 3100.0, 11.0
    z = l0 + a * q
    r = I0 * math.exp(-z) - y
    w = 1.0 / y
    f, f1, f2 = model.line_terms(np.ones((1, 1)), np.full((1, 1), I0), np.array([[l0]]), np.array([[q]]),
                                 np.array([[y]]), a)
    assert abs(f - 0.5 * w * r * r) <= 1e-13 * abs(f)
    assert abs(f1 - (-w * r * I0 * q * math.exp(-z))) <= 1e-13 * abs(f1)
    assert abs(f2 - (w * (I0 * q * math.exp(-z)) ** 2 + w * r * I0 * q * q * math.exp(-z))) <= 1e-13 * abs(f2)


def _rule(phi, dphi, d2phi, a0, n_ls=3, n_halve=8, trust=8.0, alpha_max=1e12):
    """The line-search rule as stated (reading R8), written out for a scalar
    phi given in closed form: n_ls evaluations starting at a0, each followed
    (but the last) by a Newton step kept within [a / trust, a trust] and
    below alpha_max (a kept when phi'' <= 0); accept the last evaluated a if
    phi(a) <= phi(0), else halve up to n_halve times, else 0.  Returns
    (alpha, evaluated points, clipped, halvings)."""
    a, pts, clipped = a0, [], False
    for k in range(n_ls):
        pts.append(a)
        if k + 1 < n_ls:
            if d2phi(a) > 0:
                newton = a - dphi(a) / d2phi(a)
                an = min(max(newton, a / trust), a * trust)
                clipped |= an != newton
            else:
                an = a
            a = min(an, alpha_max)
    if phi(a) <= phi(0.0):
        return a, pts, clipped, 0
    for h in range(1, n_halve + 1):
        a = 0.5 * a
        if phi(a) <= phi(0.0):
            return a, pts, clipped, h
    return 0.0, pts, clipped, n_halve + 1


@pytest.mark.parametrize("case", ["newton_inside", "clipped", "halved"])
def test_line_search_worked_example(case):
    """The oracle's safeguarded line search against the stated rule on a
    one-ray problem whose phi is known in closed form (projection domain,
    one material and energy, no penalty): a Newton step inside the trust
    region, steps clipped by the factor-8 trust bound (the minimiser far
    out), and an overshooting warm start that needs halvings.  A different
    trust factor, halving count or acceptance test changes alpha."""
    import oracle
    from oracle import psps as opsps
    I0, q = 1.0e4, 1.0e-3
    y_of = {"newton_inside": I0 * math.exp(-3.0 * q), "clipped": I0 * math.exp(-500.0 * q),
            "halved": 0.9 * I0}
    a0 = {"newton_inside": 1.0, "clipped": 1.0, "halved": 4000.0}[case]
    y = y_of[case]
    st = opsps.Setup(oracle.IdentityProjector(1), np.ones((1, 1)), np.full((1, 1), I0), np.array([[y]]), None)
    x = np.zeros((1, 1))
    p = np.full((1, 1), q)
    w = 1.0 / y

    def phi(a):
        return 0.5 * w * (I0 * math.exp(-a * q) - y) ** 2

    def dphi(a):
        return -w * (I0 * math.exp(-a * q) - y) * I0 * q * math.exp(-a * q)

    def d2phi(a):
        e = math.exp(-a * q)
        return w * (I0 * q * e) ** 2 + w * (I0 * e - y) * I0 * q * q * e
    want, pts, clipped, halvings = _rule(phi, dphi, d2phi, a0)
    got, f, _ = opsps.line_search(st, x, p, np.zeros((1, 1)), p.copy(), phi(0.0), opsps.LineSearch(), a0)
    assert abs(got - want) <= 1e-12 * max(abs(want), 1.0), (case, got, want, pts)
    if case == "clipped":
        assert clipped and want == 64.0
    if case == "halved":
        assert halvings >= 1
    if case == "newton_inside":
        assert not clipped and abs(want - 3.0) < 0.5
