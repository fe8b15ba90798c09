"""Oracle forward model, PWLS objective, gradient and SPS per-ray quantities.

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.

Notation: rays i, energies E, channels c, materials m.  l[m,i] are material
line integrals (l = A x_m for the image problems, l = x for projection-domain
decomposition), Q[E,m] mass attenuation per unit density, S[c,E] the channel
sensitivity with the gain folded in (MBIR: one energy, one channel, Q = 1,
S = I0).  Everything is FP64.

The operator outside the exponential (Eq. 1) is B S: the spectral
sensitivity S followed, optionally, by a detector blur B (``Blur``) that
mixes neighbouring detector cells of one row in every channel.  With B the
SPS quantities of Eqs. 8 and 10 couple neighbouring rays:
eta = S^T B^T Sigma^-1 B S 1 and rho = S^T B^T Sigma^-1 (B S t - y) - eta t.
"""
from __future__ import annotations

import numpy as np


class Blur:
    """Detector blur B: in every channel and detector row (n_u consecutive
    rays), [B v]_i = sum_k b_k v_{i+k} for k = -R..R, zero past the ends of
    the row.  taps = (b_-R, ..., b_R)."""

    def __init__(self, taps, n_u: int):
        self.b = np.asarray(taps, dtype=np.float64)
        assert self.b.ndim == 1 and self.b.size % 2 == 1
        self.R = self.b.size // 2
        self.n_u = int(n_u)

    def _corr(self, v, b):
        shp = v.shape
        rows = v.reshape(shp[0], -1, self.n_u)
        pad = np.zeros(rows.shape[:-1] + (self.n_u + 2 * self.R,))
        pad[..., self.R:self.R + self.n_u] = rows
        out = np.zeros_like(rows)
        for j, bk in enumerate(b):          # k = j - R
            out += bk * pad[..., j:j + self.n_u]
        return out.reshape(shp)

    def apply(self, v):
        """B v for v[c, rays]."""
        return self._corr(v, self.b)

    def applyT(self, v):
        """B^T v: [B^T v]_i = sum_k b_k v_{i-k}."""
        return self._corr(v, self.b[::-1])


def _B(blur, v):
    return v if blur is None else blur.apply(v)


def _BT(blur, v):
    return v if blur is None else blur.applyT(v)


def weights(y: np.ndarray) -> np.ndarray:
    """Inverse data covariance: Sigma_y = diag(max(y, 1)), a plug-in Poisson
    variance (the paper only says the covariance is known, Sec. II-A)."""
    return 1.0 / np.maximum(y, 1.0)


class RowCorrelation:
    """Correlated detector noise (a non-diagonal Sigma_y, Sec. II-A: the
    covariance is known): Sigma_y = D^1/2 C D^1/2 with D = diag(max(y, 1)) and,
    in every channel and detector row (n_u consecutive rays), the first-order
    autoregressive correlation C[j, k] = a^|j - k| between cells j, k of the
    row.  Its inverse is tridiagonal: (1 / (1 - a^2)) times 1 at the row ends
    and 1 + a^2 inside on the diagonal, -a next to it; so
    W = Sigma_y^-1 = D^-1/2 C^-1 D^-1/2 couples neighbouring cells only.  With
    a > 0, W has negative off-diagonal entries: the separable SPS bound then
    takes eta = S^T B^T |W| B S 1, which bounds |P| 1 elementwise for
    P = (B S)^T W (B S), and diag(|P| 1) - P is diagonally dominant, hence
    positive semidefinite."""

    def __init__(self, a: float, n_u: int):
        assert 0.0 <= a < 1.0 and n_u >= 2   # the closed-form inverse needs two cells per row
        self.a = float(a)
        self.n_u = int(n_u)

    def _cinv(self, v, sign):
        rows = v.reshape(v.shape[0], -1, self.n_u)
        a = self.a
        out = rows.copy()
        out[..., 1:-1] *= 1.0 + a * a
        out[..., 1:] += sign * a * rows[..., :-1]
        out[..., :-1] += sign * a * rows[..., 1:]
        return (out / (1.0 - a * a)).reshape(v.shape)

    def W(self, v, y):
        """Sigma_y^-1 v for v[c, rays]."""
        s = np.sqrt(weights(y))
        return s * self._cinv(s * v, -1.0)

    def absW(self, v, y):
        """|Sigma_y^-1| v (elementwise absolute value of the matrix)."""
        s = np.sqrt(weights(y))
        return s * self._cinv(s * v, +1.0)


def _W(noise, v, y):
    return weights(y) * v if noise is None else noise.W(v, y)


def _absW(noise, v, y):
    return weights(y) * v if noise is None else noise.absW(v, y)


def transmission(Q: np.ndarray, l: np.ndarray) -> np.ndarray:
    """t[E,i] = exp(-sum_m Q[E,m] l[m,i])  (the exp(-A x) of Eq. 1)."""
    return np.exp(-(Q @ l))


def forward_model(Q: np.ndarray, S: np.ndarray, l: np.ndarray, blur: Blur | None = None) -> np.ndarray:
    """Mean counts y_bar[c,i] = [B sum_E S[c,E] exp(-[Q l]_E)]_i  (Eq. 1 with the
    operator outside the exponential B -> B S, inside A -> Q or QA)."""
    return _B(blur, S @ transmission(Q, l))


def data_objective(Q, S, l, y, blur: Blur | None = None, noise: RowCorrelation | None = None) -> float:
    """L = 1/2 (y - y_bar)^T Sigma^-1 (y - y_bar)  (Eq. 3)."""
    r = forward_model(Q, S, l, blur) - y
    return 0.5 * float(np.sum(r * _W(noise, r, y)))


def data_grad_l(Q, S, l, y, blur: Blur | None = None, noise: RowCorrelation | None = None) -> np.ndarray:
    """dL/dl[m,i] = -sum_E Q[E,m] t[E,i] sum_c S[c,E] [B^T W (y_bar - y)][c,i]."""
    t = transmission(Q, l)
    r = _B(blur, S @ t) - y
    v = S.T @ _BT(blur, _W(noise, r, y))
    return -(Q.T @ (t * v))


def sps_eta_rho(Q, S, l, y, blur: Blur | None = None, noise: RowCorrelation | None = None):
    """eta = (B S)^T Sigma^-1 (B S) 1 and rho = (B S)^T Sigma^-1 (B S) t
    - eta t - (B S)^T Sigma^-1 y, per (energy, ray) (Eqs. 8, 10; the paper's
    rho printed with x^n where the current transmission t^n belongs).  With
    correlated noise eta uses |Sigma^-1| (see RowCorrelation)."""
    t = transmission(Q, l)
    r = _B(blur, S @ t) - y
    ones = np.broadcast_to(S.sum(axis=1)[:, None], r.shape)   # S 1 = sigma_c per ray
    eta = S.T @ _BT(blur, _absW(noise, _B(blur, np.array(ones)), y))
    rho = S.T @ _BT(blur, _W(noise, r, y)) - eta * t
    return eta, rho, t


def sps_curvature(Q, S, l, y, blur: Blur | None = None, noise: RowCorrelation | None = None) -> np.ndarray:
    """Per (energy, ray) maximum curvature c of the separable surrogate.

    The data term is majorised, for each ray and energy, by the 1-D function
    h(z) = 1/2 eta e^{-2z} + rho e^{-z} of z = [Q l]_E (Sec. II-B, Eqs. 4-11),
    with eta = B^T Sigma^-1 B 1 and rho = B^T Sigma^-1 B t^n - eta t^n
    - B^T Sigma^-1 y (the paper's rho printed with x^n where the current
    transmission t^n belongs).  h''(z) = 2 eta u^2 + rho u with u = e^{-z} is a
    convex quadratic in u, so its maximum over z >= min(0, z^n) sits at an
    end point: c = max(0, 2 eta u_hi^2 + rho u_hi), u_hi = max(1, t^n).  (The
    cited maximum-curvature rule is not in the paper; this is its derivation
    for this h.)
    """
    eta, rho, t = sps_eta_rho(Q, S, l, y, blur, noise)
    u_hi = np.maximum(1.0, t)
    return np.maximum(0.0, 2.0 * eta * u_hi * u_hi + rho * u_hi)


def curvature_numerator(Q, S, l, y, gamma_m: np.ndarray, blur: Blur | None = None,
                        noise: RowCorrelation | None = None) -> np.ndarray:
    """kappa[m,i] = sum_E Q[E,m] gamma[E,i] c[E,i] with gamma[E,i] =
    sum_m Q[E,m] gamma_m[m,i]; the separable curvature is then
    d = A^T kappa (Eq. 6: d = diag(A^T D{gamma} c) with A -> QA)."""
    c = sps_curvature(Q, S, l, y, blur, noise)
    gE = Q @ gamma_m
    return Q.T @ (gE * c)


def line_terms(Q, S, l, q, y, alpha: float, blur: Blur | None = None, noise: RowCorrelation | None = None):
    """Data part of phi(alpha) = L(l + alpha q) and its first two derivatives
    in alpha, summed over all rays."""
    la = l + alpha * q
    t = transmission(Q, la)
    r = _B(blur, S @ t) - y
    dz = Q @ q
    dyb = -_B(blur, S @ (t * dz))
    d2yb = _B(blur, S @ (t * dz * dz))
    Wr, Wd = _W(noise, r, y), _W(noise, dyb, y)
    f = 0.5 * float(np.sum(r * Wr))
    f1 = float(np.sum(dyb * Wr))
    f2 = float(np.sum(dyb * Wd + d2yb * Wr))
    return f, f1, f2


def water_fit(Q, S, y, water: int = 0, n_newton: int = 10) -> np.ndarray:
    """Per-ray single-material (water) line-integral estimate used to
    approximate D = D{exp(-Q l_hat)} before reconstruction (Sec. II-D: assume
    all attenuation is water).  Gauss-Newton on the per-ray PWLS misfit,
    10 iterations from l = 0, clamped to l >= 0."""
    w = weights(y)
    qw = Q[:, water][:, None]                 # [E, 1]
    lw = np.zeros(y.shape[1])
    for _ in range(n_newton):
        t = np.exp(-qw * lw[None, :])         # [E, i]
        r = S @ t - y                         # [c, i]
        J = -(S @ (qw * t))                   # d y_bar / d lw  [c, i]
        g = np.sum(w * r * J, axis=0)
        h = np.sum(w * J * J, axis=0)
        step = np.where(h > 0, g / np.where(h > 0, h, 1.0), 0.0)
        lw = np.maximum(lw - step, 0.0)
    return lw


def fisher_blocks(Q, S, y, t_hat: np.ndarray) -> np.ndarray:
    """Per-ray F_i = Q^T D_i S^T Sigma_i^-1 S D_i Q  ([i, m, m']), the block of
    the Fisher information in line-integral space (Sec. II-D/E Hessians with
    B = I, G folded into S), with D_i = diag(t_hat[:, i])."""
    w = weights(y)                            # [c, i]
    J = S[:, :, None] * (t_hat[None, :, :])   # [c, E, i] : S_cE t_Ei
    Jm = np.einsum("cei,em->cmi", J, Q)       # [c, m, i]
    return np.einsum("cmi,ci,cni->imn", Jm, w, Jm)
