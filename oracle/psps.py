"""Oracle (preconditioned) separable-parabolic-surrogates iteration.

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.

One iteration in the preconditioned basis x = M x' (Sec. II-B, II-C):
  1. l = A x is kept incrementally (l += alpha q) and recomputed exactly
     every ``reproject_every`` iterations and at the end;
  2. data gradient numerator g and curvature numerator kappa per ray;
  3. grad_x = A^T g + R x,  C = A^T kappa;
  4. grad' = M^T grad_x,  d' = |M|^T C + |M|^T |R| |M| 1;
  5. p' = -grad'/d' (zero where d' = 0), p = M p', q = A p;
  6. step length alpha: 1 (classic SPS) or the safeguarded line search below;
  7. x += alpha p, l += alpha q.
With M = I this is the paper's plain SPS update (Eq. 7): the surrogate
gradient at x^n equals the true gradient, the curvature is A^T D{gamma} c
plus the penalty's separable bound |R| 1.  ``gamma~ = A |M| 1`` generalises
gamma = A 1 (Eq. 9) to the signed operator A M.

Line search (not in the paper; the step direction is the SPS step):
evaluate phi(alpha) = Phi(x + alpha p), phi', phi'' starting from the step
length accepted in the previous iteration (1 at the first), and take Newton
steps alpha_{k+1} = alpha_k - phi'/phi'' kept inside [alpha_k/8, 8 alpha_k]
and below alpha_max (alpha kept when phi'' <= 0, divided by 8 when phi is not
finite or z = Q(l + alpha q) leaves z >= z_min there) for ``n_ls``
evaluations in total; accept the last evaluated alpha if phi there does not
exceed phi(0), else halve it up to ``n_halve`` times, else use alpha = 0 (the
next iteration then starts below the last halving).  Only comparisons
against phi(0) decide, never near-equal values of phi at two nearby alphas.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import model
from .penalty import NoPenalty, Penalty


@dataclasses.dataclass
class LineSearch:
    n_ls: int = 3
    n_halve: int = 8
    alpha_max: float = 1e12
    trust: float = 8.0
    z_min: float = -20.0
    warm: bool = True


class Setup:
    """Everything one reconstruction needs: projector (A, or identity for
    projection-domain decomposition), spectral model Q, S, data y, penalty."""

    def __init__(self, proj, Q, S, y, beta=None, blur=None, noise=None):
        self.proj = proj
        self.blur = blur              # optional detector blur B (model.Blur)
        self.noise = noise            # optional correlated noise (model.RowCorrelation)
        self.Q = np.asarray(Q, dtype=np.float64)
        self.S = np.asarray(S, dtype=np.float64)
        self.y = np.asarray(y, dtype=np.float64).reshape(self.S.shape[0], -1)
        self.nm = self.Q.shape[1]
        self.shape = tuple(proj.image_shape)
        if beta is None or not np.any(beta):
            self.pen = NoPenalty()
        else:
            self.pen = Penalty(beta)

    def zeros(self):
        return np.zeros((self.nm,) + self.shape)

    def objective(self, x, l=None):
        if l is None:
            l = self.proj.project(x)
        return model.data_objective(self.Q, self.S, l, self.y, self.blur, self.noise) + self.pen.value(x)

    def gradient(self, x):
        l = self.proj.project(x)
        return (self.proj.backproject(model.data_grad_l(self.Q, self.S, l, self.y, self.blur, self.noise))
                + self.pen.apply(x))


def line_search(st: Setup, x, p, l, q, phi0: float, ls: LineSearch, a0: float = 1.0):
    """Returns (alpha, phi(alpha), next starting alpha)."""
    pen = st.pen
    Rx = pen.apply(x)
    Rp = pen.apply(p)
    R0 = 0.5 * float(np.sum(x * Rx))
    pRx = float(np.sum(p * Rx))
    pRp = float(np.sum(p * Rp))

    def phi(a):
        # points outside the domain z = Q (l + a q) >= z_min are rejected
        if np.min(st.Q @ (l + a * q)) < ls.z_min:
            return np.inf, np.nan, np.nan
        f, f1, f2 = model.line_terms(st.Q, st.S, l, q, st.y, a, st.blur, st.noise)
        return f + R0 + a * pRx + 0.5 * a * a * pRp, f1 + pRx + a * pRp, f2 + pRp

    a = a0
    for k in range(ls.n_ls):
        with np.errstate(over="ignore", invalid="ignore"):
            f, f1, f2 = phi(a)
        if k + 1 < ls.n_ls:
            if not (np.isfinite(f) and np.isfinite(f1) and np.isfinite(f2)):
                an = a / ls.trust
            elif f2 > 0:
                an = min(max(a - f1 / f2, a / ls.trust), a * ls.trust)
            else:
                an = a
            a = min(an, ls.alpha_max)
    if np.isfinite(f) and f <= phi0:
        return a, f, a
    cand = a
    for _ in range(ls.n_halve):
        a = 0.5 * a
        with np.errstate(over="ignore", invalid="ignore"):
            f = phi(a)[0]
        if np.isfinite(f) and f <= phi0:
            return a, f, a
    return 0.0, phi0, cand / 2.0 ** (ls.n_halve + 1)


def run(st: Setup, precond, n_iter: int, line_search_cfg: LineSearch | None = None,
        nonneg: bool = False, reproject_every: int = 10, x0=None, return_alphas: bool = False):
    """Run ``n_iter`` iterations; returns (x, objective history of length
    n_iter + 1)."""
    Q, S, y, A, B, N = st.Q, st.S, st.y, st.proj, st.blur, st.noise
    x = st.zeros() if x0 is None else np.array(x0, dtype=np.float64)
    l = A.project(x)
    absM1 = precond.absM(np.ones_like(x))
    gamma_m = A.project(absM1)
    dR = precond.absMT(st.pen.abs_apply(absM1))
    hist, alphas = [], []
    a_prev = 1.0
    for n in range(n_iter):
        if n > 0 and reproject_every and n % reproject_every == 0:
            l = A.project(x)
        phi0 = model.data_objective(Q, S, l, y, B, N) + st.pen.value(x)
        hist.append(phi0)
        g = model.data_grad_l(Q, S, l, y, B, N)
        kappa = model.curvature_numerator(Q, S, l, y, gamma_m, B, N)
        grad = A.backproject(g) + st.pen.apply(x)
        C = A.backproject(kappa)
        gp = precond.MT(grad)
        dp = precond.absMT(C) + dR
        pp = np.where(dp > 0, -gp / np.where(dp > 0, dp, 1.0), 0.0)
        p = precond.M(pp)
        q = A.project(p)
        if line_search_cfg is not None:
            alpha, _, a_next = line_search(st, x, p, l, q, phi0, line_search_cfg,
                                           a_prev if line_search_cfg.warm else 1.0)
            a_prev = a_next
        else:
            alpha = 1.0
        alphas.append(alpha)
        if nonneg:
            x = np.maximum(x + alpha * p, 0.0)
            l = A.project(x)
        else:
            x = x + alpha * p
            l = l + alpha * q
    l = A.project(x)
    hist.append(model.data_objective(Q, S, l, y, B, N) + st.pen.value(x))
    if return_alphas:
        return x, np.array(hist), np.array(alphas)
    return x, np.array(hist)
