"""Oracle preconditioner construction (one time, before iteration 1).

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.

The Hessian at the solution is approximated with D estimated from the data
(Sec. II-C: "an effective approximation for D is available"):
* standard CT (one material, one energy): D = y / I0, the gain-corrected
  measurement (Sec. II-D), so D G Sigma^-1 G D = y^2 / max(y, 1);
* spectral data: D = exp(-Q l_w) from a per-ray water-only fit (Sec. II-E).
H v = A^T [F_i (A v)_i] + R v with the per-ray Fisher blocks F_i.
"""
from __future__ import annotations

import numpy as np

from . import model, precond
from .psps import Setup

KINDS = ("none", "fourier", "mod_fourier", "haar", "block", "block_fourier", "block_haar")


def t_hat(st: Setup) -> np.ndarray:
    if st.Q.shape == (1, 1) and st.S.shape == (1, 1):
        return st.y / st.S[0, 0]
    lw = model.water_fit(st.Q, st.S, st.y)
    return np.exp(-np.outer(st.Q[:, 0], lw))


def fisher(st: Setup) -> np.ndarray:
    return model.fisher_blocks(st.Q, st.S, st.y, t_hat(st))


def make_apply_H(st: Setup, F: np.ndarray):
    def apply_H(v):
        lv = st.proj.project(v)                        # [m, i]
        return st.proj.backproject(np.einsum("imn,ni->mi", F, lv)) + st.pen.apply(v)
    return apply_H


def m0_blocks(st: Setup, F: np.ndarray) -> np.ndarray:
    """Blocks of (F+R)1_k (Eqs. 42, 54): column k of every per-pixel block is
    the response to the all-ones image of material k."""
    nm = st.nm
    apply_H = make_apply_H(st, F)
    H = np.zeros((int(np.prod(st.shape)), nm, nm))
    for k in range(nm):
        one = np.zeros((nm,) + st.shape)
        one[k] = 1.0
        r = apply_H(one).reshape(nm, -1)
        H[:, :, k] = r.T
    return precond.inv_sqrt_blocks(H, floor="block", zero_rule=True)


def build(st: Setup, kind: str, sides: int | None = None):
    """The preconditioner of one kind; sides: where M0 enters the Fourier and
    wavelet kinds (1: M = M0^T C; 2: the literal M0^T C M0 of Eqs. 33, 34, 57,
    61); None: each kind's default (2 for the one-material kinds, 1 for the
    cross-material ones; see ``precond``)."""
    if sides is None:
        sides = 1 if kind in ("block_fourier", "block_haar") else 2
    if kind == "none":
        return precond.Identity()
    F = fisher(st)
    apply_H = make_apply_H(st, F)
    if kind == "fourier":
        return precond.Fourier(precond.fourier_eigenvalues(apply_H, st.shape))
    B = m0_blocks(st, F)
    M0 = precond.Block(B, st.shape)
    if kind == "block":
        return M0
    if st.nm == 1:
        m0 = B[:, 0, 0].reshape(st.shape)

        def apply_N(v):
            return m0[None] * apply_H(m0[None] * v)
        if kind == "mod_fourier":
            return precond.Fourier(precond.fourier_eigenvalues(apply_N, st.shape), m0, sides)
        if kind == "haar":
            return precond.Haar(precond.haar_eigenvalues(apply_N, st.shape), m0, sides)
    if kind == "block_fourier":
        L = precond.cross_fourier_blocks(apply_H, M0, st.shape, st.nm)
        return precond.CrossFourier(L, M0, sides)
    if kind == "block_haar":
        K = precond.cross_haar_blocks(apply_H, M0, st.shape, st.nm)
        return precond.CrossHaar(K, M0, sides)
    raise ValueError(kind)
