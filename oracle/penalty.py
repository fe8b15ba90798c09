"""Oracle quadratic roughness penalty R(x) = 1/2 x^T R x with R = beta (x) Gamma.

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.

Gamma is the first-order smoothness kernel of Eqs. 26 and 52: Gamma_jj = |N_j|,
Gamma_jj' = -1 for j' in N_j, with N_j the 4-neighbourhood (2-D) or
6-neighbourhood (3-D) of pixel j inside the grid (no wrap-around; edge pixels
have fewer neighbours).  beta is the symmetric n_mat x n_mat strength matrix
(a 1x1 matrix for standard CT).  The paper's summation form (Eq. 49) counts
every neighbour pair twice relative to its matrix form 1/2 x^T R x; the matrix
form is the one used here, i.e. 1/2 sum_{k,k'} beta_kk' sum_{unordered pairs}
(x_jk - x_j'k)(x_jk' - x_j'k').
"""
from __future__ import annotations

import numpy as np


def neighbour_count(shape) -> np.ndarray:
    """|N_j| for every pixel of a grid of the given shape."""
    cnt = np.zeros(shape)
    for ax in range(len(shape)):
        n = shape[ax]
        if n < 2:
            continue
        sl = [slice(None)] * len(shape)
        sl[ax] = slice(0, n - 1)
        cnt[tuple(sl)] += 1
        sl[ax] = slice(1, n)
        cnt[tuple(sl)] += 1
    return cnt


def neighbour_sum(v: np.ndarray) -> np.ndarray:
    """sum_{j' in N_j} v_j' for one image."""
    out = np.zeros_like(v)
    for ax in range(v.ndim):
        n = v.shape[ax]
        if n < 2:
            continue
        lo = [slice(None)] * v.ndim
        hi = [slice(None)] * v.ndim
        lo[ax] = slice(0, n - 1)
        hi[ax] = slice(1, n)
        out[tuple(lo)] += v[tuple(hi)]
        out[tuple(hi)] += v[tuple(lo)]
    return out


def gamma_apply(v: np.ndarray) -> np.ndarray:
    """(Gamma v)_j = |N_j| v_j - sum_{j' in N_j} v_j'."""
    return neighbour_count(v.shape) * v - neighbour_sum(v)


def gamma_abs_apply(v: np.ndarray) -> np.ndarray:
    """(|Gamma| v)_j = |N_j| v_j + sum_{j' in N_j} v_j'."""
    return neighbour_count(v.shape) * v + neighbour_sum(v)


class Penalty:
    """R = beta (x) Gamma over images x[n_mat][*shape]."""

    def __init__(self, beta):
        self.beta = np.atleast_2d(np.asarray(beta, dtype=np.float64))

    def apply(self, x: np.ndarray) -> np.ndarray:
        gx = np.stack([gamma_apply(x[k]) for k in range(x.shape[0])])
        return np.einsum("kl,l...->k...", self.beta, gx)

    def value(self, x: np.ndarray) -> float:
        return 0.5 * float(np.sum(x * self.apply(x)))

    def abs_apply(self, v: np.ndarray) -> np.ndarray:
        gv = np.stack([gamma_abs_apply(v[k]) for k in range(v.shape[0])])
        return np.einsum("kl,l...->k...", np.abs(self.beta), gv)


class NoPenalty:
    """R = 0 (projection-domain decomposition)."""

    def apply(self, x):
        return np.zeros_like(x)

    def value(self, x):
        return 0.0

    def abs_apply(self, v):
        return np.zeros_like(v)
