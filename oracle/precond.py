"""Oracle preconditioners x = M x' (Sec. II-C to II-E): builds and applies.

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.

Every preconditioner offers M v, M^T v and the elementwise-absolute |M| v,
|M|^T v on arrays v[n_mat][*shape].  |M| (any elementwise upper bound of the
absolute entries of M) is what makes the separable SPS curvature valid for a
signed operator A M: d' = |M|^T A^T(gamma~ c) + |M|^T |R| |M| 1 with
gamma~ = A |M| 1.

Readings of the paper used here:
* Eigenvalue estimate (Eq. 18): Lambda~ = D{U dx}^-1 D{U H dx}, evaluated as
  written: the ratio of the two transforms.  For a shift-variant H the
  phase-corrected Fourier ratio is complex and its real part goes negative at
  some frequencies (a Joseph impulse response is not point-symmetric), which
  the -1/2 power cannot take; the modulus |Lambda~| is used instead, and for
  N_k x N_k blocks its matrix analogue, the Hermitian polar factor
  (L^H L)^1/2, of which the real part is kept.  Both equal Lambda exactly when
  H is circulant.
* Haar test functions: Eq. 18 with the single test function U^T 1 (the
  paper's choice) lets every coefficient's response overlap with all others;
  on CT Hessians that gives estimates from -4x to 6x the true diagonal
  u_k^T H u_k.  The same estimator is therefore applied with a family of test
  functions U^T xi, each xi the indicator of one subband of one level
  restricted to one class of a P x P lattice of positions (P = 3), so that the
  coefficients excited together are well separated; the union covers every
  coefficient once.  ``lattice=0`` selects the paper's single U^T 1.
* Fourier: periodic unitary 2-D DFT per material on the image grid (no
  padding); the test impulse sits at the centre pixel (ny//2, nx//2).
* Eigenvalues are clamped to >= 1e-6 x the largest before the -1/2 power.
* Where M0 goes (Eqs. 33, 34, 57, 61).  The paper writes M = M0^T U^H
  Lambda~^-1/2 U M0 with Lambda~ the spectrum of N = M0^T H M0.  Then
  M^T H M = M0^T C N C M0 = M0^T M0 when N is diagonal in U (C = U^H
  Lambda~^-1/2 U), not the I that Sec. II-C sets as the goal.  For a scalar
  M0 (one material) that remainder is diagonal and the separable SPS
  curvature absorbs it, so the literal form is kept there (``sides=2``, the
  default of Fourier and Haar).  For per-pixel N_k x N_k blocks the
  remainder M0^T M0 couples the materials of a pixel, which a separable
  surrogate cannot absorb (the literal cross-material Fourier PSPS does not
  converge on the 3-material slice); there the one-sided M = M0^T C is used
  (``sides=1``, the default of CrossFourier and CrossHaar), for which
  M^T H M = C N C = I and M M^T = M0^T N^-1 M0 = H^-1 in that case.
* M0 = D{(F+R)1}^-1/2 (Eq. 30) or, with several materials, the per-pixel /
  per-ray N_k x N_k blocks of (F+R)1_k (Eqs. 42, 53-54) raised to -1/2; a
  block's eigenvalues are clamped to >= 1e-6 x its largest one, and pixels
  whose block trace is <= 1e-12 x the largest trace get M0 = 0 (outside the
  field of view).
"""
from __future__ import annotations

import numpy as np

from . import haar

EIG_FLOOR = 1e-6
ZERO_FLOOR = 1e-12


def inv_sqrt_blocks(H: np.ndarray, floor: str = "block", zero_rule: bool = True) -> np.ndarray:
    """Symmetric inverse square root of every N_k x N_k block in H[n, k, k]
    (symmetrised first).  floor='block' clamps each block's eigenvalues to
    >= EIG_FLOOR x its own largest; floor='global' to EIG_FLOOR x the largest
    over all blocks."""
    H = 0.5 * (H + np.swapaxes(H, -1, -2))
    lam, V = np.linalg.eigh(H)
    lmax = lam.max(axis=-1, keepdims=True)
    if floor == "global":
        lo = EIG_FLOOR * lam.max()
    else:
        lo = EIG_FLOOR * lmax
    lam_c = np.maximum(lam, lo)
    out = np.einsum("nij,nj,nkj->nik", V, 1.0 / np.sqrt(np.maximum(lam_c, 1e-300)), V)
    if zero_rule:
        tr = np.trace(H, axis1=-2, axis2=-1)
        dead = tr <= ZERO_FLOOR * tr.max()
        out[dead] = 0.0
    return out


# ---------------------------------------------------------------------------
# block-diagonal M0 (per pixel / per ray)
# ---------------------------------------------------------------------------

class Block:
    """M = blockdiag(M0_j); blocks B[n_pix, m, m] act on v[m][*shape]."""

    def __init__(self, B: np.ndarray, shape):
        self.B = np.asarray(B, dtype=np.float64)
        self.shape = tuple(shape)
        self.nm = self.B.shape[-1]

    def _mul(self, B, v):
        vf = v.reshape(self.nm, -1)
        return np.einsum("nij,jn->in", B, vf).reshape((self.nm,) + self.shape)

    def M(self, v):
        return self._mul(self.B, v)

    def MT(self, v):
        return self._mul(np.swapaxes(self.B, 1, 2), v)

    def absM(self, v):
        return self._mul(np.abs(self.B), v)

    def absMT(self, v):
        return self._mul(np.swapaxes(np.abs(self.B), 1, 2), v)


class Identity:
    def M(self, v):
        return v.copy()

    MT = absM = absMT = M


# ---------------------------------------------------------------------------
# Fourier family
# ---------------------------------------------------------------------------

def centre_index(shape):
    return tuple(n // 2 for n in shape)


def fourier_eigenvalues(apply_H, shape, k: int = 0, nm: int = 1) -> np.ndarray:
    """Lambda~ of Eq. 18 (as Eq. 28 / 32) for one material: |DFT(H delta_j) / DFT(delta_j)|
    with delta_j the unit impulse at the centre pixel."""
    d = np.zeros((nm,) + tuple(shape))
    d[(k,) + centre_index(shape)] = 1.0
    r = apply_H(d)
    lam = np.fft.fftn(r[k]) / np.fft.fftn(d[k])
    return np.abs(lam)


def clamp_eigs(lam: np.ndarray) -> np.ndarray:
    return np.maximum(lam, EIG_FLOOR * lam.max())


class Fourier:
    """M = m0 C m0 with C = U^H diag(lam^-1/2) U (Eq. 29 with m0 = 1, Eq. 33
    with the zero-frequency normalisation m0 = M0 of Eq. 30; sides=1: the
    one-sided m0 C).  One material.  |M| = m0 |C| m0 (m0 |C|) with |C| the
    circulant of the absolute kernel |IDFT(lam^-1/2)|."""

    def __init__(self, lam: np.ndarray, m0: np.ndarray | None = None, sides: int = 2):
        self.s = 1.0 / np.sqrt(clamp_eigs(lam))
        self.shape = lam.shape
        self.m0 = np.ones(self.shape) if m0 is None else np.asarray(m0, dtype=np.float64).reshape(self.shape)
        self.sides = sides
        kern = np.fft.ifftn(self.s).real
        self.s_abs = np.fft.fftn(np.abs(kern)).real

    def _filt(self, spec, v, transpose):
        pre = self.m0 if (self.sides == 2 or transpose) else 1.0
        post = self.m0 if (self.sides == 2 or not transpose) else 1.0
        out = np.empty_like(v, dtype=np.float64)
        for k in range(v.shape[0]):
            out[k] = post * np.fft.ifftn(spec * np.fft.fftn(pre * v[k])).real
        return out

    def M(self, v):
        return self._filt(self.s, v, False)

    def MT(self, v):
        return self._filt(self.s, v, True)

    def absM(self, v):
        return self._filt(self.s_abs, v, False)

    def absMT(self, v):
        return self._filt(self.s_abs, v, True)


class CrossFourier:
    """Cross-material Fourier preconditioner (Eq. 57): M = M0 C with
    C = U^H L^-1/2 U, L block diagonal over spatial frequencies (one N_k x N_k
    block per frequency), M0 the per-pixel blocks; sides=2: the literal
    M0^T C M0."""

    def __init__(self, L: np.ndarray, M0: Block, sides: int = 1):
        self.sides = sides
        # L[f..., k', k] real symmetric blocks
        self.shape = L.shape[:-2]
        nm = L.shape[-1]
        L = polar_real(L) if np.iscomplexobj(L) else L
        flat = L.reshape(-1, nm, nm)
        Li = inv_sqrt_blocks(flat, floor="global", zero_rule=False)
        self.Li = Li.reshape(L.shape)
        kern = np.fft.ifftn(self.Li, axes=tuple(range(len(self.shape)))).real
        self.Li_abs = np.fft.fftn(np.abs(kern), axes=tuple(range(len(self.shape)))).real
        self.M0 = M0

    def _mid(self, W, v):
        ax = tuple(range(1, v.ndim))
        V = np.fft.fftn(v, axes=ax)
        out = np.einsum("...ij,j...->i...", W, V)
        return np.fft.ifftn(out, axes=ax).real

    def M(self, v):
        inner = self.M0.M(v) if self.sides == 2 else v
        return self.M0.MT(self._mid(self.Li, inner))

    def MT(self, v):
        out = self._mid(np.swapaxes(self.Li, -1, -2), self.M0.M(v))
        return self.M0.MT(out) if self.sides == 2 else out

    def absM(self, v):
        inner = self.M0.absM(v) if self.sides == 2 else v
        return self.M0.absMT(self._mid(self.Li_abs, inner))

    def absMT(self, v):
        out = self._mid(np.swapaxes(self.Li_abs, -1, -2), self.M0.absM(v))
        return self.M0.absMT(out) if self.sides == 2 else out


def cross_fourier_blocks(apply_H, M0: Block, shape, nm: int) -> np.ndarray:
    """L_k of Eq. 56 for every material k: DFT of the zero-frequency-
    normalised response M0^T H M0 delta_jk divided by DFT(delta_jk), stacked as
    L[f..., k', k] (complex; see ``polar_real``)."""
    L = np.zeros(tuple(shape) + (nm, nm), dtype=complex)
    ax = tuple(range(1, len(shape) + 1))
    for k in range(nm):
        d = np.zeros((nm,) + tuple(shape))
        d[(k,) + centre_index(shape)] = 1.0
        r = M0.MT(apply_H(M0.M(d)))
        den = np.fft.fftn(d[k])
        R = np.fft.fftn(r, axes=ax) / den[None]
        L[..., :, k] = np.moveaxis(R, 0, -1)
    return L


def polar_real(L: np.ndarray) -> np.ndarray:
    """Re((L^H L)^1/2), symmetrised, for every block L[..., k, k] (the block
    analogue of |lambda|)."""
    shp = L.shape
    flat = L.reshape(-1, shp[-1], shp[-1])
    G = np.einsum("nji,njk->nik", flat.conj(), flat)
    lam, V = np.linalg.eigh(G)
    P = np.einsum("nij,nj,nkj->nik", V, np.sqrt(np.maximum(lam, 0.0)), V.conj())
    P = P.real
    P = 0.5 * (P + np.swapaxes(P, -1, -2))
    return P.reshape(shp)


# ---------------------------------------------------------------------------
# Haar wavelet
# ---------------------------------------------------------------------------

class Haar:
    """M = M0 U_DWT^T Lambda~^-1/2 U_DWT M0 (Eq. 34; sides=1: the one-sided
    M0 U^T Lambda~^-1/2 U); |M| uses |U| and |M0|.  One material, 2-D images
    or 3-D volumes."""

    def __init__(self, lam: np.ndarray, m0: np.ndarray | None = None, sides: int = 2):
        self.s = 1.0 / np.sqrt(clamp_eigs(lam))
        self.shape = lam.shape
        self.m0 = np.ones(self.shape) if m0 is None else np.asarray(m0, dtype=np.float64).reshape(self.shape)
        self.sides = sides

    def _op(self, v, absolute, transpose):
        pre = self.m0 if (self.sides == 2 or transpose) else 1.0
        post = self.m0 if (self.sides == 2 or not transpose) else 1.0
        out = np.empty_like(v, dtype=np.float64)
        for k in range(v.shape[0]):
            c = haar.forward(pre * v[k], absolute)
            out[k] = post * haar.transpose(self.s * c, absolute)
        return out

    def M(self, v):
        return self._op(v, False, False)

    def MT(self, v):
        return self._op(v, False, True)

    def absM(self, v):
        return self._op(v, True, False)

    def absMT(self, v):
        return self._op(v, True, True)


class CrossHaar:
    """Cross-material wavelet preconditioner (Eq. 61):
    M = M0 U^T K^-1/2 U (sides=2: the literal M0^T U^T K^-1/2 U M0) with U the
    orthonormal Haar transform (2-D or 3-D) applied
    to every material and K block diagonal over the wavelet coefficients (one
    N_k x N_k block per coefficient).  The estimated blocks are not symmetric;
    as for the cross-material Fourier blocks, K^-1/2 is taken of the polar
    factor (K^T K)^1/2 with the eigenvalue floor 1e-6 of the largest over all
    blocks.  |M| = |M0|^T |U|^T |K^-1/2| |U| |M0| (R7: elementwise absolute
    values of the factors bound |M| elementwise)."""

    def __init__(self, K: np.ndarray, M0: Block, sides: int = 1):
        self.sides = sides
        self.shape = K.shape[:-2]
        nm = K.shape[-1]
        P = polar_real(K)
        self.Ki = inv_sqrt_blocks(P.reshape(-1, nm, nm), floor="global", zero_rule=False).reshape(K.shape)
        self.Ki_abs = np.abs(self.Ki)
        self.M0 = M0

    def _mid(self, W, v, absolute):
        c = np.stack([haar.forward(v[k], absolute) for k in range(v.shape[0])])
        out = np.einsum("...ij,j...->i...", W, c)
        return np.stack([haar.transpose(out[k], absolute) for k in range(v.shape[0])])

    def M(self, v):
        inner = self.M0.M(v) if self.sides == 2 else v
        return self.M0.MT(self._mid(self.Ki, inner, False))

    def MT(self, v):
        out = self._mid(np.swapaxes(self.Ki, -1, -2), self.M0.M(v), False)
        return self.M0.MT(out) if self.sides == 2 else out

    def absM(self, v):
        inner = self.M0.absM(v) if self.sides == 2 else v
        return self.M0.absMT(self._mid(self.Ki_abs, inner, True))

    def absMT(self, v):
        out = self._mid(np.swapaxes(self.Ki_abs, -1, -2), self.M0.absM(v), True)
        return self.M0.absMT(out) if self.sides == 2 else out


def cross_haar_blocks(apply_H, M0: Block, shape, nm: int, lattice: int = 3) -> np.ndarray:
    """K_k of Eqs. 59-60 for every material k, with the wavelet test
    functions of the Haar reading (``haar_test_sets``): for each coefficient
    set xi the test function dx = U^T xi placed in material k gives column k
    of the blocks of the coefficients j in the set,
    K[j][k', k] = [U M0^T H M0 dx_k]_{k'}(j) / [U dx](j).  Returned as
    K[h, w, k', k] (real, not symmetric in general)."""
    K = np.zeros(tuple(shape) + (nm, nm))
    for sel in haar_test_sets(shape, lattice):
        dx = haar.transpose(sel.astype(np.float64))
        den = haar.forward(dx)
        for k in range(nm):
            d = np.zeros((nm,) + tuple(shape))
            d[k] = dx
            r = M0.MT(apply_H(M0.M(d)))
            for kp in range(nm):
                K[..., kp, k][sel] = haar.forward(r[kp])[sel] / den[sel]
    return K


def haar_test_sets(shape, lattice: int = 3):
    """Coefficient sets (boolean masks in the Mallat layout) whose indicator
    xi gives one test function U^T xi: per level, per detail subband (HL top
    right, LH bottom left, HH bottom right) and per class (a, c) of the
    position within the subband modulo ``lattice``; the final LL block is one
    more set.  ``lattice=0`` returns the single all-ones set."""
    if lattice == 0:
        return [np.ones(shape, dtype=bool)]
    if len(shape) == 3:
        return _haar_test_sets3(shape, lattice)
    sets = []
    ii, jj = np.meshgrid(np.arange(shape[0]), np.arange(shape[1]), indexing="ij")
    lv = haar._levels(*shape)
    for h, w in lv:
        h2, w2 = h // 2, w // 2
        for (r0, c0) in ((0, w2), (h2, 0), (h2, w2)):
            inband = (ii >= r0) & (ii < r0 + h2) & (jj >= c0) & (jj < c0 + w2)
            for a in range(min(lattice, h2)):
                for c in range(min(lattice, w2)):
                    sel = inband & ((ii - r0) % lattice == a) & ((jj - c0) % lattice == c)
                    if sel.any():
                        sets.append(sel)
    h, w = lv[-1] if lv else shape
    sets.append((ii < h // 2 if lv else ii < h) & (jj < w // 2 if lv else jj < w))
    return sets


def _haar_test_sets3(shape, lattice: int):
    """3-D: per level, per detail octant (sz, sy, sx) != (0, 0, 0) and per
    class (a, b, c) of the position within the octant modulo ``lattice``,
    then the final low-pass block."""
    sets = []
    zz, yy, xx = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    lv = haar.levels3(*shape)
    for d, h, w in lv:
        d2, h2, w2 = d // 2, h // 2, w // 2
        for s in haar.OCTANTS[1:]:
            z0, y0, x0 = s[0] * d2, s[1] * h2, s[2] * w2
            inband = ((zz >= z0) & (zz < z0 + d2) & (yy >= y0) & (yy < y0 + h2) & (xx >= x0) & (xx < x0 + w2))
            for a in range(min(lattice, d2)):
                for b in range(min(lattice, h2)):
                    for c in range(min(lattice, w2)):
                        sel = (inband & ((zz - z0) % lattice == a) & ((yy - y0) % lattice == b)
                               & ((xx - x0) % lattice == c))
                        if sel.any():
                            sets.append(sel)
    d, h, w = (lv[-1][0] // 2, lv[-1][1] // 2, lv[-1][2] // 2) if lv else shape
    sets.append((zz < d) & (yy < h) & (xx < w))
    return sets


def haar_eigenvalues(apply_H, shape, lattice: int = 3, part=None) -> np.ndarray:
    """Eq. 18 with wavelet test functions dx = U^T xi (Sec. II-D-3):
    Lambda~_k = [U H dx]_k / [U dx]_k for the coefficients k that xi excites.
    part = (i, n): only every n-th test set from the i-th (the other
    coefficients stay 0), so that the sets can be split among processes; the
    n parts add up to the whole estimate."""
    lam = np.zeros(shape)
    sets = haar_test_sets(shape, lattice)
    if part is not None:
        sets = sets[part[0]::part[1]]
    for sel in sets:
        dx = haar.transpose(sel.astype(np.float64))
        r = haar.forward(apply_H(dx[None])[0])
        den = haar.forward(dx)
        lam[sel] = r[sel] / den[sel]
    return np.abs(lam)
