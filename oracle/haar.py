"""Oracle orthonormal 2-D and 3-D Haar transforms (Mallat pyramid), their
transposes and the sign-free variant |U| used for the separable-curvature
bound.

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.

Level step on the current low-pass block (top-left h x w corner, h and w
even): for every 2x2 group (a b / c d) the four outputs are
    LL = (a+b+c+d)/2,  HL = (a-b+c-d)/2,  LH = (a+b-c-d)/2,  HH = (a-b-c+d)/2
stored at (i, j), (i, j+w/2), (i+h/2, j), (i+h/2, j+w/2).  The pyramid recurses
on the LL block while both sides are even and > 1 (full depth, log2 N levels
for an N x N power-of-two image).  With ``absolute=True`` every tap is +1/2,
which is the elementwise absolute value of the transform matrix because every
pixel enters each Haar coefficient through exactly one product of taps.

3-D volumes [z, y, x]: the level step takes every 2x2x2 group v[dz, dy, dx]
of the current low-pass block (d x h x w, all even) to the eight outputs
    c[sz, sy, sx] = 2^-3/2 sum_{dz,dy,dx} (-1)^(sz dz + sy dy + sx dx) v[dz, dy, dx]
stored in octant (sz, sy, sx) of the block, at (sz d/2 + i, sy h/2 + j,
sx w/2 + k) for the group (i, j, k); the pyramid recurses on octant (0, 0, 0)
while all three sides are even and > 1.  |U| uses +2^-3/2 for every tap.
The 8-point sign matrix is symmetric and orthogonal after the scaling, so the
transpose of one step applies the same sums to the octants' coefficients.
"""
from __future__ import annotations

import itertools

import numpy as np


def _levels(h: int, w: int):
    out = []
    while h >= 2 and w >= 2 and h % 2 == 0 and w % 2 == 0:
        out.append((h, w))
        h //= 2
        w //= 2
    return out


def forward(img: np.ndarray, absolute: bool = False) -> np.ndarray:
    """U img (or |U| img) for one 2-D image or 3-D volume."""
    if np.ndim(img) == 3:
        return _forward3(img, absolute)
    out = np.array(img, dtype=np.float64, copy=True)
    for h, w in _levels(*out.shape):
        blk = out[:h, :w].copy()
        a, b = blk[0::2, 0::2], blk[0::2, 1::2]
        c, d = blk[1::2, 0::2], blk[1::2, 1::2]
        h2, w2 = h // 2, w // 2
        if absolute:
            s = 0.5 * (a + b + c + d)
            out[:h2, :w2] = s
            out[:h2, w2:w] = s
            out[h2:h, :w2] = s
            out[h2:h, w2:w] = s
        else:
            out[:h2, :w2] = 0.5 * (a + b + c + d)
            out[:h2, w2:w] = 0.5 * (a - b + c - d)
            out[h2:h, :w2] = 0.5 * (a + b - c - d)
            out[h2:h, w2:w] = 0.5 * (a - b - c + d)
    return out


def transpose(coef: np.ndarray, absolute: bool = False) -> np.ndarray:
    """U^T coef (or |U|^T coef); U^T = U^-1 for the signed transform."""
    if np.ndim(coef) == 3:
        return _transpose3(coef, absolute)
    out = np.array(coef, dtype=np.float64, copy=True)
    for h, w in reversed(_levels(*out.shape)):
        h2, w2 = h // 2, w // 2
        LL = out[:h2, :w2].copy()
        HL = out[:h2, w2:w].copy()
        LH = out[h2:h, :w2].copy()
        HH = out[h2:h, w2:w].copy()
        if absolute:
            s = 0.5 * (LL + HL + LH + HH)
            a = b = c = d = s
        else:
            a = 0.5 * (LL + HL + LH + HH)
            b = 0.5 * (LL - HL + LH - HH)
            c = 0.5 * (LL + HL - LH - HH)
            d = 0.5 * (LL - HL - LH + HH)
        blk = np.empty((h, w))
        blk[0::2, 0::2] = a
        blk[0::2, 1::2] = b
        blk[1::2, 0::2] = c
        blk[1::2, 1::2] = d
        out[:h, :w] = blk
    return out


# ---------------------------------------------------------------------------
# 3-D
# ---------------------------------------------------------------------------

OCTANTS = tuple(itertools.product((0, 1), repeat=3))   # (sz, sy, sx) / (dz, dy, dx)


def levels3(d: int, h: int, w: int):
    out = []
    while min(d, h, w) >= 2 and d % 2 == 0 and h % 2 == 0 and w % 2 == 0:
        out.append((d, h, w))
        d //= 2
        h //= 2
        w //= 2
    return out


def _sign(s, t) -> float:
    return -1.0 if (s[0] * t[0] + s[1] * t[1] + s[2] * t[2]) % 2 else 1.0


def _octant(d2, h2, w2, s):
    return (slice(s[0] * d2, (s[0] + 1) * d2), slice(s[1] * h2, (s[1] + 1) * h2), slice(s[2] * w2, (s[2] + 1) * w2))


def _forward3(vol: np.ndarray, absolute: bool) -> np.ndarray:
    out = np.array(vol, dtype=np.float64, copy=True)
    r = 2.0 ** -1.5
    for d, h, w in levels3(*out.shape):
        blk = out[:d, :h, :w].copy()
        v = {t: blk[t[0]::2, t[1]::2, t[2]::2] for t in OCTANTS}
        for s in OCTANTS:
            acc = np.zeros((d // 2, h // 2, w // 2))
            for t in OCTANTS:
                acc += (1.0 if absolute else _sign(s, t)) * v[t]
            out[_octant(d // 2, h // 2, w // 2, s)] = r * acc
    return out


def _transpose3(coef: np.ndarray, absolute: bool) -> np.ndarray:
    out = np.array(coef, dtype=np.float64, copy=True)
    r = 2.0 ** -1.5
    for d, h, w in reversed(levels3(*out.shape)):
        c = {s: out[_octant(d // 2, h // 2, w // 2, s)].copy() for s in OCTANTS}
        blk = np.empty((d, h, w))
        for t in OCTANTS:
            acc = np.zeros((d // 2, h // 2, w // 2))
            for s in OCTANTS:
                acc += (1.0 if absolute else _sign(s, t)) * c[s]
            blk[t[0]::2, t[1]::2, t[2]::2] = r * acc
        out[:d, :h, :w] = blk
    return out
