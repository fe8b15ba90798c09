"""Oracle orthonormal 2-D Haar transform (Mallat pyramid), its transpose and
the sign-free variant |U| used for the separable-curvature bound.

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.

Level step on the current low-pass block (top-left h x w corner, h and w
even): for every 2x2 group (a b / c d) the four outputs are
    LL = (a+b+c+d)/2,  HL = (a-b+c-d)/2,  LH = (a+b-c-d)/2,  HH = (a-b-c+d)/2
stored at (i, j), (i, j+w/2), (i+h/2, j), (i+h/2, j+w/2).  The pyramid recurses
on the LL block while both sides are even and > 1 (full depth, log2 N levels
for an N x N power-of-two image).  With ``absolute=True`` every tap is +1/2,
which is the elementwise absolute value of the transform matrix because every
pixel enters each Haar coefficient through exactly one product of taps.
"""
from __future__ import annotations

import numpy as np


def _levels(h: int, w: int):
    out = []
    while h >= 2 and w >= 2 and h % 2 == 0 and w % 2 == 0:
        out.append((h, w))
        h //= 2
        w //= 2
    return out


def forward(img: np.ndarray, absolute: bool = False) -> np.ndarray:
    """U img (or |U| img) for one 2-D image."""
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
