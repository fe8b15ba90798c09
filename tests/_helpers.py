"""Shared helpers for the GPU parity tests (inputs come from ``synth``;
expected values from ``oracle``)."""
import math

import numpy as np

import synth
from synth import FAN2D, PAR2D, Geometry


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def to_dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device="cuda")


def to_host(t):
    return t.detach().double().cpu().numpy()


def small_geoms():
    """Several tiles' worth of rays with ragged sizes (non-multiples of the
    block sizes), parallel and fan."""
    return {
        "par2d_c1": synth.config1().geom,
        "par2d_ragged": Geometry(PAR2D, 37, 29, 1, 0.9, 1.1, 1.0, 31, 0.2, math.pi, 45, 1, 1.05, 1.0),
        "fan2d_ragged": Geometry(FAN2D, 50, 43, 1, 0.8, 0.7, 1.0, 47, 0.1, 2 * math.pi, 61, 1, 1.3, 1.0, 80.0, 170.0),
        "fan2d_c2_128": synth.config2(nx=128, n_views=180, n_u=222).geom,
    }


def phantom(geom, seed=0, nm=1):
    rng = np.random.default_rng(seed)
    out = []
    for m in range(nm):
        shapes = synth.random_ellipses(rng, 4, radius=0.4 * min(geom.nx * geom.dx, geom.ny * geom.dy),
                                       amin=0.05 * geom.nx * geom.dx, amax=0.15 * geom.nx * geom.dx,
                                       vmin=0.01, vmax=0.03)
        out.append(synth.render(geom, shapes, supersample=2) + 0.002 * rng.random(geom.image_shape))
    return np.stack(out)
