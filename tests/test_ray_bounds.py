"""The bounds on the rays of one view that reach one pixel / voxel, which set
the fixed-point scales of the tile transposes (2-D: floor(2 / delta) + 2;
3-D: the cube image bound of the cone plans), checked against brute-force
counts from the FP64 scan geometry on the test scans (CPU).

A ray reaches pixel (voxel) j when its Joseph sample on j's driving-axis
plane has j among its two (four) interpolation taps, i.e. the sample's
interpolated coordinates lie within one pixel of j's centre."""
import math

import numpy as np
import pytest

import synth
from _helpers import cone_geoms, small_geoms


def _bound_2d(g) -> int:
    pix = max(g.dx, g.dy)
    if g.kind == synth.PAR2D:
        delta = g.du / pix
    else:
        R = math.hypot((0.5 * g.nx + 1.0) * g.dx, (0.5 * g.ny + 1.0) * g.dy)
        delta = (g.sid - R) * (g.du / g.sdd) / pix
    return int(math.floor(2.0 / delta)) + 2


def _bound_3d(g) -> int:
    s = max(g.dx, g.dy, g.dz)
    R = math.hypot((0.5 * g.nx + 1.0) * g.dx, (0.5 * g.ny + 1.0) * g.dy)
    Z = (0.5 * g.nz + 1.0) * g.dz
    D = g.sid - R
    side = 2.0 * math.sqrt(2.0) * s
    Eu = g.sdd * (1.0 + R / D) * side / D
    Ev = g.sdd * (1.0 + Z / D) * side / D
    return int((math.floor(Eu / g.du) + 2.0) * (math.floor(Ev / g.dv) + 2.0))


def _count_2d(g) -> int:
    """Largest number of rays of one view reaching one pixel."""
    best = 0
    n = [g.nx, g.ny]
    d = [g.dx, g.dy]
    c = [0.5 * (g.nx - 1), 0.5 * (g.ny - 1)]
    bins = np.arange(g.n_u) - 0.5 * (g.n_u - 1)
    for v in range(g.n_views):
        a = g.angle0 + v * g.angle_span / g.n_views
        if g.kind == synth.PAR2D:
            t = bins * g.du
            p = np.stack([-math.sin(a) * t, math.cos(a) * t], 1)
            u = np.tile([-math.cos(a), -math.sin(a)], (g.n_u, 1))
        else:
            ga = bins * g.du / g.sdd
            p = np.tile([g.sid * math.cos(a), g.sid * math.sin(a)], (g.n_u, 1))
            u = np.stack([-np.cos(a - ga), -np.sin(a - ga)], 1)
        counts = np.zeros((g.ny, g.nx), dtype=np.int64)
        for ax in (0, 1):
            o = 1 - ax
            sel = (np.abs(u[:, ax]) >= np.abs(u[:, o])) if ax == 0 else (np.abs(u[:, 1]) > np.abs(u[:, 0]))
            if not sel.any():
                continue
            i = np.arange(n[ax])
            pa = (i - c[ax]) * d[ax]                                           # plane coordinates
            tt = (pa[None, :] - p[sel, ax][:, None]) / u[sel, ax][:, None]
            f = (p[sel, o][:, None] + tt * u[sel, o][:, None]) / d[o] + c[o]  # interpolated index
            lo = np.floor(f).astype(np.int64)
            for tap in (0, 1):
                j = lo + tap
                ok = (j >= 0) & (j < n[o])
                ii = np.broadcast_to(i[None, :], j.shape)[ok]
                jj = j[ok]
                pix = (ii * g.nx + jj) if ax == 1 else (jj * g.nx + ii)        # [y][x]
                counts += np.bincount(pix, minlength=g.nx * g.ny).reshape(g.ny, g.nx)
        best = max(best, int(counts.max()))
    return best


def _count_3d(g, views=None) -> int:
    """Largest number of rays of one view reaching one voxel (any driving
    axis), from the flat-detector cone geometry in FP64."""
    n = [g.nx, g.ny, g.nz]
    d = [g.dx, g.dy, g.dz]
    c = [0.5 * (g.nx - 1), 0.5 * (g.ny - 1), 0.5 * (g.nz - 1)]
    iu, iv = np.meshgrid(np.arange(g.n_u) - 0.5 * (g.n_u - 1), np.arange(g.n_v) - 0.5 * (g.n_v - 1))
    uu, vv = (iu * g.du).ravel(), (iv * g.dv).ravel()
    best = 0
    for v in (range(g.n_views) if views is None else views):
        a = g.angle0 + v * g.angle_span / g.n_views
        ca, sa = math.cos(a), math.sin(a)
        S = np.array([g.sid * ca, g.sid * sa, 0.0])
        # detector cell centres: S - sdd (cos a, sin a, 0) + u e_u + w e_v
        P = np.stack([S[0] - g.sdd * ca - uu * sa, S[1] - g.sdd * sa + uu * ca, vv], 1)
        u = P - S[None, :]
        au = np.abs(u)
        axis = np.where((au[:, 0] >= au[:, 1]) & (au[:, 0] >= au[:, 2]), 0, np.where(au[:, 1] >= au[:, 2], 1, 2))
        counts = np.zeros(g.nx * g.ny * g.nz, dtype=np.int64)
        for ax in range(3):
            sel = axis == ax
            if not sel.any():
                continue
            b = 1 if ax == 0 else 0
            cc = 1 if ax == 2 else 2
            i = np.arange(n[ax])
            pa = (i - c[ax]) * d[ax]
            tt = (pa[None, :] - S[ax]) / u[sel, ax][:, None]
            fb = (S[b] + tt * u[sel, b][:, None]) / d[b] + c[b]
            fc = (S[cc] + tt * u[sel, cc][:, None]) / d[cc] + c[cc]
            lb, lc = np.floor(fb).astype(np.int64), np.floor(fc).astype(np.int64)
            ii = np.broadcast_to(i[None, :], lb.shape)
            for tb in (0, 1):
                for tc in (0, 1):
                    jb, jc = lb + tb, lc + tc
                    ok = (jb >= 0) & (jb < n[b]) & (jc >= 0) & (jc < n[cc])
                    idx = [None, None, None]
                    idx[ax], idx[b], idx[cc] = ii[ok], jb[ok], jc[ok]
                    vox = (idx[2] * g.ny + idx[1]) * g.nx + idx[0]
                    counts += np.bincount(vox, minlength=counts.size)
        best = max(best, int(counts.max()))
    return best


@pytest.mark.parametrize("name", ["par2d_ragged", "fan2d_ragged", "fan2d_c2_128"])
def test_bound_2d_holds(name):
    g = small_geoms()[name]
    got, bound = _count_2d(g), _bound_2d(g)
    assert 1 <= got <= bound, (name, got, bound)


@pytest.mark.parametrize("name", ["cone_small", "cone_ragged", "c5_64"])
def test_bound_3d_holds(name):
    if name == "c5_64":
        g = synth.config5(n=64, n_views=90, n_u=128, n_v=96, rays=False).geom
        views = range(0, 90, 9)
    else:
        g = cone_geoms()[name]
        views = None
    got, bound = _count_3d(g, views), _bound_3d(g)
    assert 1 <= got <= bound, (name, got, bound)
    # not loose by more than the factors the derivation gives away (the cube's
    # diagonal, the magnification range, one extra cell per axis)
    assert bound <= 12 * got, (name, got, bound)
