"""Pins for the oracle Joseph projector (CPU).

The projector is not in the paper; its definition (Joseph's method on a
pixel-centred grid, parallel / fan-curved / cone-flat rays) is checked here
against things that do not depend on it: the adjoint identity, exactness on
linear images (the midpoint rule along the driving axis and linear
interpolation across it are both exact there), axis-aligned constant images,
and closed-form chord lengths through off-centre disks and spheres, with the
ray geometry restated from its convention, not taken from the projector.
"""
import math

import numpy as np
import pytest

import synth
from synth import CONE3D, FAN2D, PAR2D, Geometry


def spec_rays(g: Geometry):
    """Ray origins/directions restated from the convention in ``synth``."""
    return g.rays()


def geoms():
    return {
        "par2d": Geometry(PAR2D, 16, 12, 1, 1.0, 0.8, 1.0, 23, 0.1, math.pi, 29, 1, 0.9, 1.0),
        "fan2d": Geometry(FAN2D, 14, 18, 1, 0.7, 0.6, 1.0, 19, 0.2, 2 * math.pi, 31, 1, 1.1, 1.0, 40.0, 90.0),
        "cone3d": Geometry(CONE3D, 9, 8, 7, 0.9, 0.8, 0.7, 11, 0.3, 2 * math.pi, 13, 9, 1.3, 1.1, 30.0, 70.0),
    }


@pytest.mark.parametrize("name", ["par2d", "fan2d", "cone3d"])
def test_adjoint_identity(oracle_lib, name):
    g = geoms()[name]
    A = oracle_lib.Projector(g)
    rng = np.random.default_rng(1)
    x = rng.standard_normal((1,) + g.image_shape)
    y = rng.standard_normal((1, g.n_rays))
    lhs = float(np.sum(A.project(x) * y))
    rhs = float(np.sum(x * A.backproject(y)))
    scale = np.linalg.norm(A.project(x)) * np.linalg.norm(y)
    assert abs(lhs - rhs) <= 1e-12 * scale


def test_dense_columns_equal_rows(oracle_lib):
    """The matrix assembled column by column (projecting pixel impulses) equals
    the one assembled row by row (backprojecting ray impulses), transposed."""
    g = Geometry(FAN2D, 6, 5, 1, 1.0, 1.2, 1.0, 7, 0.0, 2 * math.pi, 9, 1, 1.0, 1.0, 20.0, 45.0)
    A = oracle_lib.Projector(g)
    cols = np.stack([A.project(np.eye(g.n_pix)[j].reshape(1, 5, 6))[0] for j in range(g.n_pix)], 1)
    rows = np.stack([A.backproject(np.eye(g.n_rays)[i][None])[0].ravel() for i in range(g.n_rays)], 0)
    assert np.array_equal(cols, rows)
    assert (cols >= 0).all() and cols.sum() > 0


def _linear_image(g, coef):
    zc = (np.arange(g.nz) - (g.nz - 1) / 2) * g.dz
    yc = (np.arange(g.ny) - (g.ny - 1) / 2) * g.dy
    xc = (np.arange(g.nx) - (g.nx - 1) / 2) * g.dx
    if g.kind == CONE3D:
        Z, Y, X = np.meshgrid(zc, yc, xc, indexing="ij")
        return coef[0] + coef[1] * X + coef[2] * Y + coef[3] * Z
    Y, X = np.meshgrid(yc, xc, indexing="ij")
    return coef[0] + coef[1] * X + coef[2] * Y


@pytest.mark.parametrize("name", ["par_tall", "par_wide", "fan_tall", "cone"])
def test_linear_image_exact(oracle_lib, name):
    """For rays whose every interpolation stays inside the grid, Joseph's sum
    of a linear image equals the exact line integral over the slab spanned by
    the driving axis: length/|u_axis| times the value at the slab centre."""
    if name == "par_tall":
        g = Geometry(PAR2D, 10, 60, 1, 1.0, 0.7, 1.0, 9, -0.3, 0.6, 41, 1, 0.8, 1.0)
    elif name == "par_wide":
        g = Geometry(PAR2D, 60, 10, 1, 0.7, 1.0, 1.0, 9, math.pi / 2 - 0.3, 0.6, 41, 1, 0.8, 1.0)
    elif name == "fan_tall":
        g = Geometry(FAN2D, 10, 70, 1, 1.0, 0.9, 1.0, 7, -0.2, 0.4, 31, 1, 1.0, 1.0, 80.0, 160.0)
    else:
        g = Geometry(CONE3D, 8, 30, 30, 1.0, 0.8, 0.7, 5, -0.2, 0.4, 15, 11, 0.8, 0.8, 60.0, 120.0)
    coef = (0.3, 0.05, -0.02, 0.04)
    img = _linear_image(g, coef)
    A = oracle_lib.Projector(g)
    got = A.project(img[None])[0]
    o, u = spec_rays(g)
    dims = 3 if g.kind == CONE3D else 2
    n = [g.nx, g.ny, g.nz][:dims]
    d = [g.dx, g.dy, g.dz][:dims]
    checked = 0
    for r in range(g.n_rays):
        a = int(np.argmax(np.abs(u[r])))
        xa = (np.arange(n[a]) - (n[a] - 1) / 2) * d[a]
        t = (xa - o[r, a]) / u[r, a]
        ok = True
        for b in range(dims):
            if b == a:
                continue
            fb = (o[r, b] + t * u[r, b]) / d[b] + (n[b] - 1) / 2
            ok &= bool(np.all((fb >= 0) & (fb <= n[b] - 1)))
        if not ok:
            continue
        tm = (0.0 - o[r, a]) / u[r, a]
        pm = o[r] + tm * u[r]
        fm = coef[0] + sum(coef[1 + k] * pm[k] for k in range(dims))
        want = n[a] * d[a] / abs(u[r, a]) * fm
        assert abs(got[r] - want) <= 1e-12 * max(1.0, abs(want)), (r, got[r], want)
        checked += 1
    assert checked >= 20


def test_axis_aligned_constant(oracle_lib):
    g = Geometry(PAR2D, 13, 11, 1, 0.9, 1.0, 1.0, 1, 0.0, math.pi, 9, 1, 1.0, 1.0)
    A = oracle_lib.Projector(g)
    got = A.project(np.full((1, 11, 13), 2.5))[0]
    # rays along -x at y = t_b; all 9 bins lie inside the 11 row centres
    assert np.allclose(got, 13 * 0.9 * 2.5, rtol=0, atol=1e-12)


@pytest.mark.parametrize("kind", [PAR2D, FAN2D])
def test_disk_chords(oracle_lib, kind):
    """Closed-form chords 2 sqrt(r^2 - d^2) through an off-centre uniform disk,
    d the distance of the disk centre from the ray line (restated geometry)."""
    if kind == PAR2D:
        g = Geometry(PAR2D, 96, 96, 1, 0.5, 0.5, 1.0, 24, 0.05, math.pi, 120, 1, 0.5, 1.0)
    else:
        g = Geometry(FAN2D, 96, 96, 1, 0.5, 0.5, 1.0, 24, 0.05, 2 * math.pi, 120, 1, 0.9, 1.0, 100.0, 200.0)
    c = np.array([6.3, -4.1])
    rad = 12.0
    disk = synth.Ellipse(c[0], c[1], rad, rad, 0.0, 1.0)
    img = synth.render(g, [disk], supersample=16)
    A = oracle_lib.Projector(g)
    got = A.project(img[None])[0]
    o, u = spec_rays(g)
    dist = np.abs((c[0] - o[:, 0]) * u[:, 1] - (c[1] - o[:, 1]) * u[:, 0])
    want = 2 * np.sqrt(np.clip(rad * rad - dist * dist, 0, None))
    inner = dist < rad - 1.5
    outer = dist > rad + 1.5
    assert inner.sum() > 100
    rel = np.abs(got[inner] - want[inner]) / want[inner]
    assert rel.max() < 0.02, rel.max()
    assert np.sqrt(np.mean((got[inner] - want[inner]) ** 2)) < 0.003 * 2 * rad
    assert np.abs(got[outer]).max() < 1e-12


def test_sphere_chords_cone(oracle_lib):
    g = Geometry(CONE3D, 40, 40, 40, 0.5, 0.5, 0.5, 6, 0.2, 2 * math.pi, 36, 36, 0.8, 0.8, 60.0, 120.0)
    c = np.array([1.7, -2.2, 1.1])
    rad = 6.0
    ball = synth.Ellipsoid(c[0], c[1], c[2], rad, rad, rad, 0.0, 1.0)
    img = synth.render(g, [ball], supersample=6)
    A = oracle_lib.Projector(g)
    got = A.project(img[None])[0]
    o, u = spec_rays(g)
    w = c[None, :] - o
    dist = np.linalg.norm(w - np.sum(w * u, 1, keepdims=True) * u, axis=1)
    want = 2 * np.sqrt(np.clip(rad * rad - dist * dist, 0, None))
    inner = dist < rad - 1.0
    assert inner.sum() > 100
    err = np.abs(got[inner] - want[inner])
    # partial-volume discretisation: at most about half a voxel of path length
    assert err.max() < 0.5 * g.dx, err.max()
    assert np.sqrt(np.mean(err ** 2)) < 0.01 * 2 * rad
    assert np.abs(got[dist > rad + 1.0]).max() < 1e-12


def test_project_rays_matches_full(oracle_lib):
    g = geoms()["fan2d"]
    A = oracle_lib.Projector(g)
    x = np.random.default_rng(3).random(g.image_shape)
    full = A.project(x[None])[0]
    rays = np.array([0, 5, 77, g.n_rays - 1])
    assert np.array_equal(A.project_rays(x, rays), full[rays])
