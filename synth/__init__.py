"""Seeded synthetic inputs shared by the FP64 oracle, the CUDA path, the tests
and the benchmark.

This module only *generates inputs*: scan geometries, ellipse/ellipsoid
phantoms, analytic (exact) line integrals of those phantoms, x-ray spectra,
basis-material attenuation tables and Poisson counts.  It holds none of the
reconstruction method's arithmetic (no Joseph projector, no SPS, no
preconditioner): the measurement is simulated from analytic chord lengths so
that neither implementation under test is used to make its own data.

Conventions (shared by every consumer):

* image pixel (ix, iy[, iz]) has its centre at ((ix-(nx-1)/2)*dx, ...), arrays
  are row-major ``[iz][iy][ix]``; several materials are stacked as ``[m][...]``;
* 2-D sinograms are ``[view][bin]``, 3-D ones ``[view][row][col]``;
* parallel beam: view angle th, ray direction -(cos th, sin th), bin b crosses
  the centre line at offset t_b = (b-(n_u-1)/2)*du along (-sin th, cos th);
* fan beam, curved detector: source at sid*(cos be, sin be), bin b has fan
  angle ga_b = (b-(n_u-1)/2)*du/sdd and direction -(cos(be-ga), sin(be-ga)),
  so that small positive ga passes the centre at positive offset along
  (-sin be, cos be), like the parallel beam;
* cone beam, flat detector: source at (sid cos be, sid sin be, 0), detector
  plane at distance sdd with axes e_u=(-sin be, cos be, 0), e_v=(0,0,1), pixel
  (iu, iv) at offsets ((iu-(n_u-1)/2)*du, (iv-(n_v-1)/2)*dv).

Seeds: ``numpy.random.SeedSequence(20101371, spawn_key=(config, purpose))``.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence

import numpy as np

ROOT_SEED = 20101371
PURPOSES = {"phantom": 0, "materials": 1, "noise": 2, "slices": 3, "misc": 4}

PAR2D, FAN2D, CONE3D = 0, 1, 2


def rng(config: int, purpose: str) -> np.random.Generator:
    ss = np.random.SeedSequence(ROOT_SEED, spawn_key=(int(config), PURPOSES[purpose]))
    return np.random.Generator(np.random.PCG64(ss))


@dataclasses.dataclass
class Geometry:
    """Scan geometry; field names and meaning mirror ``mbir_geometry`` in
    ``include/mbir.h``.  Lengths in mm, angles in radians."""
    kind: int
    nx: int
    ny: int
    nz: int = 1
    dx: float = 1.0
    dy: float = 1.0
    dz: float = 1.0
    n_views: int = 1
    angle0: float = 0.0
    angle_span: float = math.pi
    n_u: int = 1
    n_v: int = 1
    du: float = 1.0
    dv: float = 1.0
    sid: float = 0.0
    sdd: float = 0.0

    @property
    def image_shape(self):
        return (self.ny, self.nx) if self.kind != CONE3D else (self.nz, self.ny, self.nx)

    @property
    def sino_shape(self):
        return (self.n_views, self.n_u) if self.kind != CONE3D else (self.n_views, self.n_v, self.n_u)

    @property
    def n_pix(self) -> int:
        return int(np.prod(self.image_shape))

    @property
    def n_rays(self) -> int:
        return int(np.prod(self.sino_shape))

    def view_angles(self) -> np.ndarray:
        return self.angle0 + np.arange(self.n_views) * (self.angle_span / self.n_views)

    def rays(self):
        """(origins, unit directions) for every ray, shape [n_rays, 2|3], in
        sinogram order.  Used only to simulate data analytically."""
        ang = self.view_angles()
        if self.kind == PAR2D:
            t = (np.arange(self.n_u) - (self.n_u - 1) / 2.0) * self.du
            c, s = np.cos(ang)[:, None], np.sin(ang)[:, None]
            ox = -s * t[None, :]
            oy = c * t[None, :]
            o = np.stack([ox, oy], -1).reshape(-1, 2)
            d = np.stack([-c * np.ones_like(t), -s * np.ones_like(t)], -1).reshape(-1, 2)
            return o, d
        if self.kind == FAN2D:
            ga = (np.arange(self.n_u) - (self.n_u - 1) / 2.0) * self.du / self.sdd
            be = ang[:, None]
            ox = self.sid * np.cos(be) * np.ones_like(ga)
            oy = self.sid * np.sin(be) * np.ones_like(ga)
            dx_ = -np.cos(be - ga[None, :])
            dy_ = -np.sin(be - ga[None, :])
            return (np.stack([ox, oy], -1).reshape(-1, 2),
                    np.stack([dx_, dy_], -1).reshape(-1, 2))
        if self.kind == CONE3D:
            u = (np.arange(self.n_u) - (self.n_u - 1) / 2.0) * self.du
            v = (np.arange(self.n_v) - (self.n_v - 1) / 2.0) * self.dv
            be = ang[:, None, None]
            sx = self.sid * np.cos(be)
            sy = self.sid * np.sin(be)
            # detector point = s - sdd*e_r + u*e_u + v*e_z
            px = sx - self.sdd * np.cos(be) + u[None, None, :] * (-np.sin(be))
            py = sy - self.sdd * np.sin(be) + u[None, None, :] * np.cos(be)
            shape = (self.n_views, self.n_v, self.n_u)
            pz = np.broadcast_to(v[None, :, None], shape)
            px = np.broadcast_to(px, shape)
            py = np.broadcast_to(py, shape)
            pz = np.broadcast_to(pz, shape)
            ox = np.broadcast_to(sx, shape)
            oy = np.broadcast_to(sy, shape)
            oz = np.zeros(shape)
            d = np.stack([px - ox, py - oy, pz - oz], -1).reshape(-1, 3)
            d = d / np.linalg.norm(d, axis=1, keepdims=True)
            o = np.stack([ox, oy, oz], -1).reshape(-1, 3)
            return o, d
        raise ValueError(self.kind)


# ---------------------------------------------------------------------------
# phantoms
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Ellipse:
    cx: float
    cy: float
    a: float          # semi-axis along the rotated x axis (mm)
    b: float
    phi: float        # rotation (rad)
    value: float      # additive value inside (mu in 1/mm, or density)


@dataclasses.dataclass
class Ellipsoid:
    cx: float
    cy: float
    cz: float
    a: float
    b: float
    c: float
    phi: float        # rotation about z
    value: float


def _ellipse_inside(e: Ellipse, x, y):
    cp, sp = math.cos(e.phi), math.sin(e.phi)
    xr = (x - e.cx) * cp + (y - e.cy) * sp
    yr = -(x - e.cx) * sp + (y - e.cy) * cp
    return (xr / e.a) ** 2 + (yr / e.b) ** 2 <= 1.0


def _ellipsoid_inside(e: Ellipsoid, x, y, z):
    cp, sp = math.cos(e.phi), math.sin(e.phi)
    xr = (x - e.cx) * cp + (y - e.cy) * sp
    yr = -(x - e.cx) * sp + (y - e.cy) * cp
    zr = z - e.cz
    return (xr / e.a) ** 2 + (yr / e.b) ** 2 + (zr / e.c) ** 2 <= 1.0


def render(geom: Geometry, shapes: Sequence, supersample: int = 4) -> np.ndarray:
    """Pixel-average rendering of additive ellipses/ellipsoids (FP64)."""
    ss = supersample
    off = (np.arange(ss) + 0.5) / ss - 0.5
    if geom.kind != CONE3D:
        xc = (np.arange(geom.nx) - (geom.nx - 1) / 2.0) * geom.dx
        yc = (np.arange(geom.ny) - (geom.ny - 1) / 2.0) * geom.dy
        img = np.zeros((geom.ny, geom.nx))
        for oy in off:
            for ox in off:
                X = (xc + ox * geom.dx)[None, :]
                Y = (yc + oy * geom.dy)[:, None]
                for e in shapes:
                    img += e.value * _ellipse_inside(e, X, Y)
        return img / (ss * ss)
    xc = (np.arange(geom.nx) - (geom.nx - 1) / 2.0) * geom.dx
    yc = (np.arange(geom.ny) - (geom.ny - 1) / 2.0) * geom.dy
    zc = (np.arange(geom.nz) - (geom.nz - 1) / 2.0) * geom.dz
    img = np.zeros((geom.nz, geom.ny, geom.nx))
    for oz in off:
        for oy in off:
            for ox in off:
                X = (xc + ox * geom.dx)[None, None, :]
                Y = (yc + oy * geom.dy)[None, :, None]
                Z = (zc + oz * geom.dz)[:, None, None]
                for e in shapes:
                    img += e.value * _ellipsoid_inside(e, X, Y, Z)
    return img / ss ** 3


def chord_lengths(shapes: Sequence, origins: np.ndarray, dirs: np.ndarray) -> np.ndarray:
    """Exact line integrals sum_k value_k * |ray ∩ shape_k| over full lines."""
    out = np.zeros(origins.shape[0])
    for e in shapes:
        if isinstance(e, Ellipse):
            cp, sp = math.cos(e.phi), math.sin(e.phi)
            px = origins[:, 0] - e.cx
            py = origins[:, 1] - e.cy
            ox = (px * cp + py * sp) / e.a
            oy = (-px * sp + py * cp) / e.b
            ux = (dirs[:, 0] * cp + dirs[:, 1] * sp) / e.a
            uy = (-dirs[:, 0] * sp + dirs[:, 1] * cp) / e.b
            A = ux * ux + uy * uy
            B = 2 * (ox * ux + oy * uy)
            C = ox * ox + oy * oy - 1.0
        else:
            cp, sp = math.cos(e.phi), math.sin(e.phi)
            px = origins[:, 0] - e.cx
            py = origins[:, 1] - e.cy
            pz = origins[:, 2] - e.cz
            ox = (px * cp + py * sp) / e.a
            oy = (-px * sp + py * cp) / e.b
            oz = pz / e.c
            ux = (dirs[:, 0] * cp + dirs[:, 1] * sp) / e.a
            uy = (-dirs[:, 0] * sp + dirs[:, 1] * cp) / e.b
            uz = dirs[:, 2] / e.c
            A = ux * ux + uy * uy + uz * uz
            B = 2 * (ox * ux + oy * uy + oz * uz)
            C = ox * ox + oy * oy + oz * oz - 1.0
        disc = B * B - 4 * A * C
        ok = disc > 0
        L = np.zeros_like(disc)
        L[ok] = np.sqrt(disc[ok]) / A[ok]
        out += e.value * L
    return out


def random_ellipses(g: np.random.Generator, n: int, radius: float, amin: float, amax: float,
                    vmin: float, vmax: float, centre=(0.0, 0.0), max_tries: int = 10000) -> List[Ellipse]:
    """Non-overlapping ellipses (rejection on bounding circles) inside a disk."""
    out: List[Ellipse] = []
    tries = 0
    while len(out) < n and tries < max_tries:
        tries += 1
        a = g.uniform(amin, amax)
        b = g.uniform(amin, amax)
        r = max(a, b)
        if r >= radius:
            continue
        rho = (radius - r) * math.sqrt(g.uniform())
        th = g.uniform(0, 2 * math.pi)
        cx, cy = centre[0] + rho * math.cos(th), centre[1] + rho * math.sin(th)
        if any(math.hypot(cx - e.cx, cy - e.cy) < r + max(e.a, e.b) for e in out):
            continue
        out.append(Ellipse(cx, cy, a, b, g.uniform(0, math.pi), g.uniform(vmin, vmax)))
    return out


# ---------------------------------------------------------------------------
# spectra and materials (keV grid, 1 keV spacing)
# ---------------------------------------------------------------------------

def mu_al(E):
    """Aluminium-like attenuation (1/mm) used only to shape the spectra."""
    E = np.asarray(E, dtype=np.float64)
    return 0.27 * (E / 30.0) ** -3 + 0.035 * (E / 30.0) ** -0.3


def kramers(E, kvp: float, al_mm: float = 2.0):
    """Normalised filtered Kramers spectrum s(E) ∝ (kVp-E) exp(-mu_Al(E) al_mm)."""
    E = np.asarray(E, dtype=np.float64)
    s = np.clip(kvp - E, 0.0, None) * np.exp(-mu_al(E) * al_mm)
    return s / s.sum()


MATERIAL_RANGES = {
    "water": ((0.15, 0.25), (0.15, 0.20)),
    "bone": ((0.8, 1.2), (0.15, 0.25)),
    "iodine": ((8.0, 12.0), (0.2, 0.3)),
}


def material_Q(E, names: Sequence[str], g: np.random.Generator) -> np.ndarray:
    """Q[E][m] in 1/(mm*g/cm^3): 0.1*(a (E/30)^-3 + b (E/30)^-0.3), seeded a, b;
    the iodine-like material gets a 6x K-edge step for E >= 33.2 keV."""
    E = np.asarray(E, dtype=np.float64)
    Q = np.zeros((E.size, len(names)))
    for m, nm in enumerate(names):
        (alo, ahi), (blo, bhi) = MATERIAL_RANGES[nm]
        a, b = g.uniform(alo, ahi), g.uniform(blo, bhi)
        mu = a * (E / 30.0) ** -3 + b * (E / 30.0) ** -0.3
        if nm == "iodine":
            mu = np.where(E >= 33.2, 6.0 * mu, mu)
        Q[:, m] = 0.1 * mu
    return Q


def poisson(g: np.random.Generator, mean: np.ndarray) -> np.ndarray:
    return g.poisson(np.maximum(mean, 0.0)).astype(np.float64)


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Problem:
    """One reconstruction problem: geometry (None for projection-domain
    decomposition), spectral model, data and the penalty."""
    name: str
    geom: Geometry | None
    Q: np.ndarray            # [n_energy][n_mat]
    S: np.ndarray            # [n_chan][n_energy], photons (gain folded in)
    y: np.ndarray            # [n_chan][n_rays] counts
    beta: np.ndarray         # [n_mat][n_mat]
    truth: np.ndarray        # [n_mat][image...] (or [n_mat][n_rays])
    n_iter: int
    precond: str
    n_rays: int

    @property
    def n_mat(self):
        return self.Q.shape[1]


def mbir_problem(config: int, geom: Geometry, shapes, I0: float, beta: float, n_iter: int,
                 precond: str, name: str) -> Problem:
    o, d = geom.rays()
    lint = chord_lengths(shapes, o, d)
    y = poisson(rng(config, "noise"), I0 * np.exp(-lint))
    truth = render(geom, shapes, supersample=4)[None]
    return Problem(name, geom, np.ones((1, 1)), np.full((1, 1), float(I0)), y[None],
                   np.full((1, 1), float(beta)), truth, n_iter, precond, geom.n_rays)


def config1() -> Problem:
    """2-D parallel beam, 64x64 at 1 mm, 1-6 ellipses mu in [0.01, 0.03]/mm,
    90 views over 180 deg, 96 bins of 1 mm, I0=1e4, beta=1e3, 50 iterations."""
    g = rng(1, "phantom")
    geom = Geometry(PAR2D, 64, 64, 1, 1.0, 1.0, 1.0, 90, 0.0, math.pi, 96, 1, 1.0, 1.0)
    n = int(g.integers(1, 7))
    shapes = random_ellipses(g, n, radius=29.0, amin=3.0, amax=20.0, vmin=0.01, vmax=0.03)
    return mbir_problem(1, geom, shapes, 1e4, 1e3, 50, "fourier", "c1_par2d_64")


def water_phantom(g: np.random.Generator, scale: float) -> list:
    water = Ellipse(0.0, 0.0, 110.0 * scale, 90.0 * scale, 0.0, 0.02)
    inserts = random_ellipses(g, 6, radius=80.0 * scale, amin=4.0 * scale, amax=20.0 * scale,
                              vmin=-0.01, vmax=0.02)
    return [water] + inserts


def config2(nx: int = 512, n_views: int = 720, n_u: int = 888) -> Problem:
    """2-D fan beam, 512x512 at 0.5 mm, 720 views over 360 deg, 888 curved bins
    of 1 mm at SDD 1000, SID 500; water ellipse with inserts; I0=1e5;
    beta=1e4; 100 iterations; Haar preconditioner.  Smaller nx/n_views/n_u
    scale the same scan down (same field of view) for oracle-sized runs."""
    g = rng(2, "phantom")
    dx = 0.5 * 512 / nx
    geom = Geometry(FAN2D, nx, nx, 1, dx, dx, 1.0, n_views, 0.0, 2 * math.pi, n_u, 1,
                    1.0 * 888 / n_u, 1.0, 500.0, 1000.0)
    shapes = water_phantom(g, 1.0)
    return mbir_problem(2, geom, shapes, 1e5, 1e4, 100, "haar", f"c2_fan2d_{nx}")


def config3(n_views: int = 720, n_u: int = 888) -> Problem:
    """Projection-domain decomposition: 2 materials (water, bone), 80/140 kVp
    channels (each normalised to I0=1e5), iid line integrals water [0,300],
    bone [0,30] mm*g/cm^3, per-ray 2x2 block preconditioner, R = 0."""
    E = np.arange(20.0, 141.0)
    Q = material_Q(E, ["water", "bone"], rng(3, "materials"))
    I0 = 1e5
    S = np.stack([I0 * kramers(E, 80.0), I0 * kramers(E, 140.0)])
    n = n_views * n_u
    g = rng(3, "phantom")
    l = np.stack([g.uniform(0, 300, n), g.uniform(0, 30, n)])
    ybar = S @ np.exp(-(Q @ l))
    y = poisson(rng(3, "noise"), ybar)
    return Problem("c3_projdomain", None, Q, S, y, np.zeros((2, 2)), l, 100, "block", n)


def pc_channels(E, kvp: float, thresholds, I0: float):
    """Photon-counting channels with ideal bins [t_c, t_{c+1}) over a spectrum."""
    s = kramers(E, kvp)
    edges = list(thresholds) + [kvp + 1]
    return np.stack([I0 * s * ((E >= lo) & (E < hi)) for lo, hi in zip(edges[:-1], edges[1:])])


def mbmd_problem(config: int, geom: Geometry, mats, names, Q, S, beta, n_iter: int, precond: str,
                 name: str) -> Problem:
    """One-step MBMD data: per-material analytic line integrals of additive
    density ellipses, polyenergetic expected counts, Poisson noise."""
    o, d = geom.rays()
    l = np.stack([chord_lengths(shapes, o, d) for shapes in mats])       # [m, rays] (mm * g/cm^3)
    ybar = S @ np.exp(-(Q @ l))
    y = poisson(rng(config, "noise"), ybar)
    truth = np.stack([render(geom, shapes, supersample=2) for shapes in mats])
    return Problem(name, geom, Q, S, y, np.asarray(beta, dtype=np.float64), truth, n_iter, precond, geom.n_rays)


def mbmd_phantom(g: np.random.Generator, scale: float):
    """Water body with bone-like and iodine-like inserts (densities in g/cm^3:
    water 1.0, bone 0.3-1.5, iodine 0.005-0.02, inside the water)."""
    water = [Ellipse(0.0, 0.0, 110.0 * scale, 90.0 * scale, 0.0, 1.0)]
    bone = random_ellipses(g, 4, radius=75.0 * scale, amin=5.0 * scale, amax=18.0 * scale, vmin=0.3, vmax=1.5)
    iod = random_ellipses(g, 4, radius=75.0 * scale, amin=4.0 * scale, amax=12.0 * scale, vmin=0.005, vmax=0.02)
    return [water, bone, iod]


# written by oracle/derive_config4_beta.py (rounded)
CONFIG4_BETA = np.array([[0.5, 0.1, 3.1], [0.1, 2.1, 6.4], [3.1, 6.4, 1960.0]])


def config4_slice(nx: int = 512, n_views: int = 720, n_u: int = 888, slice_id: int = 0) -> Problem:
    """One slice of the one-step MBMD workload: 3 materials (water, bone-like,
    iodine-like with a 6x K-edge at 33.2 keV), 4 photon-counting channels
    [25,40) [40,60) [60,80) [80,120] keV under a 120 kVp spectrum (I0 = 1e5),
    fan beam like config 2 (bins scaled with the slice: the field of view
    follows the image), per-pixel 3x3 blocks + cross-material Fourier.
    beta (density units) = CONFIG4_BETA: 0.05 x the mean diagonal Fisher
    information over 2|N| at full size, with positive cross terms
    0.1 sqrt(beta_kk beta_k'k'), rounded."""
    E = np.arange(20.0, 121.0)
    Q = material_Q(E, ["water", "bone", "iodine"], rng(4, "materials"))
    S = pc_channels(E, 120.0, [25.0, 40.0, 60.0, 80.0], 1e5)
    g = rng(4, "phantom")
    for _ in range(slice_id):
        g = np.random.Generator(np.random.PCG64(g.integers(2 ** 63)))
    dx = 0.5 * 512 / nx
    geom = Geometry(FAN2D, nx, nx, 1, dx, dx, 1.0, n_views, 0.0, 2 * math.pi, n_u, 1, 1.0 * 888 / n_u, 1.0,
                    500.0, 1000.0)
    return mbmd_problem(4, geom, mbmd_phantom(g, 1.0), ["water", "bone", "iodine"], Q, S, CONFIG4_BETA, 100,
                        "block_fourier", f"c4_mbmd_{nx}")


CONFIG4_SIZES = (256, 320, 384, 448, 512)


def config4(n_slices: int = 16, n_views: int = 720, shrink: int = 1) -> list:
    """The batched one-step MBMD workload: n_slices independent slices whose
    sizes are drawn (seeded) from 256^2 .. 512^2; pixels stay 0.5 mm, so the
    field of view follows the slice, and each slice gets 4 ceil(888 N / 2048)
    curved bins of 1 mm (fan beam as config 2, 3 materials, 4 photon-counting
    channels, CONFIG4_BETA).  shrink > 1 divides every size, the bin count and
    the phantom by it (pixels and bins grow by the same factor) for
    oracle-sized runs of the same batch."""
    E = np.arange(20.0, 121.0)
    Q = material_Q(E, ["water", "bone", "iodine"], rng(4, "materials"))
    S = pc_channels(E, 120.0, [25.0, 40.0, 60.0, 80.0], 1e5)
    sizes = rng(4, "slices").choice(CONFIG4_SIZES, size=n_slices)
    g = rng(4, "phantom")
    out = []
    for k, n_full in enumerate(sizes):
        n_full = int(n_full)
        n = n_full // shrink
        n_u = 4 * math.ceil(888 * n_full / (4 * 512)) // shrink
        dx = 0.5 * shrink
        geom = Geometry(FAN2D, n, n, 1, dx, dx, 1.0, n_views, 0.0, 2 * math.pi, n_u, 1, 1.0 * shrink, 1.0,
                        500.0, 1000.0)
        gk = np.random.Generator(np.random.PCG64(g.integers(2 ** 63)))
        out.append(mbmd_problem(4, geom, mbmd_phantom(gk, n_full / 512.0), ["water", "bone", "iodine"], Q, S,
                                CONFIG4_BETA, 100, "block_fourier", f"c4_slice{k}_{n_full}"))
    return out


CONFIG5_BETA = np.array([[0.5, 3.0], [3.0, 2000.0]])


def config5(n: int = 256, n_views: int = 360, n_u: int = 512, n_v: int = 384, rays: bool = True,
            first_views: int | None = None) -> Problem:
    """3-D cone-beam one-step MBMD: 2 materials (water, iodine-like), 80/140 kVp
    dual-energy channels (each normalised to I0 = 5e4), 256^3 at 0.5 mm, 360
    views over 360 deg onto a 512 x 384 flat detector of 0.8 mm pixels, SID 600,
    SDD 1200; seeded ellipsoid phantom; per-voxel 2x2 blocks.  Smaller n /
    views / detector scale the same scan down (same field of view);
    first_views keeps only the first views of the orbit (same volume, same
    view spacing: a bounded part of the scan).  beta in
    density units: the water and iodine strengths of CONFIG4_BETA (rounded)
    with the cross term 0.1 sqrt(beta_11 beta_22)."""
    E = np.arange(20.0, 141.0)
    Q = material_Q(E, ["water", "iodine"], rng(5, "materials"))
    I0 = 5e4
    S = np.stack([I0 * kramers(E, 80.0), I0 * kramers(E, 140.0)])
    scale = 256.0 / n
    nv, span = n_views, 2 * math.pi
    if first_views is not None and first_views < n_views:
        nv, span = first_views, 2 * math.pi * first_views / n_views
    geom = Geometry(CONE3D, n, n, n, 0.5 * scale, 0.5 * scale, 0.5 * scale, nv, 0.0, span, n_u, n_v,
                    0.8 * 512 / n_u, 0.8 * 384 / n_v, 600.0, 1200.0)
    g = rng(5, "phantom")
    water = [Ellipsoid(0.0, 0.0, 0.0, 55.0, 45.0, 50.0, 0.0, 1.0)]
    iod = []
    for _ in range(5):
        r = g.uniform(4.0, 10.0)
        th = g.uniform(0, 2 * math.pi)
        rho = g.uniform(0, 30.0)
        iod.append(Ellipsoid(rho * math.cos(th), rho * math.sin(th), g.uniform(-25, 25), r, r * g.uniform(0.7, 1.3),
                             r * g.uniform(0.7, 1.3), g.uniform(0, math.pi), g.uniform(0.005, 0.02)))
    mats = [water, iod]
    truth = np.stack([render(geom, shapes, supersample=2) for shapes in mats])
    if not rays:
        return Problem("c5_cone3d", geom, Q, S, np.zeros((2, 0)), CONFIG5_BETA, truth, 50, "block", geom.n_rays)
    o, d = geom.rays()
    l = np.stack([chord_lengths(shapes, o, d) for shapes in mats])
    y = poisson(rng(5, "noise"), S @ np.exp(-(Q @ l)))
    return Problem("c5_cone3d", geom, Q, S, y, CONFIG5_BETA, truth, 50, "block", geom.n_rays)


# Detector cross-talk taps for the blurred-detector variants: a symmetric
# 3-cell kernel and an asymmetric 7-cell one (both sum to 1).
BLUR_TAPS = {"r1": (0.15, 0.70, 0.15), "r3": (0.02, 0.06, 0.20, 0.44, 0.18, 0.07, 0.03)}


def with_detector_blur(prob: Problem, taps: Sequence[float], n_u: int | None = None) -> Problem:
    """The same scan read out by a detector whose cells leak into their row
    neighbours: new counts are Poisson draws around the row-wise weighted sum
    of the measured counts with ``taps`` (2 r + 1 weights b_-r..b_r, cells past
    a row's ends contribute nothing).  Rows are n_u consecutive rays (default:
    the geometry's detector columns)."""
    b = np.asarray(taps, dtype=np.float64)
    r = b.size // 2
    n_u = int(n_u if n_u is not None else prob.geom.n_u)
    rows = prob.y.reshape(prob.y.shape[0], -1, n_u)
    pad = np.zeros(rows.shape[:-1] + (n_u + 2 * r,))
    pad[..., r:r + n_u] = rows
    mean = np.zeros_like(rows)
    for j, bj in enumerate(b):
        mean += bj * pad[..., j:j + n_u]
    y = poisson(rng(len(b), "misc"), mean.reshape(prob.y.shape))
    return dataclasses.replace(prob, y=y, name=prob.name + f"_blur{r}")
