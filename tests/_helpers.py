"""Shared helpers for the GPU parity tests (inputs come from ``synth``;
expected values from ``oracle``)."""
import math

import numpy as np

import synth
from synth import FAN2D, PAR2D, Geometry


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    e = float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
    try:                      # the session's error log (tests/conftest.py)
        import conftest
        conftest._ERRORS.note(e)
    except Exception:
        pass
    return e


def to_dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device="cuda")


def to_host(t):
    return t.detach().double().cpu().numpy()


def cone_geoms():
    return {
        "cone_small": synth.config5(n=32, n_views=24, n_u=64, n_v=48, rays=False).geom,
        "cone_ragged": Geometry(synth.CONE3D, 21, 18, 13, 0.9, 1.0, 1.2, 17, 0.3, 2 * math.pi, 37, 23, 1.1, 1.3,
                                 60.0, 130.0),
    }


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
    if geom.kind == synth.CONE3D:
        for m in range(nm):
            shapes = [synth.Ellipsoid(*rng.uniform(-3, 3, 3), *rng.uniform(3, 8, 3), rng.uniform(0, 3),
                                      rng.uniform(0.01, 0.03)) for _ in range(3)]
            out.append(synth.render(geom, shapes, supersample=2) + 0.002 * rng.random(geom.image_shape))
        return np.stack(out)
    for m in range(nm):
        shapes = synth.random_ellipses(rng, 4, radius=0.4 * min(geom.nx * geom.dx, geom.ny * geom.dy),
                                       amin=0.05 * geom.nx * geom.dx, amax=0.15 * geom.nx * geom.dx,
                                       vmin=0.01, vmax=0.03)
        out.append(synth.render(geom, shapes, supersample=2) + 0.002 * rng.random(geom.image_shape))
    return np.stack(out)


def oracle_precond(oracle_lib, prob, kind, lattice=3, proj=True, blur=None, sides=None):
    """Oracle preconditioner for a problem plus the data that defines it
    (eigenvalues, m0, blocks in the library's [m][k][n] layout).  blur: an
    ``oracle.model.Blur`` in the outer operator (the preconditioners use the
    blur-free Fisher blocks either way)."""
    from oracle import build, precond, psps as opsps
    A = oracle_lib.Projector(prob.geom) if proj else oracle_lib.IdentityProjector(prob.n_rays)
    st = opsps.Setup(A, prob.Q, prob.S, prob.y, prob.beta if proj else None, blur=blur)
    if kind == "none":
        return st, precond.Identity(), {}
    F = build.fisher(st)
    aH = build.make_apply_H(st, F)
    if sides is None:        # each kind's default
        sides = 1 if kind in ("block_fourier", "block_haar") else 2
    if kind == "fourier":
        lam = precond.fourier_eigenvalues(aH, st.shape)
        return st, precond.Fourier(lam), {"lam": lam}
    B = build.m0_blocks(st, F)
    blocks = np.ascontiguousarray(np.transpose(B, (1, 2, 0)))
    if kind == "block":
        return st, precond.Block(B, st.shape), {"blocks": blocks}
    if kind == "block_fourier":
        M0 = precond.Block(B, st.shape)
        L = precond.cross_fourier_blocks(aH, M0, st.shape, st.nm)
        P = precond.polar_real(L)
        lam = np.ascontiguousarray(np.transpose(P.reshape(-1, st.nm, st.nm), (1, 2, 0)))
        return st, precond.CrossFourier(L, M0, sides), {"lam": lam, "blocks": blocks}
    if kind == "block_haar":
        M0 = precond.Block(B, st.shape)
        K = precond.cross_haar_blocks(aH, M0, st.shape, st.nm, lattice)
        P = precond.polar_real(K)
        lam = np.ascontiguousarray(np.transpose(P.reshape(-1, st.nm, st.nm), (1, 2, 0)))
        return st, precond.CrossHaar(K, M0, sides), {"lam": lam, "blocks": blocks}
    m0 = B[:, 0, 0].reshape(st.shape)

    def aN(v):
        return m0[None] * aH(m0[None] * v)
    if kind == "mod_fourier":
        lam = precond.fourier_eigenvalues(aN, st.shape)
        return st, precond.Fourier(lam, m0, sides), {"lam": lam, "m0": m0}
    if kind == "haar":
        lam = precond.haar_eigenvalues(aN, st.shape, lattice=lattice)
        return st, precond.Haar(lam, m0, sides), {"lam": lam, "m0": m0}
    raise ValueError(kind)


def gpu_precond_from(psps, plan, spec, kind, data, sides=None):
    """The library's preconditioner created from the oracle's data."""
    if kind == "none":
        return None
    kw = {k: to_dev(v) for k, v in data.items()}
    return psps.Precond(plan, spec, kind, sides=sides, **kw)


def _haar_part(job):
    """Worker: one share of the oracle's Haar test sets for a seeded problem
    (rebuilt here from its synth builder and keywords)."""
    builder, kw, i, n = job
    import oracle
    from oracle import build, precond, psps as opsps
    oracle.build_c()
    prob = getattr(synth, builder)(**kw)
    st = opsps.Setup(oracle.Projector(prob.geom), prob.Q, prob.S, prob.y, prob.beta)
    F = build.fisher(st)
    aH = build.make_apply_H(st, F)
    m0 = build.m0_blocks(st, F)[:, 0, 0].reshape(st.shape)
    return precond.haar_eigenvalues(lambda v: m0[None] * aH(m0[None] * v), st.shape, part=(i, n))


def oracle_haar_parallel(oracle_lib, builder, kw, processes=None):
    """The oracle's Haar preconditioner (Eq. 34 with the lattice test
    functions) of a seeded problem, its test sets evaluated in spawned
    processes (single-threaded BLAS each); returns (Setup, preconditioner)."""
    import multiprocessing as mp
    import os
    from oracle import build, precond, psps as opsps
    prob = getattr(synth, builder)(**kw)
    st = opsps.Setup(oracle_lib.Projector(prob.geom), prob.Q, prob.S, prob.y, prob.beta)
    m0 = build.m0_blocks(st, build.fisher(st))[:, 0, 0].reshape(st.shape)
    try:
        n = processes or len(os.sched_getaffinity(0))
    except AttributeError:
        n = processes or (os.cpu_count() or 1)
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    try:
        with mp.get_context("spawn").Pool(n) as pool:
            parts = pool.map(_haar_part, [(builder, kw, i, n) for i in range(n)])
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return st, precond.Haar(sum(parts), m0)   # the kind's default (literal) form
