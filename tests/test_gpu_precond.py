"""GPU preconditioner applies and builds against the oracle.

Applies are checked with the preconditioner created from the oracle's own
eigenvalues / blocks (tolerance 1e-5: the FP32 FFT and Haar kernels).  The
GPU build itself applies the Hessian in FP32; its arrays are bounded element
by element in test_gpu_build.py (Weyl: an eigenvalue estimate moves by up to
eps_b lambda_max, eps_b ~ 8 n 2^-24).  Here the built preconditioner's
operators M, M^T, |M|, |M|^T are compared with the FP64 build's, in relative
L2, at a tolerance per kind a few times the measured error: plain Fourier
1e-3 (its spectrum spans about three and a half decades, so its smallest
eigenvalues carry ~1e-4..1e-3), modified Fourier and the cross-material kinds
1e-4, Haar and the blocks 1e-5.
"""
import numpy as np
import pytest

import synth
from _helpers import gpu_precond_from, oracle_precond, rel_l2, to_dev, to_host

pytestmark = pytest.mark.gpu

APPLY_TOL = 1e-5
BUILD_TOLS = {"fourier": 1e-3, "mod_fourier": 1e-4, "haar": 1e-5, "block": 1e-5, "block_fourier": 1e-4,
              "block_haar": 1e-4}


@pytest.fixture(scope="module")
def psps():
    import paper_2010_01371_gb300 as p
    p.lib()
    return p


def problems():
    return {"c1": synth.config1(), "c2_64": synth.config2(nx=64, n_views=90, n_u=111)}


OPS = ["M", "MT", "absM", "absMT"]


def check_ops(psps, pc, P, shape, tol, seed=3, log=None, name=""):
    v = np.random.default_rng(seed).standard_normal(shape)
    for op in OPS:
        got = to_host(psps.psps_precondition(pc, op, to_dev(v)))
        want = getattr(P, op)(v)
        if log is not None:
            log.add(name, f"apply {op}", rel_l2(got, want), tol)
        assert rel_l2(got, want) < tol, (op, rel_l2(got, want))


@pytest.mark.parametrize("pname", ["c1", "c2_64"])
@pytest.mark.parametrize("kind", ["fourier", "mod_fourier", "haar", "block"])
def test_apply_parity(psps, oracle_lib, pname, kind):
    prob = problems()[pname]
    st, P, data = oracle_precond(oracle_lib, prob, kind)
    plan, spec = psps.Plan(prob.geom), psps.Spectrum(prob.Q, prob.S)
    pc = gpu_precond_from(psps, plan, spec, kind, data)
    check_ops(psps, pc, P, (1,) + prob.geom.image_shape, APPLY_TOL)


@pytest.mark.parametrize("pname", ["c1", "c2_64"])
@pytest.mark.parametrize("kind", ["mod_fourier", "haar", "block_fourier", "block_haar"])
@pytest.mark.parametrize("sides", [1, 2])
def test_sides_apply_parity(psps, oracle_lib, pname, kind, sides):
    """Both placements of M0 (psps_precondition_set_sides): the one-sided
    M0^T C and the literal two-sided M0^T C M0 of Eqs. 33, 34, 57, 61, against
    the oracle's; and the kinds' defaults (2 for one material, 1 for the
    cross-material kinds) match the oracle's defaults."""
    prob = problems()[pname] if kind in ("mod_fourier", "haar") else synth.config4_slice(nx=64, n_views=90, n_u=111)
    st, P, data = oracle_precond(oracle_lib, prob, kind, sides=sides)
    plan, spec = psps.Plan(prob.geom), psps.Spectrum(prob.Q, prob.S)
    pc = gpu_precond_from(psps, plan, spec, kind, data, sides=sides)
    check_ops(psps, pc, P, (st.nm,) + prob.geom.image_shape, APPLY_TOL)
    default = 1 if kind.startswith("block_") else 2
    if sides == default:
        check_ops(psps, gpu_precond_from(psps, plan, spec, kind, data), P, (st.nm,) + prob.geom.image_shape,
                  APPLY_TOL)
    with pytest.raises(psps.MbirError):
        psps.lib()
        from paper_2010_01371_gb300 import _abi
        _abi.check(psps.lib().psps_precondition_set_sides(pc.h, 3))


@pytest.mark.parametrize("pname", ["c1", "c2_64"])
@pytest.mark.parametrize("kind", ["fourier", "mod_fourier", "haar", "block"])
def test_build_parity(psps, oracle_lib, error_log, pname, kind):
    prob = problems()[pname]
    st, P, _ = oracle_precond(oracle_lib, prob, kind)
    plan, spec = psps.Plan(prob.geom), psps.Spectrum(prob.Q, prob.S)
    pc = psps.Precond(plan, spec, kind, to_dev(prob.y), prob.beta)
    check_ops(psps, pc, P, (1,) + prob.geom.image_shape, BUILD_TOLS[kind], log=error_log,
              name=f"GPU-built {pname} {kind}")


@pytest.mark.parametrize("kind", ["block", "block_fourier", "block_haar"])
def test_mbmd_apply_and_build(psps, oracle_lib, error_log, kind):
    """One-step MBMD (3 materials): per-pixel 3x3 blocks, the cross-material
    Fourier (Eq. 57) and the cross-material wavelet (Eq. 61) preconditioners,
    created from the oracle's data (apply tolerance) and built on the GPU
    (build tolerance)."""
    prob = synth.config4_slice(nx=64, n_views=90, n_u=111)
    st, P, data = oracle_precond(oracle_lib, prob, kind)
    plan, spec = psps.Plan(prob.geom), psps.Spectrum(prob.Q, prob.S)
    shape = (3,) + prob.geom.image_shape
    check_ops(psps, gpu_precond_from(psps, plan, spec, kind, data), P, shape, APPLY_TOL)
    check_ops(psps, psps.Precond(plan, spec, kind, to_dev(prob.y), prob.beta), P, shape, BUILD_TOLS[kind],
              log=error_log, name=f"GPU-built c4_64 {kind}")


def test_projection_domain_block(psps, oracle_lib):
    prob = synth.config3(n_views=10, n_u=333)
    st, P, data = oracle_precond(oracle_lib, prob, "block", proj=False)
    spec = psps.Spectrum(prob.Q, prob.S)
    shape = (2, prob.n_rays)
    check_ops(psps, gpu_precond_from(psps, None, spec, "block", data), P, shape, APPLY_TOL)
    check_ops(psps, psps.Precond(None, spec, "block", to_dev(prob.y)), P, shape, APPLY_TOL)


def test_paper_single_test_function(psps, oracle_lib):
    """haar_lattice = 0 is Eq. 18 with the single test function U^T 1.  Its
    estimate is a sum of responses that nearly cancel, so the FP32 build
    carries ~1e-3 relative error; checked at 1e-2."""
    prob = problems()["c1"]
    st, P, data = oracle_precond(oracle_lib, prob, "haar", lattice=0)
    plan, spec = psps.Plan(prob.geom), psps.Spectrum(prob.Q, prob.S)
    check_ops(psps, gpu_precond_from(psps, plan, spec, "haar", data), P, (1, 64, 64), APPLY_TOL)
    pc = psps.Precond(plan, spec, "haar", to_dev(prob.y), prob.beta, haar_lattice=0)
    check_ops(psps, pc, P, (1, 64, 64), 1e-2)


def mixed_radix_problem():
    """Non-square image whose sides need the radix-3, 5 and 7 FFT passes
    (45 = 3^2 5, 56 = 2^3 7), parallel beam."""
    import math
    g = synth.rng(1, "phantom")
    geom = synth.Geometry(synth.PAR2D, 45, 56, 1, 1.0, 1.0, 1.0, 60, 0.0, math.pi, 80, 1, 1.0, 1.0)
    shapes = synth.random_ellipses(g, 4, radius=20.0, amin=3.0, amax=12.0, vmin=0.01, vmax=0.03)
    return synth.mbir_problem(1, geom, shapes, 1e4, 1e3, 50, "fourier", "mixed_radix_45x56")


@pytest.mark.parametrize("kind", ["fourier", "mod_fourier"])
def test_mixed_radix_fourier(psps, oracle_lib, kind):
    """Fourier preconditioners (Eqs. 27-33) on a 45 x 56 image: apply from the
    oracle's spectrum and GPU build, against numpy's FFT in the oracle."""
    prob = mixed_radix_problem()
    st, P, data = oracle_precond(oracle_lib, prob, kind)
    plan, spec = psps.Plan(prob.geom), psps.Spectrum(prob.Q, prob.S)
    shape = (1,) + prob.geom.image_shape
    check_ops(psps, gpu_precond_from(psps, plan, spec, kind, data), P, shape, APPLY_TOL)
    check_ops(psps, psps.Precond(plan, spec, kind, to_dev(prob.y), prob.beta), P, shape, BUILD_TOLS[kind])


@pytest.mark.parametrize("n", [40, 48, 56])
def test_mixed_radix_cross_material(psps, oracle_lib, n):
    """Cross-material Fourier (Eq. 57) on the uneven slice sizes of the batched
    MBMD workload (320/384/448 shrunk by 8: radix 5, 3 and 7)."""
    prob = next(p for p in synth.config4(n_views=90, shrink=8) if p.geom.nx == n)
    st, P, data = oracle_precond(oracle_lib, prob, "block_fourier")
    plan, spec = psps.Plan(prob.geom), psps.Spectrum(prob.Q, prob.S)
    shape = (3,) + prob.geom.image_shape
    check_ops(psps, gpu_precond_from(psps, plan, spec, "block_fourier", data), P, shape, APPLY_TOL)
    check_ops(psps, psps.Precond(plan, spec, "block_fourier", to_dev(prob.y), prob.beta), P, shape,
              BUILD_TOLS["block_fourier"])


def cone_mbir_problem():
    """One-material cone-beam problem on the 32^3 scaled-down config-5 scan."""
    g = synth.config5(n=32, n_views=24, n_u=64, n_v=48, rays=False).geom
    shapes = [synth.Ellipsoid(0.0, 0.0, 0.0, 50.0, 40.0, 45.0, 0.3, 0.02),
              synth.Ellipsoid(15.0, -10.0, 5.0, 12.0, 9.0, 10.0, 0.0, 0.01)]
    return synth.mbir_problem(5, g, shapes, 1e4, 1e3, 50, "fourier", "cone_mbir_32")


@pytest.mark.parametrize("kind", ["fourier", "mod_fourier"])
def test_3d_fourier(psps, oracle_lib, kind):
    """3-D Fourier preconditioners (Eqs. 27-33 over the voxel grid, 3-D FFT):
    apply from the oracle's spectrum and GPU build."""
    prob = cone_mbir_problem()
    st, P, data = oracle_precond(oracle_lib, prob, kind)
    plan, spec = psps.Plan(prob.geom), psps.Spectrum(prob.Q, prob.S)
    shape = (1,) + prob.geom.image_shape
    check_ops(psps, gpu_precond_from(psps, plan, spec, kind, data), P, shape, APPLY_TOL)
    check_ops(psps, psps.Precond(plan, spec, kind, to_dev(prob.y), prob.beta), P, shape, BUILD_TOLS[kind])


def test_3d_cross_material_fourier(psps, oracle_lib):
    """Cross-material Fourier (Eq. 57) over the voxel grid with per-voxel 2x2
    M0 on the two-material cone-beam workload (32^3)."""
    prob = synth.config5(n=32, n_views=24, n_u=64, n_v=48)
    st, P, data = oracle_precond(oracle_lib, prob, "block_fourier")
    plan, spec = psps.Plan(prob.geom), psps.Spectrum(prob.Q, prob.S)
    shape = (2,) + prob.geom.image_shape
    check_ops(psps, gpu_precond_from(psps, plan, spec, "block_fourier", data), P, shape, APPLY_TOL)
    check_ops(psps, psps.Precond(plan, spec, "block_fourier", to_dev(prob.y), prob.beta), P, shape,
              BUILD_TOLS["block_fourier"])


def cone_haar_problem(n=16):
    """One-material cone-beam problem on the config-5 scan scaled to n^3."""
    g = synth.config5(n=n, n_views=12 * n // 16, n_u=2 * n, n_v=3 * n // 2, rays=False).geom
    shapes = [synth.Ellipsoid(0.0, 0.0, 0.0, 50.0, 40.0, 45.0, 0.3, 0.02),
              synth.Ellipsoid(15.0, -10.0, 5.0, 12.0, 9.0, 10.0, 0.0, 0.01)]
    return synth.mbir_problem(5, g, shapes, 1e4, 1e3, 50, "haar", f"cone_mbir_{n}")


@pytest.mark.parametrize("n", [16, 32, 64])
def test_3d_haar_apply(psps, oracle_lib, n):
    """3-D Haar preconditioner (Eq. 34 over the voxel grid) from given
    eigenvalues and m0: 16^3 is one shared-memory tile, 32^3 and 64^3 add the
    coarse low-pass stage (2^3 and 4^3 tiles)."""
    from oracle import precond
    geom = synth.config5(n=n, n_views=12, n_u=2 * n, n_v=3 * n // 2, rays=False).geom
    rng = np.random.default_rng(n)
    lam = rng.uniform(0.1, 10.0, geom.image_shape)
    m0 = rng.uniform(0.5, 2.0, geom.image_shape)
    P = precond.Haar(lam, m0)
    plan, spec = psps.Plan(geom), psps.Spectrum(np.ones((1, 1)), np.full((1, 1), 1e4))
    pc = psps.Precond(plan, spec, "haar", lam=to_dev(lam), m0=to_dev(m0))
    check_ops(psps, pc, P, (1,) + geom.image_shape, APPLY_TOL)


def test_3d_cross_haar_apply(psps, oracle_lib):
    """Cross-material wavelet (Eq. 61) over a 32^3 volume from given blocks."""
    from oracle import precond
    geom = synth.config5(n=32, n_views=12, n_u=64, n_v=48, rays=False).geom
    nm, shape = 2, geom.image_shape
    n = int(np.prod(shape))
    rng = np.random.default_rng(5)
    G = rng.standard_normal(shape + (nm, nm))
    K = np.einsum("...ij,...kj->...ik", G, G) + 0.3 * np.eye(nm) + 0.2 * rng.standard_normal(shape + (nm, nm))
    Gb = rng.standard_normal((n, nm, nm))
    B = np.einsum("nij,nkj->nik", Gb, Gb) + np.eye(nm)
    M0 = precond.Block(B, shape)
    P = precond.CrossHaar(K, M0)
    Pp = precond.polar_real(K)
    lam = np.ascontiguousarray(np.transpose(Pp.reshape(-1, nm, nm), (1, 2, 0)))
    blocks = np.ascontiguousarray(np.transpose(B, (1, 2, 0)))
    E = np.arange(20.0, 141.0)
    spec = psps.Spectrum(synth.material_Q(E, ["water", "iodine"], rng), np.ones((2, E.size)))
    pc = psps.Precond(psps.Plan(geom), spec, "block_haar", lam=to_dev(lam), blocks=to_dev(blocks))
    check_ops(psps, pc, P, (nm,) + shape, APPLY_TOL)


def test_3d_haar_build(psps, oracle_lib):
    """GPU build of the 3-D Haar eigenvalues (Eq. 18 with the 3-D lattice test
    functions) against the FP64 build on a 16^3 cone-beam problem."""
    prob = cone_haar_problem(16)
    st, P, data = oracle_precond(oracle_lib, prob, "haar")
    plan, spec = psps.Plan(prob.geom), psps.Spectrum(prob.Q, prob.S)
    shape = (1,) + prob.geom.image_shape
    check_ops(psps, gpu_precond_from(psps, plan, spec, "haar", data), P, shape, APPLY_TOL)
    check_ops(psps, psps.Precond(plan, spec, "haar", to_dev(prob.y), prob.beta), P, shape, BUILD_TOLS["haar"])


def test_3d_cross_material_wavelet_build(psps, oracle_lib):
    """Cross-material wavelet blocks (Eqs. 59-60) over a 16^3 volume with the
    two-material cone-beam workload: apply from the oracle's blocks and GPU
    build (batched (set, material) probes)."""
    prob = synth.config5(n=16, n_views=12, n_u=32, n_v=24)
    st, P, data = oracle_precond(oracle_lib, prob, "block_haar")
    plan, spec = psps.Plan(prob.geom), psps.Spectrum(prob.Q, prob.S)
    shape = (2,) + prob.geom.image_shape
    check_ops(psps, gpu_precond_from(psps, plan, spec, "block_haar", data), P, shape, APPLY_TOL)
    check_ops(psps, psps.Precond(plan, spec, "block_haar", to_dev(prob.y), prob.beta), P, shape,
              BUILD_TOLS["block_haar"])


def test_3d_haar_rejects_non_cubes(psps):
    from paper_2010_01371_gb300._abi import MbirError
    geom = synth.Geometry(synth.CONE3D, 16, 16, 8, 1.0, 1.0, 1.0, 12, 0.0, 6.283185307179586, 32, 24, 1.0, 1.0,
                          60.0, 120.0)
    plan, spec = psps.Plan(geom), psps.Spectrum(np.ones((1, 1)), np.full((1, 1), 1e4))
    with pytest.raises(MbirError):
        psps.Precond(plan, spec, "haar", lam=to_dev(np.ones(geom.image_shape)))
