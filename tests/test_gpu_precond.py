"""GPU preconditioner applies and builds against the oracle.

Applies are checked with the preconditioner created from the oracle's own
eigenvalues / blocks (tolerance 1e-5: the FP32 FFT and Haar kernels).  The
GPU build itself runs in FP32 (impulse responses through the FP32 projector,
FP32 FFT) and is checked against the FP64 build at 1e-3: the eigenvalues at
the smallest frequencies are differences of large responses, where FP32
rounding of ~1e-7 of the largest response becomes ~1e-4 of the smallest.
"""
import numpy as np
import pytest

import synth
from _helpers import gpu_precond_from, oracle_precond, rel_l2, to_dev, to_host

pytestmark = pytest.mark.gpu

APPLY_TOL = 1e-5
BUILD_TOL = 1e-3


@pytest.fixture(scope="module")
def psps():
    import paper_2010_01371_gb300 as p
    p.lib()
    return p


def problems():
    return {"c1": synth.config1(), "c2_64": synth.config2(nx=64, n_views=90, n_u=111)}


OPS = ["M", "MT", "absM", "absMT"]


def check_ops(psps, pc, P, shape, tol, seed=3):
    v = np.random.default_rng(seed).standard_normal(shape)
    for op in OPS:
        got = to_host(psps.psps_precondition(pc, op, to_dev(v)))
        want = getattr(P, op)(v)
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
@pytest.mark.parametrize("kind", ["fourier", "mod_fourier", "haar", "block"])
def test_build_parity(psps, oracle_lib, pname, kind):
    prob = problems()[pname]
    st, P, _ = oracle_precond(oracle_lib, prob, kind)
    plan, spec = psps.Plan(prob.geom), psps.Spectrum(prob.Q, prob.S)
    pc = psps.Precond(plan, spec, kind, to_dev(prob.y), prob.beta)
    check_ops(psps, pc, P, (1,) + prob.geom.image_shape, BUILD_TOL)


@pytest.mark.parametrize("kind", ["block", "block_fourier", "block_haar"])
def test_mbmd_apply_and_build(psps, oracle_lib, kind):
    """One-step MBMD (3 materials): per-pixel 3x3 blocks, the cross-material
    Fourier (Eq. 57) and the cross-material wavelet (Eq. 61) preconditioners,
    created from the oracle's data (apply tolerance) and built on the GPU
    (build tolerance)."""
    prob = synth.config4_slice(nx=64, n_views=90, n_u=111)
    st, P, data = oracle_precond(oracle_lib, prob, kind)
    plan, spec = psps.Plan(prob.geom), psps.Spectrum(prob.Q, prob.S)
    shape = (3,) + prob.geom.image_shape
    check_ops(psps, gpu_precond_from(psps, plan, spec, kind, data), P, shape, APPLY_TOL)
    check_ops(psps, psps.Precond(plan, spec, kind, to_dev(prob.y), prob.beta), P, shape, BUILD_TOL)


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
    check_ops(psps, psps.Precond(plan, spec, kind, to_dev(prob.y), prob.beta), P, shape, BUILD_TOL)


@pytest.mark.parametrize("n", [40, 48, 56])
def test_mixed_radix_cross_material(psps, oracle_lib, n):
    """Cross-material Fourier (Eq. 57) on the uneven slice sizes of the batched
    MBMD workload (320/384/448 shrunk by 8: radix 5, 3 and 7)."""
    prob = next(p for p in synth.config4(n_views=90, shrink=8) if p.geom.nx == n)
    st, P, data = oracle_precond(oracle_lib, prob, "block_fourier")
    plan, spec = psps.Plan(prob.geom), psps.Spectrum(prob.Q, prob.S)
    shape = (3,) + prob.geom.image_shape
    check_ops(psps, gpu_precond_from(psps, plan, spec, "block_fourier", data), P, shape, APPLY_TOL)
    check_ops(psps, psps.Precond(plan, spec, "block_fourier", to_dev(prob.y), prob.beta), P, shape, BUILD_TOL)


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
    check_ops(psps, psps.Precond(plan, spec, kind, to_dev(prob.y), prob.beta), P, shape, BUILD_TOL)


def test_3d_cross_material_fourier(psps, oracle_lib):
    """Cross-material Fourier (Eq. 57) over the voxel grid with per-voxel 2x2
    M0 on the two-material cone-beam workload (32^3)."""
    prob = synth.config5(n=32, n_views=24, n_u=64, n_v=48)
    st, P, data = oracle_precond(oracle_lib, prob, "block_fourier")
    plan, spec = psps.Plan(prob.geom), psps.Spectrum(prob.Q, prob.S)
    shape = (2,) + prob.geom.image_shape
    check_ops(psps, gpu_precond_from(psps, plan, spec, "block_fourier", data), P, shape, APPLY_TOL)
    check_ops(psps, psps.Precond(plan, spec, "block_fourier", to_dev(prob.y), prob.beta), P, shape, BUILD_TOL)
    with pytest.raises(RuntimeError):
        psps.Precond(plan, spec, "block_haar", to_dev(prob.y), prob.beta)
