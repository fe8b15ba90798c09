"""GPU Joseph projector / backprojector parity with the FP64 oracle."""
import math

import numpy as np
import pytest

import synth
from _helpers import cone_geoms, phantom, rel_l2, small_geoms, to_dev, to_host
from synth import FAN2D, PAR2D, Geometry

pytestmark = pytest.mark.gpu

TOL = 1e-5   # relative L2, projections and backprojections


@pytest.fixture(scope="module")
def psps():
    import paper_2010_01371_gb300 as p
    p.lib()
    return p


@pytest.mark.parametrize("name", list(small_geoms()))
@pytest.mark.parametrize("nm", [1, 2])
@pytest.mark.parametrize("mode", ["tile", "ray", "strip"])
def test_project_parity(psps, oracle_lib, name, nm, mode):
    g = small_geoms()[name]
    x = phantom(g, seed=1, nm=nm)
    plan = psps.Plan(g)
    plan.set_projector(mode)
    got = to_host(psps.mbir_project(plan, to_dev(x)))
    want = oracle_lib.Projector(g).project(x)
    assert got.shape == want.shape
    assert rel_l2(got, want) < TOL, rel_l2(got, want)


@pytest.mark.parametrize("name", list(small_geoms()))
@pytest.mark.parametrize("mode", ["tile", "gather", "atomic"])
def test_backproject_parity(psps, oracle_lib, name, mode):
    g = small_geoms()[name]
    rng = np.random.default_rng(2)
    s = rng.random((2, g.n_rays))
    plan = psps.Plan(g)
    plan.set_backprojector(mode)
    got = to_host(psps.mbir_backproject(plan, to_dev(s)))
    want = oracle_lib.Projector(g).backproject(s)
    assert rel_l2(got, want) < TOL, rel_l2(got, want)
    # accumulate = 1 adds to the existing contents
    base = to_dev(np.ones((2,) + g.image_shape))
    psps.mbir_backproject(plan, to_dev(s), base, accumulate=True)
    assert rel_l2(to_host(base), want + 1.0) < TOL


@pytest.mark.parametrize("nm", [3, 4, 5])
@pytest.mark.parametrize("mode", ["tile", "ray", "strip"])
def test_material_packing(psps, oracle_lib, nm, mode):
    g = small_geoms()["fan2d_ragged"]
    x = phantom(g, seed=3, nm=nm)
    plan = psps.Plan(g)
    plan.set_projector(mode)
    got = to_host(psps.mbir_project(plan, to_dev(x)))
    assert rel_l2(got, oracle_lib.Projector(g).project(x)) < TOL


@pytest.mark.parametrize("nch", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("mode", ["tile", "gather"])
def test_transpose_channels(psps, oracle_lib, nch, mode):
    """The transposes handle 1..5 channels (groups of 4 / 2 / 1)."""
    for name in ["par2d_ragged", "fan2d_ragged"]:
        g = small_geoms()[name]
        s = np.random.default_rng(7).random((nch, g.n_rays))
        plan = psps.Plan(g)
        plan.set_backprojector(mode)
        got = to_host(psps.mbir_backproject(plan, to_dev(s)))
        assert rel_l2(got, oracle_lib.Projector(g).backproject(s)) < TOL


def test_transposes_agree(psps):
    g = synth.config2().geom
    s = to_dev(np.random.default_rng(8).random((2, g.n_rays)))
    out = {}
    for mode in ["tile", "gather", "atomic"]:
        p = psps.Plan(g)
        p.set_backprojector(mode)
        out[mode] = to_host(psps.mbir_backproject(p, s))
    assert rel_l2(out["tile"], out["gather"]) < 1e-6
    assert rel_l2(out["atomic"], out["gather"]) < 1e-6
    # the gather is deterministic: bitwise equal on a second run
    p = psps.Plan(g)
    p.set_backprojector("gather")
    assert np.array_equal(out["gather"], to_host(psps.mbir_backproject(p, s)))


@pytest.mark.parametrize("vs", [1, 7, 60, 180])
def test_transpose_view_split(psps, oracle_lib, vs):
    """Any number of views per CTA of the tile transpose gives the same A^T y
    (a chunk may end mid-scan, including a last chunk of one view)."""
    for name in ["par2d_ragged", "fan2d_ragged"]:
        g = small_geoms()[name]
        s = np.random.default_rng(9).random((2, g.n_rays))
        plan = psps.Plan(g)
        plan.set_tiling(vs)
        got = to_host(psps.mbir_backproject(plan, to_dev(s)))
        assert rel_l2(got, oracle_lib.Projector(g).backproject(s)) < TOL
    with pytest.raises(RuntimeError):
        plan.set_tiling(0)
    with pytest.raises(RuntimeError):
        plan.set_tiling(181)


def test_adjoint_fp32(psps):
    g = small_geoms()["fan2d_c2_128"]
    rng = np.random.default_rng(4)
    x = rng.random((1,) + g.image_shape)
    y = rng.random((1, g.n_rays))
    plan = psps.Plan(g)
    Ax = to_host(psps.mbir_project(plan, to_dev(x)))
    Aty = to_host(psps.mbir_backproject(plan, to_dev(y)))
    lhs, rhs = float(np.sum(Ax * y)), float(np.sum(x * Aty))
    assert abs(lhs - rhs) <= 1e-6 * abs(lhs)


@pytest.mark.parametrize("mode", ["tile", "ray", "strip"])
def test_full_size_sampled(psps, oracle_lib, mode):
    """Full 512^2 / 720 x 888 fan-beam geometry: every 97th ray (plus the
    first and last) against the oracle ray by ray, and the adjoint identity
    at full size."""
    prob = synth.config2()
    g = prob.geom
    x = prob.truth
    plan = psps.Plan(g)
    plan.set_projector(mode)
    got = to_host(psps.mbir_project(plan, to_dev(x)))[0]
    rays = np.unique(np.concatenate([np.arange(0, g.n_rays, 97), [g.n_rays - 1]]))
    want = oracle_lib.Projector(g).project_rays(x[0], rays)
    assert rel_l2(got[rays], want) < TOL, rel_l2(got[rays], want)
    rng = np.random.default_rng(5)
    y = rng.random((1, g.n_rays))
    Aty = to_host(psps.mbir_backproject(plan, to_dev(y)))
    lhs, rhs = float(np.sum(got * y[0])), float(np.sum(x * Aty))
    assert abs(lhs - rhs) <= 1e-6 * abs(lhs)


def test_empty_and_errors(psps):
    import torch
    g = small_geoms()["par2d_ragged"]
    plan = psps.Plan(g, n_mat_max=2)
    x = torch.zeros((3,) + g.image_shape, device="cuda")
    with pytest.raises(psps.MbirError):
        psps.mbir_project(plan, x, n_mat=3)
    # an all-zero image projects to zeros
    z = psps.mbir_project(plan, torch.zeros((1,) + g.image_shape, device="cuda"))
    assert float(z.abs().max()) == 0.0


@pytest.mark.parametrize("name", list(cone_geoms()))
@pytest.mark.parametrize("nm", [1, 2, 3])
def test_cone_project_parity(psps, oracle_lib, name, nm):
    """Cone forward, both marches: each lane over its own range and the
    warp-aligned one, which takes the same samples in the same order (bitwise
    equal)."""
    g = cone_geoms()[name]
    x = phantom(g, seed=11, nm=nm)
    plan = psps.Plan(g)
    got = to_host(psps.mbir_project(plan, to_dev(x)))
    want = oracle_lib.Projector(g).project(x)
    assert rel_l2(got, want) < TOL, rel_l2(got, want)
    plan.set_projector("aligned")
    assert np.array_equal(to_host(psps.mbir_project(plan, to_dev(x))), got)


@pytest.mark.parametrize("name", list(cone_geoms()))
@pytest.mark.parametrize("mode", ["tile", "gather", "atomic", "split"])
@pytest.mark.parametrize("nch", [1, 2, 3, 5])
def test_cone_backproject_parity(psps, oracle_lib, name, mode, nch):
    """3-D transposes: the fixed-point tile scatter (default, 'tile'), the
    direct voxel-driven gather ('gather'; channel groups of 4 / 2 / 1), the
    ray-driven atomic scatter and the gather with split tables ('split');
    accumulate adds."""
    g = cone_geoms()[name]
    s = np.random.default_rng(12).random((nch, g.n_rays))
    plan = psps.Plan(g)
    plan.set_backprojector(mode)
    got = to_host(psps.mbir_backproject(plan, to_dev(s)))
    want = oracle_lib.Projector(g).backproject(s)
    assert rel_l2(got, want) < TOL, rel_l2(got, want)
    base = to_dev(np.ones((nch,) + g.image_shape))
    psps.mbir_backproject(plan, to_dev(s), base, accumulate=True)
    assert rel_l2(to_host(base), want + 1.0) < TOL


@pytest.mark.parametrize("name", ["fan2d_ragged", "fan2d_c2_128"])
def test_tile_transpose_deterministic(psps, name):
    """The 2-D tile transpose sums in fixed point (exact integer adds), so two
    runs, and the accumulate mode on a zero image, are bitwise equal."""
    g = small_geoms()[name]
    rng = np.random.default_rng(15)
    s = to_dev(rng.standard_normal((3, g.n_rays)) * rng.uniform(0.01, 100.0, (3, 1)))
    plan = psps.Plan(g)
    a = to_host(psps.mbir_backproject(plan, s))
    b = to_host(psps.mbir_backproject(plan, s))
    assert np.array_equal(a, b)
    import torch
    z = torch.zeros((3,) + g.image_shape, device="cuda", dtype=torch.float32)
    c = to_host(psps.mbir_backproject(plan, s, z, accumulate=True))
    assert np.array_equal(a, c)


def test_tile_transpose_nonfinite_input(psps):
    """A NaN in a sinogram channel makes that channel's image NaN (the
    fixed-point scale cannot be formed) and leaves the other channels alone."""
    g = small_geoms()["par2d_ragged"]
    s = np.random.default_rng(16).random((2, g.n_rays))
    plan = psps.Plan(g)
    ref = to_host(psps.mbir_backproject(plan, to_dev(s)))
    s[1, 7] = np.nan
    got = to_host(psps.mbir_backproject(plan, to_dev(s)))
    assert np.array_equal(got[0], ref[0])
    assert np.isnan(got[1]).all()


@pytest.mark.parametrize("name", list(cone_geoms()) + ["c5_64"])
def test_cone_gather_deterministic(psps, name):
    """The 3-D gathers have no atomics: two runs are bitwise equal, and the
    split-table gather equals the direct gather bit for bit (same candidates,
    weights and summation order), 1, 2 and 4 channels."""
    g = cone_geoms()[name] if name != "c5_64" else synth.config5(n=64, n_views=90, n_u=128, n_v=96,
                                                                     rays=False).geom
    plan = psps.Plan(g)
    plan.set_backprojector("split")
    direct = psps.Plan(g)
    direct.set_backprojector("gather")
    for nch in [1, 2, 4]:
        s = to_dev(np.random.default_rng(14).standard_normal((nch, g.n_rays)))
        a = to_host(psps.mbir_backproject(plan, s))
        b = to_host(psps.mbir_backproject(plan, s))
        assert np.array_equal(a, b)
        assert np.array_equal(a, to_host(psps.mbir_backproject(direct, s))), nch


@pytest.mark.parametrize("depth", [16, 8])
@pytest.mark.parametrize("name", list(cone_geoms()) + ["c5_64"])
def test_cone_tile_fixed_point(psps, oracle_lib, name, depth):
    """The 3-D tile transpose sums in fixed point: two runs, and the
    accumulate mode on a zero image, are bitwise equal.  Signed data (the
    worst case: the sums cancel) spanning four decades across channels: the
    relative L2 error against the oracle stays within the projector's 1e-5,
    and the largest element-wise difference from the FP32 voxel gather (the
    same weights) within 3e-6 of the largest |A^T s| -- each term carries at
    most half a unit of M 2^-22 (M = max |w s|; about 1e-6 expected at the
    largest of these sums' independent roundings)."""
    import torch
    g = cone_geoms()[name] if name != "c5_64" else synth.config5(n=64, n_views=90, n_u=128, n_v=96,
                                                                     rays=False).geom
    rng = np.random.default_rng(18)
    plan = psps.Plan(g)
    assert plan.tuning()["backproject_mode"] == 0 and plan.tuning()["cone_tile"] == 16
    plan.set_cone_tile(depth)
    s = rng.standard_normal((5, g.n_rays)) * np.array([1.0, 1e-2, 1e2, 3.0, 0.5])[:, None]
    a = to_host(psps.mbir_backproject(plan, to_dev(s)))
    b = to_host(psps.mbir_backproject(plan, to_dev(s)))
    assert np.array_equal(a, b)
    z = torch.zeros((5,) + g.image_shape, device="cuda", dtype=torch.float32)
    assert np.array_equal(a, to_host(psps.mbir_backproject(plan, to_dev(s), z, accumulate=True)))
    want = oracle_lib.Projector(g).backproject(s)
    gather = psps.Plan(g)
    gather.set_backprojector("gather")
    ref = to_host(psps.mbir_backproject(gather, to_dev(s)))
    for c in range(5):
        assert rel_l2(a[c], want[c]) < TOL, (c, rel_l2(a[c], want[c]))
        err = float(np.abs(a[c] - ref[c]).max())
        assert err <= 3e-6 * float(np.abs(ref[c]).max()), (c, err / float(np.abs(ref[c]).max()))


def test_cone_tile_nonfinite_input(psps):
    """A NaN in a channel makes that channel's image NaN (its fixed-point
    scale cannot be formed); the other channels are unchanged."""
    g = cone_geoms()["cone_ragged"]
    s = np.random.default_rng(19).random((2, g.n_rays))
    plan = psps.Plan(g)
    ref = to_host(psps.mbir_backproject(plan, to_dev(s)))
    s[1, 11] = np.nan
    got = to_host(psps.mbir_backproject(plan, to_dev(s)))
    assert np.array_equal(got[0], ref[0])
    assert np.isnan(got[1]).all()


def test_cone_full_size_sampled(psps, oracle_lib):
    """256^3 volume, 360 views x 384 x 512 flat detector: sampled rays against
    the oracle ray by ray, and the adjoint identity at full size."""
    prob = synth.config5(rays=False)
    g = prob.geom
    plan = psps.Plan(g)
    x = prob.truth[:1]
    got = to_host(psps.mbir_project(plan, to_dev(x)))[0]
    rays = np.unique(np.concatenate([np.arange(0, g.n_rays, 70001), [g.n_rays - 1, g.n_rays // 2 + 255]]))
    want = oracle_lib.Projector(g).project_rays(x[0], rays)
    assert rel_l2(got[rays], want) < TOL, rel_l2(got[rays], want)
    rng = np.random.default_rng(13)
    y = rng.random((1, g.n_rays)).astype(np.float32)
    Aty = to_host(psps.mbir_backproject(plan, to_dev(y)))
    lhs, rhs = float(np.dot(got.astype(np.float64), y[0].astype(np.float64))), float(np.sum(x * Aty))
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


def test_autotune_keeps_parity(psps, oracle_lib):
    """The autotuner picks one of its candidate view splits that exist for the
    scan (47 views: 4 .. 45) and the transpose stays exact."""
    g = small_geoms()["fan2d_ragged"]
    plan = psps.Plan(g)
    v = plan.autotune(2)
    assert v in (4, 8, 15, 30, 45)
    t = plan.tuning()
    assert t["views_per_cta"] == v and t["forward"] in ("ray", "strip") and t["strip_bins"] in (32, 64, 128, 256)
    s = np.random.default_rng(11).random((2, g.n_rays))
    got = to_host(psps.mbir_backproject(plan, to_dev(s)))
    assert rel_l2(got, oracle_lib.Projector(g).backproject(s)) < TOL
    x = phantom(g, seed=4, nm=2)
    assert rel_l2(to_host(psps.mbir_project(plan, to_dev(x))), oracle_lib.Projector(g).project(x)) < TOL
    with pytest.raises(RuntimeError):
        plan.autotune(0)


@pytest.mark.parametrize("sb", [32, 64, 128, 256])
def test_strip_forward_shapes(psps, oracle_lib, sb):
    """Every CTA shape of the strip forward (sb bins x 256 / sb views) gives
    the same projection (within FP32) as the oracle, ragged sizes included."""
    for name in ["par2d_ragged", "fan2d_ragged", "fan2d_c2_128"]:
        g = small_geoms()[name]
        plan = psps.Plan(g)
        plan.set_projector("strip")
        plan.set_strip_bins(sb)
        x = phantom(g, seed=5, nm=3)
        assert rel_l2(to_host(psps.mbir_project(plan, to_dev(x))), oracle_lib.Projector(g).project(x)) < TOL


def test_autotune_cone(psps, oracle_lib):
    """Cone plans: the autotuner picks the tile scatter or one of the two
    gathers, and the transpose stays exact."""
    g = cone_geoms()["cone_ragged"]
    plan = psps.Plan(g)
    plan.autotune(4)
    assert plan.tuning()["backproject_mode"] in (0, 1, 3) and plan.tuning()["cone_tile"] in (8, 16)
    with pytest.raises(RuntimeError):
        plan.set_cone_tile(12)
    with pytest.raises(RuntimeError):
        psps.Plan(small_geoms()["fan2d_ragged"]).set_cone_tile(8)
    s = np.random.default_rng(17).random((4, g.n_rays))
    assert rel_l2(to_host(psps.mbir_backproject(plan, to_dev(s))), oracle_lib.Projector(g).backproject(s)) < TOL


def test_degenerate_geometries(psps, oracle_lib):
    """One view of one bin, a single-pixel image and a one-column image:
    forward and transpose against the oracle in every transpose mode."""
    cases = [
        Geometry(PAR2D, 9, 7, 1, 1.0, 1.0, 1.0, 1, 0.3, math.pi, 1, 1, 1.0, 1.0),
        Geometry(PAR2D, 1, 1, 1, 1.0, 1.0, 1.0, 5, 0.0, math.pi, 3, 1, 0.7, 1.0),
        Geometry(FAN2D, 1, 16, 1, 1.0, 1.0, 1.0, 7, 0.1, 2 * math.pi, 11, 1, 1.0, 1.0, 60.0, 120.0),
    ]
    for g in cases:
        x = phantom(g, seed=5, nm=1) + 0.1
        A = oracle_lib.Projector(g)
        for mode in ["tile", "ray"]:
            plan = psps.Plan(g)
            plan.set_projector(mode)
            assert rel_l2(to_host(psps.mbir_project(plan, to_dev(x))), A.project(x)) < TOL
        s = np.random.default_rng(6).random((2, g.n_rays))
        for mode in ["tile", "gather", "atomic"]:
            plan = psps.Plan(g)
            plan.set_backprojector(mode)
            assert rel_l2(to_host(psps.mbir_backproject(plan, to_dev(s))), A.backproject(s)) < TOL, (g, mode)


def test_fixed_point_transpose_numerators_full_size(psps, oracle_lib, error_log):
    """The tile transpose's 32-bit fixed-point sums on the real numerators of
    the 512^2 / 720 x 888 fan-beam workload (gradient g and curvature kappa
    of Eqs. 5, 8-11, from the data at x = 0 and at an iterate), element by
    element against the FP64 oracle transpose.

    Bound: every sample's value v = w_i s_i is rounded to the grid
    u = M max(2^-22, T 2^-30), M = w_max max|s| (T = views per CTA x the
    rays of one view that can reach one accumulator), as the two terms
    round(f v) and round(v) - round(f v), so each term errs by at most u;
    pixel j receives at most N = n_views x cell_rays terms, and the final
    conversion to FP32 rounds once more: |error_j| <= N u + 2^-24 |x_j|.  Pixels whose
    value is small against M carry a larger relative error; the max relative
    error over pixels above 1e-3 of the largest is recorded beside the FP32
    gather's."""
    import math as _m
    from oracle import model, psps as opsps, precond
    prob = synth.config2()
    g = prob.geom
    A = oracle_lib.Projector(g)
    st = opsps.Setup(A, prob.Q, prob.S, prob.y, prob.beta)
    xk, _ = opsps.run(st, precond.Identity(), 3, None)          # plain SPS iterate
    vs = 45
    pix = max(g.dx, g.dy)
    R = _m.hypot((0.5 * g.nx + 1.0) * g.dx, (0.5 * g.ny + 1.0) * g.dy)
    cell_rays = int(_m.floor(2.0 / ((g.sid - R) * (g.du / g.sdd) / pix))) + 2
    T = vs * cell_rays
    w_max = max(g.dx, g.dy) * _m.sqrt(2.0)
    n_terms = g.n_views * cell_rays
    plan = psps.Plan(g)
    plan.set_tiling(vs)
    gather = psps.Plan(g)
    gather.set_backprojector("gather")
    gamma = A.project(np.ones((1,) + g.image_shape))
    for label, x in [("x=0", st.zeros()), ("x=SPS iterate 3", xk)]:
        l = A.project(x)
        for name, s in [("g", model.data_grad_l(prob.Q, prob.S, l, prob.y)),
                        ("kappa", model.curvature_numerator(prob.Q, prob.S, l, prob.y, gamma))]:
            want = A.backproject(s)
            sf = np.asarray(s, dtype=np.float32)
            got = to_host(psps.mbir_backproject(plan, to_dev(sf)))
            ref = to_host(psps.mbir_backproject(gather, to_dev(sf)))
            M = w_max * float(np.abs(sf).max())
            u = M * max(2.0 ** -22, T * 2.0 ** -30)
            bound = n_terms * u + 2.0 ** -24 * np.abs(want)
            err = np.abs(got - want)
            assert np.all(err <= bound), (label, name, float(np.max(err / bound)))
            big = np.abs(want) >= 1e-3 * np.abs(want).max()
            rel = float(np.max(err[big] / np.abs(want[big])))
            rel_gather = float(np.max(np.abs(ref - want)[big] / np.abs(want[big])))
            error_log.add(f"fixed-point transpose c2 512 {label} {name}", "max |error| / (N u + 2^-24 |x|)",
                          float(np.max(err / bound)), 1.0, rel_above_floor=rel, rel_gather=rel_gather,
                          M_over_median=float(M / np.median(np.abs(sf[sf != 0]))))
            assert rel_l2(got, want) < TOL
