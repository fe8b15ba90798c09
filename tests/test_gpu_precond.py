"""GPU preconditioner builds and applies against the oracle's builds."""
import numpy as np
import pytest

import synth
from _helpers import rel_l2, to_dev, to_host

pytestmark = pytest.mark.gpu

TOL = 1e-4   # FP32 build (impulse responses, FFT) against the FP64 one


@pytest.fixture(scope="module")
def psps():
    import paper_2010_01371_gb300 as p
    p.lib()
    return p


def problems():
    return {"c1": synth.config1(), "c2_64": synth.config2(nx=64, n_views=90, n_u=111)}


@pytest.mark.parametrize("pname", ["c1", "c2_64"])
@pytest.mark.parametrize("kind", ["fourier", "mod_fourier", "haar", "block"])
def test_apply_parity(psps, oracle_lib, pname, kind):
    from oracle import build, psps as opsps
    prob = problems()[pname]
    st = opsps.Setup(oracle_lib.Projector(prob.geom), prob.Q, prob.S, prob.y, prob.beta)
    P = build.build(st, kind)
    plan = psps.Plan(prob.geom)
    spec = psps.Spectrum(prob.Q, prob.S)
    pc = psps.Precond(plan, spec, kind, to_dev(prob.y), prob.beta)
    rng = np.random.default_rng(3)
    v = rng.standard_normal((1,) + prob.geom.image_shape)
    for op, fn in [("M", P.M), ("MT", P.MT), ("absM", P.absM), ("absMT", P.absMT)]:
        got = to_host(psps.psps_precondition(pc, op, to_dev(v)))
        want = fn(v)
        assert rel_l2(got, want) < TOL, (op, rel_l2(got, want))


def test_projection_domain_block(psps, oracle_lib):
    from oracle import build, psps as opsps
    prob = synth.config3(n_views=10, n_u=333)
    st = opsps.Setup(oracle_lib.IdentityProjector(prob.n_rays), prob.Q, prob.S, prob.y, None)
    P = build.build(st, "block")
    spec = psps.Spectrum(prob.Q, prob.S)
    pc = psps.Precond(None, spec, "block", to_dev(prob.y))
    v = np.random.default_rng(4).standard_normal((2, prob.n_rays))
    for op, fn in [("M", P.M), ("MT", P.MT), ("absM", P.absM)]:
        assert rel_l2(to_host(psps.psps_precondition(pc, op, to_dev(v))), fn(v)) < 1e-5


def test_paper_single_test_function(psps, oracle_lib):
    """haar_lattice = 0 is Eq. 18 with the single test function U^T 1."""
    from oracle import build, precond, psps as opsps
    prob = problems()["c1"]
    st = opsps.Setup(oracle_lib.Projector(prob.geom), prob.Q, prob.S, prob.y, prob.beta)
    F = build.fisher(st)
    aH = build.make_apply_H(st, F)
    m0 = build.m0_blocks(st, F)[:, 0, 0].reshape(st.shape)
    lam = precond.haar_eigenvalues(lambda v: m0[None] * aH(m0[None] * v), st.shape, lattice=0)
    P = precond.Haar(lam, m0)
    plan, spec = psps.Plan(prob.geom), psps.Spectrum(prob.Q, prob.S)
    pc = psps.Precond(plan, spec, "haar", to_dev(prob.y), prob.beta, haar_lattice=0)
    v = np.random.default_rng(5).standard_normal((1,) + prob.geom.image_shape)
    assert rel_l2(to_host(psps.psps_precondition(pc, "M", to_dev(v))), P.M(v)) < TOL
