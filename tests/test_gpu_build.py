"""GPU preconditioner builds against the FP64 oracle build, element by
element, for every kind.

What is compared (``psps_precondition_export``):
* the blocks (F+R)1_k whose inverse square roots are M0 (Eqs. 30, 53-54),
* the Eq. 18 estimates (Fourier / Haar eigenvalues, cross-material polar
  factors or wavelet blocks) before the floor and the -1/2 power,
* the arrays the apply uses: M0, the scales clamp(Lambda~)^-1/2 and the
  cross-material blocks L^-1/2, K^-1/2.

Error model (first order).  The GPU applies the Hessian in FP32: sample
positions along a ray are formed as start + i * slope in pixel units, so each
interpolation weight carries an absolute error of a few ulp(n) ~ n 2^-24 for
an n-pixel grid, in the projection and again in the transpose; products and
(compensated) sums add O(2^-24) relative error each.  The computed operator
is therefore N + dN with ||dN|| <= eps_b ||N||, eps_b = C n 2^-24 (C = 8: two
passes of a few roundings each, plus the FP32 FFT / Haar of the estimate).
By Weyl's theorem an eigenvalue estimate moves by at most eps_b lambda_max,
so small eigenvalues carry relative error eps_b lambda_max / lambda_k: the
elementwise bound is
    |d lambda_k| <= eps_b max|lambda| + 2^-22 |lambda_k|,
and through the clamp and the -1/2 power (derivative -1/2 t^-3/2; for a
matrix argument the Frechet derivative of t^-1/2 is bounded by
1/2 lambda_min^-3/2 in the Frobenius norm)
    |d s_k| / s_k <= 1/2 (eps_b max|lambda| / lambda_eff,k) + 2^-22,
    ||d M0_j||_F  <= lambda_eff,j^-3/2 eps_b ||H~_j||_F + 2^-22 ||M0_j||_F
with lambda_eff the eigenvalue after the 1e-6 floor (a factor 2 of margin
for second-order terms is included in the last line).  For the projection
domain (A = I) there is no geometry: eps_b = C 2^-24.
The measured errors, their bounds and the ratio are recorded in the session
error log (PSPS_ERROR_LOG).
"""
import numpy as np
import pytest

import synth
from _helpers import to_dev, to_host

pytestmark = pytest.mark.gpu

EPS32 = 2.0 ** -24
C_GEOM = 8.0
FLOOR = 1e-6     # eigenvalue floor of the builds (x the largest)


@pytest.fixture(scope="module")
def psps():
    import paper_2010_01371_gb300 as p
    p.lib()
    return p


def eps_b(prob, proj=True):
    if not proj:
        return C_GEOM * EPS32
    g = prob.geom
    return C_GEOM * max(g.nx, g.ny, getattr(g, "nz", 1)) * EPS32


def oracle_raw(oracle_lib, prob, kind, proj=True):
    """The oracle build's intermediate and final arrays, in [n, ...] layout:
    H~ blocks [n, nm, nm], the Eq. 18 estimate ([n] or [n, nm, nm]), M0
    blocks, and the scales ([n]) or cross-material blocks ([n, nm, nm])."""
    from oracle import build, precond, psps as opsps
    A = oracle_lib.Projector(prob.geom) if proj else oracle_lib.IdentityProjector(prob.n_rays)
    st = opsps.Setup(A, prob.Q, prob.S, prob.y, prob.beta if proj else None)
    F = build.fisher(st)
    aH = build.make_apply_H(st, F)
    nm = st.nm
    Ht = np.zeros((int(np.prod(st.shape)), nm, nm))
    for k in range(nm):
        one = np.zeros((nm,) + st.shape)
        one[k] = 1.0
        Ht[:, :, k] = aH(one).reshape(nm, -1).T
    B = precond.inv_sqrt_blocks(Ht, floor="block", zero_rule=True)
    out = {"st": st, "hblocks": Ht, "blocks": B}
    if kind in ("block", "fourier"):
        if kind == "fourier":
            lam = precond.fourier_eigenvalues(aH, st.shape)
            out["estimate"], out["scales"] = lam.ravel(), precond.Fourier(lam).s.ravel()
        return out
    M0 = precond.Block(B, st.shape)
    if kind == "block_fourier":
        L = precond.cross_fourier_blocks(aH, M0, st.shape, nm)
        P = precond.polar_real(L)
        out["estimate"] = P.reshape(-1, nm, nm)
        out["scales"] = precond.CrossFourier(L, M0).Li.reshape(-1, nm, nm)
        return out
    if kind == "block_haar":
        K = precond.cross_haar_blocks(aH, M0, st.shape, nm)
        out["estimate"] = K.reshape(-1, nm, nm)
        out["scales"] = precond.CrossHaar(K, M0).Ki.reshape(-1, nm, nm)
        return out
    m0 = B[:, 0, 0].reshape(st.shape)

    def aN(v):
        return m0[None] * aH(m0[None] * v)
    lam = (precond.fourier_eigenvalues(aN, st.shape) if kind == "mod_fourier"
           else precond.haar_eigenvalues(aN, st.shape))
    out["estimate"] = lam.ravel()
    out["scales"] = (1.0 / np.sqrt(precond.clamp_eigs(lam))).ravel()
    return out


def gpu_arrays(psps, pc, kind):
    """Exports in [n, ...] layout (the library stores blocks as [m][k][n])."""
    def blk(a):
        return np.transpose(to_host(a), (2, 0, 1))
    out = {"hblocks": blk(psps.psps_precondition_export(pc, "hblocks")),
           "blocks": blk(psps.psps_precondition_export(pc, "blocks"))}
    if kind == "block":
        return out
    est = psps.psps_precondition_export(pc, "estimate")
    sc = psps.psps_precondition_export(pc, "scales")
    if kind in ("block_fourier", "block_haar"):
        out["estimate"], out["scales"] = blk(est), blk(sc)
    else:
        out["estimate"], out["scales"] = np.abs(to_host(est)), to_host(sc)
    return out


def sym_eigs(Bl):
    return np.linalg.eigvalsh(0.5 * (Bl + np.swapaxes(Bl, -1, -2)))


def check_blocks(name, got, want, eps, error_log, what):
    """H~ blocks and M0 = H~^-1/2 against the Frechet bound."""
    Ht, Hg = want["hblocks"], got["hblocks"]
    nH = np.linalg.norm(Ht, axis=(1, 2))
    live = nH > 1e-10 * nH.max()
    dH = np.linalg.norm(Hg - Ht, axis=(1, 2))
    rH = float(np.max(dH[live] / (eps * nH[live])))
    error_log.add(name, f"{what} (F+R)1_k blocks", float(np.max(dH[live] / nH[live])), eps, ratio=rH)
    assert rH <= 1.0, ("hblocks", rH)
    lam = sym_eigs(Ht)
    lam_eff = np.maximum(lam[:, 0], FLOOR * lam[:, -1])
    B, Bg = want["blocks"], got["blocks"]
    nB = np.linalg.norm(B, axis=(1, 2))
    liveB = live & (nB > 0)
    dB = np.linalg.norm(Bg - B, axis=(1, 2))
    bound = lam_eff ** -1.5 * eps * nH + 4 * EPS32 * nB
    rB = float(np.max(dB[liveB] / bound[liveB]))
    error_log.add(name, f"{what} M0 blocks", float(np.max(dB[liveB] / nB[liveB])),
                  float(np.max(bound[liveB] / nB[liveB])), ratio=rB)
    assert rB <= 1.0, ("blocks", rB)
    # dead pixels (outside the field of view) are zero on both sides
    assert np.all(Bg[~live] == 0.0)


def check_scalar(name, got, want, eps, error_log):
    lam, lg = want["estimate"], got["estimate"]
    lmax = np.abs(lam).max()
    dl = np.abs(lg - lam)
    bound = eps * lmax + 4 * EPS32 * np.abs(lam)
    r = float(np.max(dl / bound))
    error_log.add(name, "eigenvalue estimates", float(np.max(dl / np.maximum(np.abs(lam), FLOOR * lmax))),
                  float(np.max(bound / np.maximum(np.abs(lam), FLOOR * lmax))), ratio=r)
    assert r <= 1.0, ("estimate", r)
    s, sg = want["scales"], got["scales"]
    lam_eff = np.maximum(np.abs(lam), FLOOR * lmax)
    bound_s = 0.5 * (eps * lmax / lam_eff) + 4 * EPS32
    ds = np.abs(sg - s) / s
    rs = float(np.max(ds / bound_s))
    error_log.add(name, "scales clamp(Lambda)^-1/2", float(np.max(ds)), float(np.max(bound_s)), ratio=rs,
                  l2=float(np.linalg.norm(sg - s) / np.linalg.norm(s)))
    assert rs <= 1.0, ("scales", rs)


def check_cross(name, got, want, eps, error_log):
    P, Pg = want["estimate"], got["estimate"]
    nP = np.linalg.norm(P, axis=(1, 2))
    pmax = nP.max()
    dP = np.linalg.norm(Pg - P, axis=(1, 2))
    bound = eps * pmax + 4 * EPS32 * nP
    r = float(np.max(dP / bound))
    error_log.add(name, "cross-material estimates", float(np.max(dP / np.maximum(nP, FLOOR * pmax))),
                  float(np.max(bound / np.maximum(nP, FLOOR * pmax))), ratio=r)
    assert r <= 1.0, ("estimate", r)
    Pp = want["estimate"]
    Psym = 0.5 * (Pp + np.swapaxes(Pp, -1, -2))
    if np.any(np.abs(Pp - np.swapaxes(Pp, -1, -2)) > 1e-9 * pmax):     # K blocks: the polar factor is used
        from oracle.precond import polar_real
        Psym = polar_real(Pp)
    lam = sym_eigs(Psym)
    lam_eff = np.maximum(lam[:, 0], FLOOR * np.abs(lam).max())
    L, Lg = want["scales"], got["scales"]
    nL = np.linalg.norm(L, axis=(1, 2))
    dL = np.linalg.norm(Lg - L, axis=(1, 2))
    # the polar factor moves by at most sqrt(2) times the block perturbation
    bound_L = lam_eff ** -1.5 * np.sqrt(2.0) * bound + 4 * EPS32 * nL
    rL = float(np.max(dL / bound_L))
    error_log.add(name, "cross-material blocks ^-1/2", float(np.max(dL / nL)), float(np.max(bound_L / nL)),
                  ratio=rL, l2=float(np.linalg.norm(Lg - L) / np.linalg.norm(L)))
    assert rL <= 1.0, ("scales", rL)


def cone_mbir_problem():
    g = synth.config5(n=32, n_views=24, n_u=64, n_v=48, rays=False).geom
    shapes = [synth.Ellipsoid(0.0, 0.0, 0.0, 50.0, 40.0, 45.0, 0.3, 0.02),
              synth.Ellipsoid(15.0, -10.0, 5.0, 12.0, 9.0, 10.0, 0.0, 0.01)]
    return synth.mbir_problem(5, g, shapes, 1e4, 1e3, 50, "fourier", "cone_mbir_32")


def mixed_radix_problem():
    import math
    g = synth.rng(1, "phantom")
    geom = synth.Geometry(synth.PAR2D, 45, 56, 1, 1.0, 1.0, 1.0, 60, 0.0, math.pi, 80, 1, 1.0, 1.0)
    shapes = synth.random_ellipses(g, 4, radius=20.0, amin=3.0, amax=12.0, vmin=0.01, vmax=0.03)
    return synth.mbir_problem(1, geom, shapes, 1e4, 1e3, 50, "fourier", "mixed_radix_45x56")


PROBLEMS = {
    "c1": lambda: synth.config1(),
    "c2_64": lambda: synth.config2(nx=64, n_views=90, n_u=111),
    "c2_128": lambda: synth.config2(nx=128, n_views=180, n_u=222),
    "c4_64": lambda: synth.config4_slice(nx=64, n_views=90, n_u=111),
    "c4_48": lambda: next(p for p in synth.config4(n_views=90, shrink=8) if p.geom.nx == 48),
    "mixed_45x56": mixed_radix_problem,
    "cone_32": cone_mbir_problem,
    "c5_32": lambda: synth.config5(n=32, n_views=24, n_u=64, n_v=48),
    "c5_16": lambda: synth.config5(n=16, n_views=12, n_u=32, n_v=24),
}

CASES = ([("c1", k) for k in ["fourier", "mod_fourier", "haar", "block"]]
         + [("c2_64", k) for k in ["fourier", "mod_fourier", "haar", "block"]]
         + [("c2_128", "haar"), ("c4_64", "block"), ("c4_64", "block_fourier"), ("c4_64", "block_haar"),
            ("c4_48", "block_fourier"), ("mixed_45x56", "fourier"), ("mixed_45x56", "mod_fourier"),
            ("cone_32", "fourier"), ("cone_32", "mod_fourier"), ("cone_32", "haar"), ("c5_32", "block"),
            ("c5_32", "block_fourier"), ("c5_16", "block_haar")])


@pytest.mark.parametrize("pname,kind", CASES, ids=[f"{p}-{k}" for p, k in CASES])
def test_build_elementwise(psps, oracle_lib, error_log, pname, kind):
    prob = PROBLEMS[pname]()
    want = oracle_raw(oracle_lib, prob, kind)
    plan, spec = psps.Plan(prob.geom), psps.Spectrum(prob.Q, prob.S)
    pc = psps.Precond(plan, spec, kind, to_dev(prob.y), prob.beta)
    got = gpu_arrays(psps, pc, kind)
    eps = eps_b(prob)
    name = f"build {pname} {kind}"
    check_blocks(name, got, want, eps, error_log, "")
    if kind in ("fourier", "mod_fourier", "haar"):
        check_scalar(name, got, want, eps, error_log)
    elif kind in ("block_fourier", "block_haar"):
        check_cross(name, got, want, eps, error_log)


def test_build_elementwise_projection_domain(psps, oracle_lib, error_log):
    """Per-ray 2x2 blocks (A = I): no geometry, the blocks are the Fisher
    blocks of the water fit, built in FP64 on the GPU and stored in FP32."""
    prob = synth.config3(n_views=10, n_u=333)
    want = oracle_raw(oracle_lib, prob, "block", proj=False)
    spec = psps.Spectrum(prob.Q, prob.S)
    pc = psps.Precond(None, spec, "block", to_dev(prob.y))
    got = gpu_arrays(psps, pc, "block")
    check_blocks("build c3 block", got, want, eps_b(prob, proj=False), error_log, "")
