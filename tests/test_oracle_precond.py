"""Pins for the oracle Haar transform and preconditioners (CPU): exactness on
Hessians that are diagonal in the assumed basis, orthonormality, closed-form
block square roots and the elementwise bounds |M| that the separable
curvature relies on."""
import math

import numpy as np
import pytest

from synth import Geometry, PAR2D


def dense(op, shape, nm=1):
    n = nm * int(np.prod(shape))
    cols = []
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        cols.append(op(e.reshape((nm,) + tuple(shape))).ravel())
    return np.stack(cols, 1)


def even_positive(shape, rng, lo=0.5):
    G = rng.uniform(lo, 3.0, shape)
    Gr = G[tuple(np.meshgrid(*[(-np.arange(n)) % n for n in shape], indexing="ij"))]
    return 0.5 * (G + Gr)


def test_haar_orthonormal_and_abs():
    from oracle import haar
    shape = (8, 8)
    U = dense(lambda v: haar.forward(v[0])[None], shape)
    UT = dense(lambda v: haar.transpose(v[0])[None], shape)
    assert np.allclose(U @ U.T, np.eye(64), atol=1e-14)
    assert np.allclose(UT, U.T, atol=1e-15)
    Ua = dense(lambda v: haar.forward(v[0], absolute=True)[None], shape)
    UaT = dense(lambda v: haar.transpose(v[0], absolute=True)[None], shape)
    assert np.array_equal(Ua, np.abs(U))
    assert np.array_equal(UaT, np.abs(U).T)
    # the coarsest coefficient of an N x N image is its sum / N
    x = np.random.default_rng(0).random(shape)
    assert abs(haar.forward(x)[0, 0] - x.sum() / 8) < 1e-13


def test_inv_sqrt_2x2_closed_form():
    from oracle.precond import inv_sqrt_blocks
    rng = np.random.default_rng(1)
    B = rng.standard_normal((50, 2, 2))
    H = np.einsum("nij,nkj->nik", B, B) + 0.1 * np.eye(2)
    got = inv_sqrt_blocks(H, zero_rule=False)
    for h, g in zip(H, got):
        s = math.sqrt(np.linalg.det(h))
        t = math.sqrt(np.trace(h) + 2 * s)
        sq = (h + s * np.eye(2)) / t          # closed-form principal square root
        assert np.allclose(g, np.linalg.inv(sq), rtol=1e-12, atol=1e-13)


def test_fourier_exact_on_circulant():
    from oracle import precond
    shape = (12, 10)
    rng = np.random.default_rng(2)
    lam = even_positive(shape, rng)

    def apply_H(v):
        return np.stack([np.fft.ifftn(lam * np.fft.fftn(v[k])).real for k in range(v.shape[0])])
    est = precond.fourier_eigenvalues(apply_H, shape)
    assert np.allclose(est, lam, rtol=1e-12)
    P = precond.Fourier(est)
    v = rng.standard_normal((1,) + shape)
    assert np.allclose(P.MT(apply_H(P.M(v))), v, rtol=1e-11, atol=1e-11)
    # modified Fourier (Eq. 33) with Lambda~ the spectrum of N = M0 H M0.  When
    # N is circulant its estimate is exact: the one-sided M = M0 C whitens H,
    # the literal two-sided form gives M^T H M = M0 N^-1/2 N N^-1/2 M0 = M0^2.
    lamN = precond.fourier_eigenvalues(lambda z: 0.25 * apply_H(z), shape)
    P1 = precond.Fourier(lamN, np.full(shape, 0.5), sides=1)
    assert np.allclose(P1.MT(apply_H(P1.M(v))), v, rtol=1e-11, atol=1e-11)
    P2 = precond.Fourier(lamN, np.full(shape, 0.5))          # the literal form (default)
    assert np.allclose(P2.MT(apply_H(P2.M(v))), 0.25 * v, rtol=1e-11, atol=1e-11)


def _scaled(apply_N, m0):
    """H = M0^-1 N M0^-1 for a diagonal M0 (so that N = M0 H M0)."""
    return lambda v: apply_N(v / m0[None]) / m0[None]


def _scaled_blocks(apply_N, M0, nm):
    """H = M0^-1 N M0^-1 for symmetric per-pixel blocks M0."""
    Binv = np.linalg.inv(M0.B)
    inv = __import__("oracle").precond.Block(Binv, M0.shape)
    return lambda v: inv.M(apply_N(inv.M(v)))


@pytest.mark.parametrize("kind", ["mod_fourier", "haar"])
def test_one_sided_whitens_scaled_hessian(kind):
    """Where M0 goes (Eqs. 33, 34): with N = M0 H M0 diagonal in the
    transform basis and a non-constant M0, Eq. 18 recovers N's spectrum, the
    one-sided M = M0 C gives M^T H M = I and M M^T = H^-1 (dense), and the
    literal two-sided M0 C M0 (the one-material default) gives
    M^T H M = M0^2, a diagonal remainder."""
    from oracle import haar, precond
    shape = (8, 8)
    rng = np.random.default_rng(11)
    m0 = rng.uniform(0.3, 2.0, shape)
    if kind == "haar":
        lam = rng.uniform(0.2, 5.0, shape)

        def apply_N(v):
            return np.stack([haar.transpose(lam * haar.forward(v[k])) for k in range(v.shape[0])])
        est = precond.haar_eigenvalues(apply_N, shape)
        make = precond.Haar
    else:
        lam = even_positive(shape, rng)

        def apply_N(v):
            return np.stack([np.fft.ifftn(lam * np.fft.fftn(v[k])).real for k in range(v.shape[0])])
        est = precond.fourier_eigenvalues(apply_N, shape)
        make = precond.Fourier
    assert np.allclose(est, lam, rtol=1e-12)
    apply_H = _scaled(apply_N, m0)
    Hd = dense(apply_H, shape)
    P1, P2 = make(est, m0, sides=1), make(est, m0, sides=2)
    M1, M2 = dense(P1.M, shape), dense(P2.M, shape)
    assert np.allclose(dense(P1.MT, shape), M1.T, atol=1e-13)
    assert np.allclose(M1.T @ Hd @ M1, np.eye(64), atol=1e-10)
    assert np.allclose(M1 @ M1.T, np.linalg.inv(Hd), rtol=1e-9, atol=1e-9 * np.abs(np.linalg.inv(Hd)).max())
    assert np.allclose(M2.T @ Hd @ M2, np.diag(m0.ravel() ** 2), atol=1e-10)
    # |M| bounds M elementwise in both forms
    for P, Md in [(P1, M1), (P2, M2)]:
        assert (dense(P.absM, shape) >= np.abs(Md) - 1e-12).all()
        assert np.allclose(dense(P.absMT, shape), dense(P.absM, shape).T, atol=1e-12)


@pytest.mark.parametrize("kind", ["block_fourier", "block_haar"])
def test_one_sided_cross_material_whitens(kind):
    """Cross-material forms (Eqs. 57, 61) with symmetric per-pixel blocks M0:
    H = M0^-1 N M0^-1 with N block diagonal in the transform basis; the
    estimators recover N's blocks and the one-sided M = M0 C whitens H, the
    two-sided M0 C M0 gives M^T H M = M0^2."""
    from oracle import haar, precond
    shape, nm = (8, 4), 2
    if kind == "block_haar":
        shape = (8, 8)
    rng = np.random.default_rng(12)
    n = int(np.prod(shape))
    G = rng.standard_normal((n, nm, nm))
    B = np.einsum("nij,nkj->nik", G, G) + 0.5 * np.eye(nm)       # symmetric positive blocks
    M0 = precond.Block(B, shape)
    if kind == "block_haar":
        Gk = rng.standard_normal(shape + (nm, nm))
        Kt = np.einsum("...ij,...kj->...ik", Gk, Gk) + 0.5 * np.eye(nm)

        def apply_N(v):
            c = np.stack([haar.forward(v[k]) for k in range(nm)])
            out = np.einsum("...ij,j...->i...", Kt, c)
            return np.stack([haar.transpose(out[k]) for k in range(nm)])
        apply_H = _scaled_blocks(apply_N, M0, nm)
        est = precond.cross_haar_blocks(apply_H, M0, shape, nm)
        assert np.allclose(est, Kt, rtol=1e-9, atol=1e-9)
        P1, P2 = precond.CrossHaar(est, M0, sides=1), precond.CrossHaar(est, M0, sides=2)
    else:
        Gf = rng.standard_normal(shape + (nm, nm))
        idx = tuple(np.meshgrid(*[(-np.arange(k)) % k for k in shape], indexing="ij"))
        Gf = 0.5 * (Gf + Gf[idx])
        Lb = np.einsum("...ij,...kj->...ik", Gf, Gf) + 0.5 * np.eye(nm)

        def apply_N(v):
            V = np.fft.fftn(v, axes=(1, 2))
            return np.fft.ifftn(np.einsum("...ij,j...->i...", Lb, V), axes=(1, 2)).real
        apply_H = _scaled_blocks(apply_N, M0, nm)
        est = precond.cross_fourier_blocks(apply_H, M0, shape, nm)
        assert np.allclose(est, Lb, rtol=1e-9, atol=1e-9)
        P1, P2 = precond.CrossFourier(est, M0, sides=1), precond.CrossFourier(est, M0, sides=2)
    Hd = dense(apply_H, shape, nm)
    M1, M2 = dense(P1.M, shape, nm), dense(P2.M, shape, nm)
    assert np.allclose(dense(P1.MT, shape, nm), M1.T, atol=1e-12 * np.abs(M1).max())
    assert np.allclose(M1.T @ Hd @ M1, np.eye(nm * n), atol=1e-9)
    B2 = dense(lambda v: M0.M(M0.M(v)), shape, nm)
    assert np.allclose(M2.T @ Hd @ M2, B2, atol=1e-9 * np.abs(B2).max())
    for P, Md in [(P1, M1), (P2, M2)]:
        assert (dense(P.absM, shape, nm) >= np.abs(Md) - 1e-12 * np.abs(Md).max()).all()


@pytest.mark.parametrize("lattice", [0, 3])
def test_haar_exact_on_wavelet_diagonal(lattice):
    from oracle import haar, precond
    shape = (16, 16)
    rng = np.random.default_rng(3)
    lam = rng.uniform(0.2, 5.0, shape)

    def apply_H(v):
        return np.stack([haar.transpose(lam * haar.forward(v[k])) for k in range(v.shape[0])])
    est = precond.haar_eigenvalues(apply_H, shape, lattice=lattice)
    assert np.allclose(est, lam, rtol=1e-12)
    P = precond.Haar(est)
    v = rng.standard_normal((1,) + shape)
    assert np.allclose(P.MT(apply_H(P.M(v))), v, rtol=1e-11, atol=1e-11)


def test_haar_test_sets_partition():
    from oracle.precond import haar_test_sets
    for shape in [(16, 16), (64, 64), (8, 8)]:
        cnt = np.zeros(shape, int)
        for s in haar_test_sets(shape, 3):
            cnt += s
        assert (cnt == 1).all()


def test_block_exact_without_coupling(oracle_lib):
    """A = I (projection domain), R = 0: the per-ray blocks are the whole
    Hessian, so M0^T H M0 = I for every ray."""
    from oracle import build, model, psps
    rng = np.random.default_rng(4)
    E = np.arange(20.0, 81.0)
    import synth
    Q = synth.material_Q(E, ["water", "bone"], rng)
    S = np.stack([1e5 * synth.kramers(E, 60.0), 1e5 * synth.kramers(E, 80.0)])
    l = np.stack([rng.uniform(0, 200, 30), rng.uniform(0, 20, 30)])
    y = rng.poisson(model.forward_model(Q, S, l)).astype(float)
    st = psps.Setup(oracle_lib.IdentityProjector(30), Q, S, y, None)
    P = build.build(st, "block")
    F = build.fisher(st)
    for i in range(30):
        B = P.B[i]
        assert np.allclose(B.T @ F[i] @ B, np.eye(2), atol=1e-9)


def test_cross_fourier_exact_on_block_circulant():
    from oracle import precond
    shape = (8, 6)
    nm = 3
    rng = np.random.default_rng(5)
    G = rng.standard_normal(shape + (nm, nm))
    idx = tuple(np.meshgrid(*[(-np.arange(n)) % n for n in shape], indexing="ij"))
    G = 0.5 * (G + G[idx])
    Lb = np.einsum("...ij,...kj->...ik", G, G) + 0.5 * np.eye(nm)

    def apply_H(v):
        V = np.fft.fftn(v, axes=(1, 2))
        return np.fft.ifftn(np.einsum("...ij,j...->i...", Lb, V), axes=(1, 2)).real
    M0 = precond.Block(np.tile(np.eye(nm), (int(np.prod(shape)), 1, 1)), shape)
    L = precond.cross_fourier_blocks(apply_H, M0, shape, nm)
    assert np.allclose(L, Lb, rtol=1e-11, atol=1e-11)
    P = precond.CrossFourier(L, M0)
    v = rng.standard_normal((nm,) + shape)
    assert np.allclose(P.MT(apply_H(P.M(v))), v, rtol=1e-10, atol=1e-10)


def test_abs_bounds_dominate(oracle_lib):
    """|M| >= |M_ij| elementwise (dense, tiny grid) for every preconditioner
    built on a real projector-based Hessian."""
    import synth
    from oracle import build, psps
    g = Geometry(PAR2D, 8, 8, 1, 1.0, 1.0, 1.0, 12, 0.0, math.pi, 13, 1, 1.0, 1.0)
    A = oracle_lib.Projector(g)
    img = synth.render(g, [synth.Ellipse(0.5, -0.3, 2.5, 3.0, 0.2, 0.02)])
    y = np.round(1e4 * np.exp(-A.project(img[None])))
    st = psps.Setup(A, np.ones((1, 1)), np.full((1, 1), 1e4), y, np.array([[50.0]]))
    for kind, sides in [(k, sd) for k in ["fourier", "mod_fourier", "haar", "block", "block_haar"] for sd in (1, 2)]:
        P = build.build(st, kind, sides)
        Md = dense(P.M, st.shape)
        MTd = dense(P.MT, st.shape)
        Ad = dense(P.absM, st.shape)
        ATd = dense(P.absMT, st.shape)
        assert np.allclose(MTd, Md.T, atol=1e-12 * np.abs(Md).max())
        assert (Ad >= np.abs(Md) - 1e-12 * np.abs(Md).max()).all(), kind
        assert np.allclose(ATd, Ad.T, atol=1e-12 * np.abs(Ad).max())


def test_cross_haar_exact_on_wavelet_block_diagonal():
    """H = U^T K U per material with SPD cross-material blocks K (one per Haar
    coefficient), M0 = I: the estimator of Eqs. 59-60 recovers K exactly and
    the cross-material wavelet M of Eq. 61 whitens H (M^T H M = I)."""
    from oracle import haar, precond
    shape, nm = (8, 8), 3
    rng = np.random.default_rng(6)
    G = rng.standard_normal(shape + (nm, nm))
    Kt = np.einsum("...ij,...kj->...ik", G, G) + 0.5 * np.eye(nm)

    def apply_H(v):
        c = np.stack([haar.forward(v[k]) for k in range(nm)])
        out = np.einsum("...ij,j...->i...", Kt, c)
        return np.stack([haar.transpose(out[k]) for k in range(nm)])
    M0 = precond.Block(np.tile(np.eye(nm), (int(np.prod(shape)), 1, 1)), shape)
    K = precond.cross_haar_blocks(apply_H, M0, shape, nm)
    assert np.allclose(K, Kt, rtol=1e-11, atol=1e-11)
    P = precond.CrossHaar(K, M0)
    v = rng.standard_normal((nm,) + shape)
    assert np.allclose(P.MT(apply_H(P.M(v))), v, rtol=1e-10, atol=1e-10)
    # M^T is the transpose of M, and |M| dominates M elementwise
    Md = dense(P.M, shape, nm)
    assert np.allclose(dense(P.MT, shape, nm), Md.T, atol=1e-12 * np.abs(Md).max())
    assert (dense(P.absM, shape, nm) >= np.abs(Md) - 1e-12 * np.abs(Md).max()).all()


def test_cross_haar_one_material_is_haar(oracle_lib):
    """With one material the cross-material wavelet preconditioner is the Haar
    preconditioner of Eq. 34 (same test functions, modulus, floor and M0)."""
    import synth
    from oracle import build, psps
    g = Geometry(PAR2D, 16, 16, 1, 1.0, 1.0, 1.0, 24, 0.0, math.pi, 25, 1, 1.0, 1.0)
    A = oracle_lib.Projector(g)
    img = synth.render(g, [synth.Ellipse(0.5, -0.3, 5.0, 6.0, 0.2, 0.02)])
    y = np.round(1e4 * np.exp(-A.project(img[None])))
    st = psps.Setup(A, np.ones((1, 1)), np.full((1, 1), 1e4), y, np.array([[50.0]]))
    v = np.random.default_rng(7).standard_normal((1,) + st.shape)
    for sides in (1, 2):
        Ph, Pc = build.build(st, "haar", sides), build.build(st, "block_haar", sides)
        for op in ["M", "MT", "absM", "absMT"]:
            a, b = getattr(Ph, op)(v), getattr(Pc, op)(v)
            assert np.allclose(a, b, rtol=1e-10, atol=1e-12 * np.abs(a).max()), (op, sides)


# ---------------------------------------------------------------------------
# 3-D Haar (volumes [z, y, x])
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("shape", [(4, 4, 4), (2, 4, 8)])
def test_haar3_orthonormal_and_abs(shape):
    from oracle import haar
    n = int(np.prod(shape))
    U = dense(lambda v: haar.forward(v[0])[None], shape)
    UT = dense(lambda v: haar.transpose(v[0])[None], shape)
    assert np.allclose(U @ U.T, np.eye(n), atol=1e-14)
    assert np.allclose(UT, U.T, atol=1e-15)
    Ua = dense(lambda v: haar.forward(v[0], absolute=True)[None], shape)
    UaT = dense(lambda v: haar.transpose(v[0], absolute=True)[None], shape)
    assert np.allclose(Ua, np.abs(U), atol=1e-15)
    assert np.allclose(UaT, np.abs(U).T, atol=1e-15)


def _haar1_pyramid(f, n_levels):
    """Textbook 1-D Haar, level by level: returns the (low, detail) pair of
    each level, low/detail = (f[2i] +- f[2i+1]) / sqrt(2) of the previous low."""
    out, low = [], np.asarray(f, dtype=np.float64)
    for _ in range(n_levels):
        lo = (low[0::2] + low[1::2]) / math.sqrt(2.0)
        hi = (low[0::2] - low[1::2]) / math.sqrt(2.0)
        out.append((lo, hi))
        low = lo
    return out


def test_haar3_separable_volume():
    """A separable volume f(z) g(y) h(x): every 3-D Haar coefficient is the
    product of the three 1-D Haar coefficients of the same level (a detail
    octant takes the detail part along the axes where its index bit is 1),
    and the last low-pass value is the product of the three last lows."""
    from oracle import haar
    rng = np.random.default_rng(11)
    f, g, h = rng.standard_normal(8), rng.standard_normal(8), rng.standard_normal(8)
    vol = np.einsum("i,j,k->ijk", f, g, h)
    c = haar.forward(vol)
    pf, pg, ph = (_haar1_pyramid(v, 3) for v in (f, g, h))
    n = 8
    for lev in range(3):
        n2 = n // 2
        for s in haar.OCTANTS[1:]:
            want = np.einsum("i,j,k->ijk", pf[lev][s[0]], pg[lev][s[1]], ph[lev][s[2]])
            got = c[s[0] * n2:(s[0] + 1) * n2, s[1] * n2:(s[1] + 1) * n2, s[2] * n2:(s[2] + 1) * n2]
            assert np.allclose(got, want, atol=1e-13), (lev, s)
        n = n2
    assert abs(c[0, 0, 0] - pf[2][0][0] * pg[2][0][0] * ph[2][0][0]) < 1e-13


def test_haar3_test_sets_partition():
    from oracle.precond import haar_test_sets
    for shape in [(8, 8, 8), (16, 16, 16), (4, 8, 8)]:
        cnt = np.zeros(shape, int)
        for s in haar_test_sets(shape, 3):
            cnt += s
        assert (cnt == 1).all(), shape


@pytest.mark.parametrize("lattice", [0, 2, 3])
def test_haar3_exact_on_wavelet_diagonal(lattice):
    from oracle import haar, precond
    shape = (8, 8, 8)
    rng = np.random.default_rng(12)
    lam = rng.uniform(0.2, 5.0, shape)

    def apply_H(v):
        return np.stack([haar.transpose(lam * haar.forward(v[k])) for k in range(v.shape[0])])
    est = precond.haar_eigenvalues(apply_H, shape, lattice=lattice)
    assert np.allclose(est, lam, rtol=1e-12)
    P = precond.Haar(est)
    v = rng.standard_normal((1,) + shape)
    assert np.allclose(P.MT(apply_H(P.M(v))), v, rtol=1e-11, atol=1e-11)


def test_cross_haar3_exact_on_wavelet_block_diagonal():
    from oracle import haar, precond
    shape, nm = (4, 4, 4), 2
    rng = np.random.default_rng(13)
    G = rng.standard_normal(shape + (nm, nm))
    Kt = np.einsum("...ij,...kj->...ik", G, G) + 0.5 * np.eye(nm)

    def apply_H(v):
        c = np.stack([haar.forward(v[k]) for k in range(nm)])
        out = np.einsum("...ij,j...->i...", Kt, c)
        return np.stack([haar.transpose(out[k]) for k in range(nm)])
    M0 = precond.Block(np.tile(np.eye(nm), (int(np.prod(shape)), 1, 1)), shape)
    K = precond.cross_haar_blocks(apply_H, M0, shape, nm)
    assert np.allclose(K, Kt, rtol=1e-11, atol=1e-11)
    P = precond.CrossHaar(K, M0)
    v = rng.standard_normal((nm,) + shape)
    assert np.allclose(P.MT(apply_H(P.M(v))), v, rtol=1e-10, atol=1e-10)
    Md = dense(P.M, shape, nm)
    assert np.allclose(dense(P.MT, shape, nm), Md.T, atol=1e-12 * np.abs(Md).max())
    assert (dense(P.absM, shape, nm) >= np.abs(Md) - 1e-12 * np.abs(Md).max()).all()


def test_abs_bounds_dominate_3d(oracle_lib):
    """|M| >= |M_ij| for the Haar kinds on a tiny cone-beam volume."""
    import synth
    from oracle import build, psps
    g = Geometry(synth.CONE3D, 4, 4, 4, 1.0, 1.0, 1.0, 8, 0.0, 2 * math.pi, 8, 8, 1.5, 1.5, 20.0, 40.0)
    A = oracle_lib.Projector(g)
    img = synth.render(g, [synth.Ellipsoid(0.3, -0.2, 0.1, 1.5, 1.2, 1.4, 0.2, 0.02)])
    y = np.round(1e4 * np.exp(-A.project(img[None])))
    st = psps.Setup(A, np.ones((1, 1)), np.full((1, 1), 1e4), y, np.array([[50.0]]))
    for kind in ["haar", "block_haar"]:
        P = build.build(st, kind)
        Md = dense(P.M, st.shape)
        Ad = dense(P.absM, st.shape)
        assert np.allclose(dense(P.MT, st.shape), Md.T, atol=1e-12 * np.abs(Md).max())
        assert (Ad >= np.abs(Md) - 1e-12 * np.abs(Md).max()).all(), kind


def test_haar_eigenvalue_parts_add_up():
    """Splitting the Haar test sets among processes (part = (i, n)) gives
    the whole estimate once the parts are added."""
    from oracle import haar, precond
    shape = (16, 16)
    rng = np.random.default_rng(13)
    A = rng.standard_normal((256, 256))
    Hd = A @ A.T + 256 * np.eye(256)

    def apply_H(v):
        return (Hd @ v.reshape(v.shape[0], -1).T).T.reshape(v.shape)
    whole = precond.haar_eigenvalues(apply_H, shape)
    parts = sum(precond.haar_eigenvalues(apply_H, shape, part=(i, 3)) for i in range(3))
    assert np.array_equal(parts, whole)
