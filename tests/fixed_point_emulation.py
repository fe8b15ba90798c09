"""How the 3-D tile transpose's fixed-point grid shows in one PSPS step.

CPU emulation with the oracle, on the 32^3 cone scan (24 views, 64 x 48
detector, 2 materials x 2 kVp) at x = 0: the exact step is compared with
the step taken from gradient and curvature numerators that carry the
rounding noise of a fixed-point grid of G = M_c * 2^-k per term, M_c the
largest |w s| of the channel.  Each voxel receives about N_j = 24 views x
6.25 rays (a voxel spans 1.25 detector cells at the isocentre, so about
2.5 x 2.5 rays reach it per view), each term rounded to the nearest grid
point: independent errors uniform on [-G/2, G/2], variance N_j G^2 / 12.
The ray weights are at most 1.05 voxel sides (the steepest rays of this
scan).

    python tests/fixed_point_emulation.py [kind ...]    (default: none block block_haar block_fourier)

prints, per preconditioner kind and grid, the relative L2 difference of the
step's image from the exact one.  The grid M 2^-22 is the coarse words'; the
low words of the gradient channels hold each term to 2^-12 of it.
"""
from __future__ import annotations

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

import synth  # noqa: E402
from oracle import model, projector, psps as opsps  # noqa: E402
from _helpers import oracle_precond  # noqa: E402


class _Lib:
    Projector = projector.Projector
    IdentityProjector = projector.IdentityProjector


def step_errors(kind: str, grids=(20, 22, 24), seed: int = 0) -> dict:
    prob = synth.config5(n=32, n_views=24, n_u=64, n_v=48)
    st, P, _ = oracle_precond(_Lib, prob, kind)
    Q, S, y, A = st.Q, st.S, st.y, st.proj
    x = st.zeros()
    l = A.project(x)
    absM1 = P.absM(np.ones_like(x))
    gamma_m = A.project(absM1)
    dR = P.absMT(st.pen.abs_apply(absM1))
    phi0 = model.data_objective(Q, S, l, y) + st.pen.value(x)
    g = model.data_grad_l(Q, S, l, y)
    kappa = model.curvature_numerator(Q, S, l, y, gamma_m)

    def step(grad, C):
        gp = P.MT(grad)
        dp = P.absMT(C) + dR
        pp = np.where(dp > 0, -gp / np.where(dp > 0, dp, 1.0), 0.0)
        p = P.M(pp)
        alpha, _, _ = opsps.line_search(st, x, p, l, A.project(p), phi0, opsps.LineSearch(), 1.0)
        return x + alpha * p

    grad0 = A.backproject(g) + st.pen.apply(x)
    C0 = A.backproject(kappa)
    x1 = step(grad0, C0)
    w_max = 1.05 * prob.geom.dx
    n_terms = 24 * 6.25
    rng = np.random.default_rng(seed)
    out = {}
    for k in grids:
        sd_g = np.sqrt(n_terms / 12) * np.abs(g).max(axis=1) * w_max * 2.0 ** -k
        sd_k = np.sqrt(n_terms / 12) * np.abs(kappa).max(axis=1) * w_max * 2.0 ** -k
        gn = grad0 + rng.standard_normal(grad0.shape) * sd_g[:, None, None, None]
        cn = C0 + rng.standard_normal(C0.shape) * sd_k[:, None, None, None]
        out[k] = float(np.linalg.norm(step(gn, cn) - x1) / np.linalg.norm(x1))
    return out


if __name__ == "__main__":
    for kind in sys.argv[1:] or ["none", "block", "block_haar", "block_fourier"]:
        errs = step_errors(kind)
        print(kind, "  ".join(f"grid M 2^-{k}: {e:.2e}" for k, e in errs.items()), flush=True)
