"""Derives the cross-material penalty strengths of the one-step MBMD workload
(``synth.CONFIG4_BETA``) with the oracle; run once, result rounded and
stored in ``synth``.

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.

The paper gives no beta values (Eqs. 49-52 only require beta_kk' > 0).  The
reading: beta_kk = 0.05 x mean_j(F_jj,kk) / (2 |N|) with F_jj,kk the diagonal
of the Fisher information (data approximated from y as in the preconditioner
build) averaged over four pixels of the 512^2 slice, |N| = 4, and
beta_kk' = 0.1 sqrt(beta_kk beta_k'k') for k != k' (positive definite).
"""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def main():
    import oracle
    import synth
    from oracle import build, psps
    p = synth.config4_slice()
    A = oracle.Projector(p.geom)
    st = psps.Setup(A, p.Q, p.S, p.y, None)
    F = build.fisher(st)
    diag = []
    for (iy, ix) in [(256, 256), (300, 200), (200, 330), (256, 150)]:
        img = np.zeros(p.geom.image_shape)
        img[iy, ix] = 1.0
        a = A.project(img[None])[0]
        diag.append(np.einsum("i,ikk->k", a * a, F))
    beta = 0.05 * np.mean(diag, 0) / (2 * 4)
    B = np.diag(beta)
    for i in range(3):
        for j in range(3):
            if i != j:
                B[i, j] = 0.1 * np.sqrt(beta[i] * beta[j])
    print(np.array2string(B, precision=4, separator=", "))


if __name__ == "__main__":
    main()
