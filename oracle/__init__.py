"""FP64 CPU oracle for the preconditioned SPS hot path.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct
statement of what the GPU library computes: the Joseph projector (C, plain
loops), the polyenergetic forward model and PWLS objective (Eqs. 1-3), the SPS
update (Eqs. 4-11), the quadratic penalty (Eq. 26, Eqs. 49-52), the Fourier,
modified-Fourier, Haar, per-ray/per-pixel block and cross-material Fourier
preconditioners (Eqs. 17-18, 28-34, 42, 53-57), the cross-material wavelet
(Eqs. 58-61), the 2-D and 3-D Haar transforms, the detector blur in the outer
operator (B S, Eq. 1) and the preconditioned iteration (Sec. II-C).
It shares no code with the CUDA path and never imports it; only the tests,
the smoke check and the benchmark's CPU-baseline leg may use it.

Parity pins: every function here is checked in ``tests/test_oracle_*.py``
against closed forms, invariants and brute force (chord lengths, adjoint
identity, finite differences, circulant/Haar/block exactness, 8x8 brute-force
minimisers).  Whole-run iterate histories have no external pin beyond the
per-step pins: parity unpinned for 50/100-iteration trajectories as such.
"""
from .projector import IdentityProjector, Projector, build as build_c  # noqa: F401
from . import model, penalty, haar, precond, psps, build  # noqa: F401
