"""GB300 preconditioned SPS (PSPS) for PWLS CT reconstruction and model-based
material decomposition -- thin Python binding over the C ABI of
``libpsps.so`` (``include/mbir.h``).

PyTorch supplies device memory and the current CUDA stream; every step of the
computation runs in the library's CUDA kernels.  There is no CPU fallback:
importing works without a GPU, but every call needs the compiled library and
a CUDA device, and raises otherwise.

The function names mirror the C entry points (``mbir_project``,
``mbir_backproject``, ``mbmd_forward_model``, ``mbmd_objective``,
``mbmd_gradient``, ``psps_precondition``, ``psps_step``); handles are wrapped
by ``Plan``, ``Spectrum``, ``Precond`` and ``State``.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _abi
from ._abi import FLAG_GRAPH, FLAG_LINESEARCH, FLAG_NONNEG, MbirError, PSPS_APPLY, PSPS_PRECOND  # noqa: F401

__all__ = ["Plan", "Spectrum", "Precond", "State", "MbirError", "mbir_project", "mbir_backproject",
           "mbmd_forward_model", "mbmd_objective", "mbmd_gradient", "psps_precondition", "psps_step",
           "psps_get_image", "MBMDData", "lib"]


def lib():
    return _abi.load()


def _torch():
    import torch
    return torch


def _stream():
    torch = _torch()
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dev(t, name, dtype=None):
    torch = _torch()
    dtype = dtype or torch.float32
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _call(fn, *args):
    _abi.check(fn(*args))


class Plan:
    """Projector plan for one geometry (any object with the ``mbir_geometry``
    fields, e.g. ``synth.Geometry``)."""

    def __init__(self, geom, n_mat_max: int = 8):
        L = lib()
        g = _abi.MbirGeometry(int(geom.kind), int(geom.nx), int(geom.ny), int(getattr(geom, "nz", 1)),
                              float(geom.dx), float(geom.dy), float(getattr(geom, "dz", 1.0)), int(geom.n_views),
                              float(geom.angle0), float(geom.angle_span), int(geom.n_u), int(getattr(geom, "n_v", 1)),
                              float(geom.du), float(getattr(geom, "dv", 1.0)), float(getattr(geom, "sid", 0.0)),
                              float(getattr(geom, "sdd", 0.0)))
        h = ctypes.c_void_p()
        _call(L.mbir_plan_create, ctypes.byref(g), int(n_mat_max), ctypes.byref(h))
        self.h = h
        self.geom = geom
        self.n_mat_max = n_mat_max
        self.n_rays = int(L.mbir_plan_n_rays(h))
        self.n_pix = int(L.mbir_plan_n_pix(h))
        self.image_shape = tuple(geom.image_shape)
        self.sino_shape = tuple(geom.sino_shape)

    def set_backprojector(self, mode: str):
        """'tile' (default: fixed-point tile scatter, deterministic), 'gather'
        (pixel / voxel gather, FP32, deterministic), 'atomic' (ray-driven
        scatter with global atomics) or, for cone plans, 'split' (the voxel
        gather with split tables, bitwise equal to 'gather')."""
        _call(lib().mbir_plan_set_backprojector, self.h, {"tile": 0, "gather": 1, "atomic": 2, "split": 3}[mode])

    def set_tiling(self, views_per_cta: int):
        """Views per CTA of the 'tile' transpose (1..180)."""
        _call(lib().mbir_plan_set_tiling, self.h, int(views_per_cta))

    def autotune(self, n_channels: int = 2) -> int:
        """Time the tile transpose's view splits and keep the fastest
        (synchronises); returns the chosen views per CTA."""
        v = ctypes.c_int()
        _call(lib().mbir_plan_autotune, self.h, int(n_channels), _stream(), ctypes.byref(v))
        return int(v.value)

    def set_strip_bins(self, bins: int):
        """Bins per CTA of the strip forward (32, 64, 128, 256)."""
        _call(lib().mbir_plan_set_strip_bins, self.h, int(bins))

    def tuning(self) -> dict:
        """The plan's current choices (``mbir_plan_tuning``)."""
        v = [ctypes.c_int() for _ in range(5)]
        _call(lib().mbir_plan_tuning, self.h, *[ctypes.byref(x) for x in v])
        names = {0: "tile", 1: "ray", 2: "strip"}
        return {"forward": names[v[0].value], "strip_bins": v[1].value, "backproject_mode": v[2].value,
                "views_per_cta": v[3].value, "cone_tile": v[4].value}

    def set_cone_tile(self, depth: int):
        """Depth (16 or 8 voxels) of the cone tile transpose's 8 x 8 x depth
        tiles (cone plans only)."""
        _call(lib().mbir_plan_set_cone_tile, self.h, int(depth))

    def set_projector(self, mode: str):
        """2-D: 'ray' (one thread per ray), 'strip' (shared-memory strips) or
        'tile'; cone beam: 'ray' (each lane marches its own range) or
        'aligned' (the lanes of a warp march together; the same mode number
        as 'strip')."""
        _call(lib().mbir_plan_set_projector, self.h, {"tile": 0, "ray": 1, "strip": 2, "aligned": 2}[mode])

    def __del__(self):
        if getattr(self, "h", None) and _abi._lib is not None:
            _abi._lib.mbir_plan_destroy(self.h)
            self.h = None


class Spectrum:
    """Spectral model: Q[E][m], S[c][E] (host FP64)."""

    def __init__(self, Q, S):
        Q = np.ascontiguousarray(np.asarray(Q, dtype=np.float64))
        S = np.ascontiguousarray(np.asarray(S, dtype=np.float64))
        self.n_energy, self.n_mat = Q.shape
        self.n_chan = S.shape[0]
        if S.shape[1] != self.n_energy:
            raise ValueError("S must be [n_chan][n_energy] with the same energies as Q")
        h = ctypes.c_void_p()
        dp = ctypes.POINTER(ctypes.c_double)
        _call(lib().mbmd_spectrum_create, self.n_mat, self.n_energy, self.n_chan, Q.ctypes.data_as(dp),
              S.ctypes.data_as(dp), ctypes.byref(h))
        self.h = h
        self.blur = None
        self.noise = None

    def set_blur(self, taps, row: int):
        """Detector blur B of the outer operator B S (Eq. 1): odd-length taps
        b[-r..r] (r <= 3) applied along rows of `row` consecutive rays; an
        empty or None `taps` removes it."""
        taps = np.ascontiguousarray(np.asarray([] if taps is None else taps, dtype=np.float64).ravel())
        if taps.size % 2 == 0 and taps.size:
            raise ValueError("blur taps must have odd length 2 r + 1")
        radius = taps.size // 2
        dp = ctypes.POINTER(ctypes.c_double)
        _call(lib().mbmd_spectrum_set_blur, self.h, int(radius), int(row),
              taps.ctypes.data_as(dp) if taps.size else None)
        self.blur = (taps.copy(), int(row)) if radius else None

    def set_noise(self, a: float, row: int = 2):
        """Correlated detector noise: correlation a^|j-k| between cells j, k
        of a detector row of `row` rays (``mbmd_spectrum_set_noise``); a = 0
        restores the diagonal covariance."""
        _call(lib().mbmd_spectrum_set_noise, self.h, float(a), int(row))
        self.noise = (float(a), int(row)) if a > 0 else None

    def __del__(self):
        if getattr(self, "h", None) and _abi._lib is not None:
            _abi._lib.mbmd_spectrum_destroy(self.h)
            self.h = None


def mbir_project(plan: Plan, x, l=None, n_mat: int | None = None):
    torch = _torch()
    n_mat = n_mat or x.numel() // plan.n_pix
    if l is None:
        l = torch.empty((n_mat, plan.n_rays), device=x.device, dtype=torch.float32)
    _call(lib().mbir_project, plan.h, _dev(x, "x"), _dev(l, "l"), int(n_mat), _stream())
    return l


def mbir_backproject(plan: Plan, s, x=None, n_mat: int | None = None, accumulate: bool = False):
    torch = _torch()
    n_mat = n_mat or s.numel() // plan.n_rays
    if x is None:
        x = torch.empty((n_mat,) + plan.image_shape, device=s.device, dtype=torch.float32)
    _call(lib().mbir_backproject, plan.h, _dev(s, "s"), _dev(x, "x"), int(n_mat), int(bool(accumulate)), _stream())
    return x


def mbmd_forward_model(spec: Spectrum, l, ybar=None):
    torch = _torch()
    n_rays = l.numel() // spec.n_mat
    if ybar is None:
        ybar = torch.empty((spec.n_chan, n_rays), device=l.device, dtype=torch.float32)
    _call(lib().mbmd_forward_model, spec.h, _dev(l, "l"), _dev(ybar, "ybar"), int(n_rays), _stream())
    return ybar


def mbmd_objective(plan: Plan | None, spec: Spectrum, x_or_l, y):
    torch = _torch()
    out = torch.empty(1, device=y.device, dtype=torch.float64)
    n_rays = y.numel() // spec.n_chan
    _call(lib().mbmd_objective, plan.h if plan else None, spec.h, _dev(x_or_l, "x_or_l"), _dev(y, "y"), int(n_rays),
          _dev(out, "objective", torch.float64), _stream())
    return out


def mbmd_gradient(plan: Plan | None, spec: Spectrum, x_or_l, y, grad=None, with_objective: bool = True):
    torch = _torch()
    n_rays = y.numel() // spec.n_chan
    if grad is None:
        grad = torch.empty_like(x_or_l)
    obj = torch.empty(1, device=y.device, dtype=torch.float64) if with_objective else None
    _call(lib().mbmd_gradient, plan.h if plan else None, spec.h, _dev(x_or_l, "x_or_l"), _dev(y, "y"), int(n_rays),
          _dev(grad, "grad"), _dev(obj, "objective", torch.float64) if obj is not None else None, _stream())
    return grad, obj


def mbmd_curvature(plan: Plan | None, spec: Spectrum, x_or_l, y, curv=None):
    """Plain-SPS separable curvature A^T kappa (``mbmd_curvature``)."""
    torch = _torch()
    n_rays = y.numel() // spec.n_chan
    if curv is None:
        curv = torch.empty_like(x_or_l)
    _call(lib().mbmd_curvature, plan.h if plan else None, spec.h, _dev(x_or_l, "x_or_l"), _dev(y, "y"), int(n_rays),
          _dev(curv, "curv"), _stream())
    return curv


class Precond:
    """One-time preconditioner build (``psps_precondition_build``)."""

    def __init__(self, plan: Plan | None, spec: Spectrum, kind: str, y=None, beta=None, haar_lattice: int = 3,
                 lam=None, m0=None, blocks=None, sides: int | None = None):
        """Build from data (``y``) or, when ``lam`` / ``blocks`` is given,
        create from precomputed eigenvalues / blocks
        (``psps_precondition_create``).  sides: M = M0^T C (1) or the
        literal M0^T C M0 (2) for the Fourier and wavelet kinds
        (``psps_precondition_set_sides``); None keeps the kind's default (2
        for one material, 1 for the cross-material kinds)."""
        self.sides = sides
        self.kind = kind
        self.plan, self.spec = plan, spec
        self.n_rays = plan.n_rays if plan else (blocks.shape[-1] if blocks is not None else
                                                 (y.numel() // spec.n_chan if y is not None else 0))
        if y is None:
            n = plan.n_pix if plan else (blocks.shape[-1] if blocks is not None else 0)
            h = ctypes.c_void_p()
            _call(lib().psps_precondition_create, plan.h if plan else None, PSPS_PRECOND[kind], spec.n_mat, int(n),
                  _dev(lam, "lam") if lam is not None else None, _dev(m0, "m0") if m0 is not None else None,
                  _dev(blocks, "blocks") if blocks is not None else None, _stream(), ctypes.byref(h))
            self.h = h
            if sides is not None:
                _call(lib().psps_precondition_set_sides, h, int(sides))
            return
        n_rays = y.numel() // spec.n_chan
        b = None
        if beta is not None:
            self._beta = np.ascontiguousarray(np.asarray(beta, dtype=np.float64).reshape(spec.n_mat, spec.n_mat))
            b = self._beta.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        h = ctypes.c_void_p()
        _call(lib().psps_precondition_build, plan.h if plan else None, spec.h, PSPS_PRECOND[kind], _dev(y, "y"),
              int(n_rays), b, int(haar_lattice), _stream(), ctypes.byref(h))
        self.h = h
        if sides is not None:
            _call(lib().psps_precondition_set_sides, h, int(sides))

    def __del__(self):
        if getattr(self, "h", None) and _abi._lib is not None:
            _abi._lib.psps_precondition_destroy(self.h)
            self.h = None


def psps_precondition(pc: Precond, op: str, inp, out=None):
    torch = _torch()
    if out is None:
        out = torch.empty_like(inp)
    _call(lib().psps_precondition, pc.h, PSPS_APPLY[op], _dev(inp, "in"), _dev(out, "out"), _stream())
    return out


def psps_precondition_export(pc: Precond, what: str):
    """Copy of one array of a preconditioner (``psps_precondition_export``):
    'scales' (clamp(Lambda~)^-1/2 [n], or the cross-material blocks
    [n_mat][n_mat][n]), 'blocks' (M0 blocks [n_mat][n_mat][n]), 'm0' ([n]),
    'hblocks' ((F+R)1_k blocks, built only) or 'estimate' (the Eq. 18
    estimates, built Fourier / wavelet kinds only)."""
    torch = _torch()
    nm = pc.spec.n_mat
    n = pc.plan.n_pix if pc.plan else pc.n_rays
    cross = pc.kind in ("block_fourier", "block_haar")
    blocky = what in ("blocks", "hblocks") or (what in ("scales", "estimate") and cross)
    shape = (nm, nm, n) if blocky else (n,)
    out = torch.empty(shape, device="cuda", dtype=torch.float32)
    _call(lib().psps_precondition_export, pc.h, _abi.PSPS_EXPORT[what], _dev(out, "out"), int(out.numel()),
          _stream())
    return out


class State:
    """Iteration state (``psps_state_create``); keeps references to its plan,
    spectrum and preconditioner."""

    def __init__(self, plan: Plan | None, spec: Spectrum, pc: Precond | None, y, beta=None, x0=None,
                 line_search: bool = True, nonneg: bool = False, graph: bool = False, reproject_every: int = 10):
        flags = (FLAG_LINESEARCH if line_search else 0) | (FLAG_NONNEG if nonneg else 0) | (FLAG_GRAPH if graph else 0)
        n_rays = y.numel() // spec.n_chan
        b = None
        if beta is not None:
            self._beta = np.ascontiguousarray(np.asarray(beta, dtype=np.float64).reshape(spec.n_mat, spec.n_mat))
            b = self._beta.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        h = ctypes.c_void_p()
        _call(lib().psps_state_create, plan.h if plan else None, spec.h, pc.h if pc else None, _dev(y, "y"),
              int(n_rays), b, _dev(x0, "x0") if x0 is not None else None, flags, int(reproject_every), _stream(),
              ctypes.byref(h))
        self.h = h
        self.plan, self.spec, self.pc = plan, spec, pc
        self.n_mat = spec.n_mat
        self.shape = (spec.n_mat,) + (plan.image_shape if plan else (n_rays,))

    def __del__(self):
        if getattr(self, "h", None) and _abi._lib is not None:
            _abi._lib.psps_state_destroy(self.h)
            self.h = None


def psps_step(state: State, n_iter: int, history: bool = True):
    """Run n_iter iterations; returns the FP64 objective history (length
    n_iter + 1, synchronising) or None (asynchronous)."""
    if history:
        h = np.zeros(n_iter + 1)
        _call(lib().psps_step, state.h, int(n_iter), h.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _stream())
        return h
    _call(lib().psps_step, state.h, int(n_iter), None, _stream())
    return None


class Batch:
    """Independent states advanced together, one CUDA graph per iteration
    (``psps_batch_create``); keeps references to its states."""

    def __init__(self, states):
        self.states = list(states)
        arr = (ctypes.c_void_p * len(self.states))(*[s.h for s in self.states])
        h = ctypes.c_void_p()
        _call(lib().psps_batch_create, arr, len(self.states), ctypes.byref(h))
        self.h = h

    def __del__(self):
        if getattr(self, "h", None) and _abi._lib is not None:
            _abi._lib.psps_batch_destroy(self.h)
            self.h = None


def psps_batch_step(batch: Batch, n_iter: int, history: bool = True):
    """Run n_iter iterations of every state; returns the objective histories
    ([n_states, n_iter + 1], synchronising) or None (asynchronous)."""
    if history:
        h = np.zeros((len(batch.states), n_iter + 1))
        _call(lib().psps_batch_step, batch.h, int(n_iter), h.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
              _stream())
        return h
    _call(lib().psps_batch_step, batch.h, int(n_iter), None, _stream())
    return None


def psps_batch_launch_count(batch: Batch) -> int:
    c = ctypes.c_int64()
    _call(lib().psps_batch_launch_count, batch.h, ctypes.byref(c))
    return int(c.value)


def psps_state_set_data(state: State, y):
    """Copy new measured counts into the state: a host tensor (pinned for an
    asynchronous copy) or a CUDA tensor of n_chan * n_rays float32 values."""
    torch = _torch()
    if not isinstance(y, torch.Tensor) or y.dtype != torch.float32 or not y.is_contiguous():
        raise TypeError("y must be a contiguous float32 tensor")
    _call(lib().psps_state_set_data, state.h, ctypes.c_void_p(y.data_ptr()), int(y.numel()), _stream())


def psps_get_image(state: State, x=None):
    torch = _torch()
    if x is None:
        x = torch.empty(state.shape, device="cuda", dtype=torch.float32)
    _call(lib().psps_get_image, state.h, _dev(x, "x"), _stream())
    return x


def psps_get_alphas(state: State, n: int):
    a = np.zeros(n)
    _call(lib().psps_get_alphas, state.h, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(n), _stream())
    return a


def psps_profile(state: State, enable: bool = True):
    _call(lib().psps_profile, state.h, int(bool(enable)))


def psps_profile_read(state: State):
    """{stage: (total ms, timed runs)} of the enabled stage timers."""
    ms = (ctypes.c_double * len(_abi.PROF_STAGES))()
    cnt = (ctypes.c_int64 * len(_abi.PROF_STAGES))()
    _call(lib().psps_profile_read, state.h, ms, cnt)
    return {k: (ms[i], cnt[i]) for i, k in enumerate(_abi.PROF_STAGES)}


def psps_launch_count(state: State) -> int:
    c = ctypes.c_int64()
    _call(lib().psps_launch_count, state.h, ctypes.byref(c))
    return int(c.value)


class MBMDData:
    """torch.autograd.Function over the basis images: forward returns the PWLS
    data term L(x) (FP64 scalar), backward is the hand-written adjoint
    ``mbmd_gradient`` (recomputes l = A x and exp(-Q l) instead of storing
    them)."""

    _fn = None

    @classmethod
    def apply(cls, x, plan, spec, y):
        if cls._fn is None:
            torch = _torch()

            class _F(torch.autograd.Function):
                @staticmethod
                def forward(ctx, x_, plan_, spec_, y_):
                    ctx.save_for_backward(x_, y_)
                    ctx.plan, ctx.spec = plan_, spec_
                    return mbmd_objective(plan_, spec_, x_.contiguous(), y_)[0]

                @staticmethod
                def backward(ctx, gout):
                    x_, y_ = ctx.saved_tensors
                    g, _ = mbmd_gradient(ctx.plan, ctx.spec, x_.contiguous(), y_, with_objective=False)
                    return g * gout.to(g.dtype), None, None, None

            cls._fn = _F
        return cls._fn.apply(x, plan, spec, y)
