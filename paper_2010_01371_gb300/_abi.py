"""ctypes declarations of the C ABI in ``include/mbir.h`` (argument
marshalling only; every computation runs in ``libpsps.so``)."""
from __future__ import annotations

import ctypes
import os

from . import _build

c_int, c_int64, c_double, c_void_p = ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
P = ctypes.POINTER

MBIR_OK = 0
STATUS = {0: "MBIR_OK", -1: "MBIR_ERR_ARG", -2: "MBIR_ERR_CUDA", -3: "MBIR_ERR_OOM", -4: "MBIR_ERR_NONFINITE",
          -5: "MBIR_ERR_TIMEOUT", -6: "MBIR_ERR_UNIMPLEMENTED"}

PSPS_PRECOND = {"none": 0, "fourier": 1, "mod_fourier": 2, "haar": 3, "block": 4, "block_fourier": 5,
                "block_haar": 6}
PSPS_APPLY = {"M": 0, "MT": 1, "absM": 2, "absMT": 3}
PSPS_EXPORT = {"scales": 0, "blocks": 1, "m0": 2, "hblocks": 3, "estimate": 4}
FLAG_LINESEARCH, FLAG_NONNEG, FLAG_GRAPH = 1, 2, 4
PROF_STAGES = ["reproject", "model", "backproject", "precond", "project", "linesearch", "update"]


class MbirGeometry(ctypes.Structure):
    _fields_ = [("kind", c_int), ("nx", c_int), ("ny", c_int), ("nz", c_int),
                ("dx", c_double), ("dy", c_double), ("dz", c_double),
                ("n_views", c_int), ("angle0", c_double), ("angle_span", c_double),
                ("n_u", c_int), ("n_v", c_int), ("du", c_double), ("dv", c_double),
                ("sid", c_double), ("sdd", c_double)]


# (name, restype, argtypes) for every exported entry point of include/mbir.h
SIGNATURES = [
    ("mbir_plan_create", c_int, [P(MbirGeometry), c_int, P(c_void_p)]),
    ("mbir_plan_destroy", c_int, [c_void_p]),
    ("mbir_plan_n_rays", c_int64, [c_void_p]),
    ("mbir_plan_n_pix", c_int64, [c_void_p]),
    ("mbir_plan_set_backprojector", c_int, [c_void_p, c_int]),
    ("mbir_plan_set_tiling", c_int, [c_void_p, c_int]),
    ("mbir_plan_autotune", c_int, [c_void_p, c_int, c_void_p, P(c_int)]),
    ("mbir_plan_set_projector", c_int, [c_void_p, c_int]),
    ("mbir_plan_tuning", c_int, [c_void_p, P(c_int), P(c_int), P(c_int), P(c_int), P(c_int)]),
    ("mbir_plan_set_cone_tile", c_int, [c_void_p, c_int]),
    ("mbir_plan_set_strip_bins", c_int, [c_void_p, c_int]),
    ("mbir_project", c_int, [c_void_p, c_void_p, c_void_p, c_int, c_void_p]),
    ("mbir_backproject", c_int, [c_void_p, c_void_p, c_void_p, c_int, c_int, c_void_p]),
    ("mbmd_spectrum_create", c_int, [c_int, c_int, c_int, P(c_double), P(c_double), P(c_void_p)]),
    ("mbmd_spectrum_destroy", c_int, [c_void_p]),
    ("mbmd_spectrum_set_blur", c_int, [c_void_p, c_int, c_int, P(c_double)]),
    ("mbmd_spectrum_set_noise", c_int, [c_void_p, c_double, c_int]),
    ("mbmd_forward_model", c_int, [c_void_p, c_void_p, c_void_p, c_int64, c_void_p]),
    ("mbmd_objective", c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_void_p, c_void_p]),
    ("mbmd_gradient", c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_void_p, c_void_p, c_void_p]),
    ("mbmd_curvature", c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_void_p, c_void_p]),
    ("mbmd_objective_noalloc", c_int, [c_int, c_int, c_int, P(c_double), P(c_double), c_void_p, c_void_p, c_int64,
                                       c_void_p, c_void_p]),
    ("psps_precondition_build", c_int, [c_void_p, c_void_p, c_int, c_void_p, c_int64, P(c_double), c_int,
                                        c_void_p, P(c_void_p)]),
    ("psps_precondition_create", c_int, [c_void_p, c_int, c_int, c_int64, c_void_p, c_void_p, c_void_p, c_void_p,
                                         P(c_void_p)]),
    ("psps_precondition_destroy", c_int, [c_void_p]),
    ("psps_precondition", c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p]),
    ("psps_precondition_export", c_int, [c_void_p, c_int, c_void_p, c_int64, c_void_p]),
    ("psps_precondition_set_sides", c_int, [c_void_p, c_int]),
    ("psps_state_create", c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int64, P(c_double), c_void_p, c_int,
                                  c_int, c_void_p, P(c_void_p)]),
    ("psps_state_destroy", c_int, [c_void_p]),
    ("psps_state_set_data", c_int, [c_void_p, c_void_p, c_int64, c_void_p]),
    ("psps_step", c_int, [c_void_p, c_int, P(c_double), c_void_p]),
    ("psps_batch_create", c_int, [P(c_void_p), c_int, P(c_void_p)]),
    ("psps_batch_destroy", c_int, [c_void_p]),
    ("psps_batch_step", c_int, [c_void_p, c_int, P(c_double), c_void_p]),
    ("psps_batch_launch_count", c_int, [c_void_p, P(c_int64)]),
    ("psps_get_image", c_int, [c_void_p, c_void_p, c_void_p]),
    ("psps_get_alphas", c_int, [c_void_p, P(c_double), c_int, c_void_p]),
    ("psps_profile", c_int, [c_void_p, c_int]),
    ("psps_profile_read", c_int, [c_void_p, P(c_double), P(c_int64)]),
    ("psps_launch_count", c_int, [c_void_p, P(c_int64)]),
    ("mbir_last_error", ctypes.c_char_p, []),
]

_lib = None


class MbirError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def load(path: str | None = None, build: bool = True):
    """Load (building first if needed) the in-tree library.  Raises when the
    CUDA library cannot be built or loaded: there is no fallback path."""
    global _lib
    if _lib is not None:
        return _lib
    if path is None:
        path = _build.build() if build else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libpsps.so not found at {path}; run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(status: int):
    if status != MBIR_OK:
        raise MbirError(status, _lib.mbir_last_error().decode())
