"""Oracle projector: ctypes front end to ``joseph.c`` (FP64 Joseph projector).

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "joseph.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libogjoseph.so")
_lock = threading.Lock()
_lib = None


class _Geom(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
                ("n_views", ctypes.c_int), ("angle0", ctypes.c_double), ("angle_span", ctypes.c_double),
                ("n_u", ctypes.c_int), ("n_v", ctypes.c_int), ("du", ctypes.c_double), ("dv", ctypes.c_double),
                ("sid", ctypes.c_double), ("sdd", ctypes.c_double)]


def build(force: bool = False) -> str:
    """Compile ``joseph.c`` with gcc (plain C, -O2, no fast-math)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            os.makedirs(_BUILD, exist_ok=True)
            tmp = _LIB + f".{os.getpid()}.tmp"
            subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fno-fast-math", "-ffp-contract=off",
                                   "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        lib.og_project.argtypes = [P(_Geom), P(ctypes.c_double), P(ctypes.c_double)]
        lib.og_backproject.argtypes = [P(_Geom), P(ctypes.c_double), P(ctypes.c_double)]
        lib.og_project_rays.argtypes = [P(_Geom), P(ctypes.c_double), P(ctypes.c_int64), ctypes.c_int64,
                                        P(ctypes.c_double)]
        lib.og_ray.argtypes = [P(_Geom), ctypes.c_int64, P(ctypes.c_double), P(ctypes.c_double)]
        _lib = lib
    return _lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Projector:
    """A (and A^T) for one geometry; images ``[n_mat][*image_shape]`` and
    sinograms ``[n_mat][n_rays]`` in FP64."""

    def __init__(self, geom):
        self.geom = geom
        self._g = _Geom(int(geom.kind), int(geom.nx), int(geom.ny), int(geom.nz), float(geom.dx),
                        float(geom.dy), float(geom.dz), int(geom.n_views), float(geom.angle0),
                        float(geom.angle_span), int(geom.n_u), int(geom.n_v), float(geom.du), float(geom.dv),
                        float(geom.sid), float(geom.sdd))
        self.lib = _load()
        self.image_shape = tuple(geom.image_shape)
        self.n_rays = int(geom.n_rays)

    def project(self, x: np.ndarray) -> np.ndarray:
        x = np.asarray(x, dtype=np.float64)
        x = x.reshape((-1,) + self.image_shape)
        out = np.zeros((x.shape[0], self.n_rays))
        for m in range(x.shape[0]):
            xm = np.ascontiguousarray(x[m])
            self.lib.og_project(ctypes.byref(self._g), _dptr(xm), _dptr(out[m]))
        return out

    def backproject(self, s: np.ndarray) -> np.ndarray:
        s = np.asarray(s, dtype=np.float64).reshape(-1, self.n_rays)
        out = np.zeros((s.shape[0],) + self.image_shape)
        for m in range(s.shape[0]):
            sm = np.ascontiguousarray(s[m])
            om = np.zeros(self.image_shape)
            self.lib.og_backproject(ctypes.byref(self._g), _dptr(sm), _dptr(om))
            out[m] = om
        return out

    def project_rays(self, x: np.ndarray, rays: np.ndarray) -> np.ndarray:
        """[A x]_r for the listed ray indices only (one image)."""
        xm = np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(self.image_shape))
        r = np.ascontiguousarray(np.asarray(rays, dtype=np.int64))
        out = np.zeros(r.size)
        self.lib.og_project_rays(ctypes.byref(self._g), _dptr(xm),
                                 r.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), r.size, _dptr(out))
        return out

    def ray(self, r: int):
        p0 = np.zeros(3)
        u = np.zeros(3)
        self.lib.og_ray(ctypes.byref(self._g), int(r), _dptr(p0), _dptr(u))
        return p0, u


class IdentityProjector:
    """Projection-domain decomposition: the "projector" is the identity and
    the unknowns are the material line integrals themselves (x -> l)."""

    def __init__(self, n_rays: int):
        self.n_rays = int(n_rays)
        self.image_shape = (self.n_rays,)

    def project(self, x):
        return np.asarray(x, dtype=np.float64).reshape(-1, self.n_rays).copy()

    def backproject(self, s):
        return np.asarray(s, dtype=np.float64).reshape(-1, self.n_rays).copy()
