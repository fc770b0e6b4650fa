"""ctypes wrapper of the C parts of the oracle (test infrastructure only):
the direct sums in ``ewald.c`` and the influence-function loops in ``influence.c``.

The C files are compiled with gcc on first use into ``oracle/_build/`` (or by
``build()``, which ``__graft_entry__.build`` calls).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "ewald.c"), os.path.join(_HERE, "influence.c")]
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    os.makedirs(_BUILD, exist_ok=True)
    stale = not os.path.exists(_LIB) or any(os.path.getmtime(_LIB) < os.path.getmtime(s) for s in _SRCS)
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, *_SRCS, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            lib.egt_direct.restype = ctypes.c_long
            lib.egt_direct.argtypes = [ctypes.c_int, dp, dp, dp, ctypes.c_double, ctypes.c_double, dp, dp, dp]
            lib.ewald_real.restype = ctypes.c_double
            lib.ewald_real.argtypes = [ctypes.c_int, dp, dp, dp, ctypes.c_double, ctypes.c_double]
            lib.influence_ik.restype = None
            lib.influence_ik.argtypes = [dp, ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_double,
                                         ctypes.c_int, ctypes.c_int, dp]
            lib.erf_shell_sum.restype = ctypes.c_double
            lib.erf_shell_sum.argtypes = [ctypes.c_int, dp, dp, dp, ctypes.c_double, ctypes.c_double]
            _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def egt_direct(pos, q, box, beta, cut=40.0, forces=True):
    """E_Gt (Eq. DPLR:EGt), forces and virial (xx yy zz xy xz yz) by direct sum."""
    lib = _load()
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    q = np.ascontiguousarray(q, dtype=np.float64)
    box = np.ascontiguousarray(np.broadcast_to(np.asarray(box, float), (3,)), dtype=np.float64)
    n = pos.shape[0]
    e = np.zeros(1)
    f = np.zeros((n, 3)) if forces else None
    v = np.zeros(6)
    lib.egt_direct(n, _p(pos), _p(q), _p(box), float(beta), float(cut), _p(e),
                   _p(f) if forces else ctypes.POINTER(ctypes.c_double)(), _p(v))
    return dict(energy=float(e[0]), forces=f, virial=v)


def ewald_real(pos, q, box, alpha, rcut):
    lib = _load()
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    q = np.ascontiguousarray(q, dtype=np.float64)
    box = np.ascontiguousarray(np.broadcast_to(np.asarray(box, float), (3,)), dtype=np.float64)
    return float(lib.ewald_real(pos.shape[0], _p(pos), _p(q), _p(box), float(alpha), float(rcut)))


def ewald_full(pos, q, box, alpha, rcut=None, cut=40.0):
    """Classical point-charge Ewald energy with a conducting boundary:
    real (erfc) + reciprocal (the E_Gt sum with beta = alpha) - self."""
    if rcut is None:
        rcut = 6.5 / alpha  # erfc(6.5) ~ 4e-20
    q = np.asarray(q, float)
    e_real = ewald_real(pos, q, box, alpha, rcut)
    e_rec = egt_direct(pos, q, box, alpha, cut=cut, forces=False)["energy"]
    e_self = alpha / math.sqrt(math.pi) * float(np.sum(q * q))
    return e_real + e_rec - e_self


def erf_shell_sum(pos, q, box, beta, R):
    lib = _load()
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    q = np.ascontiguousarray(q, dtype=np.float64)
    box = np.ascontiguousarray(np.broadcast_to(np.asarray(box, float), (3,)), dtype=np.float64)
    return float(lib.erf_shell_sum(pos.shape[0], _p(pos), _p(q), _p(box), float(beta), float(R)))


def influence_ik(box, mesh, p, beta, alias=2, denom_range=20):
    """Full-spectrum optimal ik influence function G, shape mesh (see influence.c)."""
    lib = _load()
    box = np.ascontiguousarray(np.broadcast_to(np.asarray(box, float), (3,)), dtype=np.float64)
    m = np.ascontiguousarray(mesh, dtype=np.int32)
    G = np.zeros(tuple(int(x) for x in mesh))
    lib.influence_ik(_p(box), m.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), int(p), float(beta),
                     int(alias), int(denom_range), _p(G))
    return G
