"""ctypes binding of cellverlet.c: the paper's Verlet-list method on the CPU in FP64.

A CPU baseline for bench.py, checked against the all-pairs oracle in tests/ (test and benchmark
infrastructure only; see the package docstring).  The method: cell grid and counting sort
(Sec. 2.2, Fig. 3) with the particle reorder of Sec. 3.3, half pair list within r_s stored as
KeyPointer / SortedList (Sec. 2.3-2.4, Alg. 1, Fig. 6), branch-free force with one division per
pair and Newton's third law (Alg. 4-6), velocity-Verlet (Sec. 4.5), rebuild once a particle moved
more than margin/2.
"""
from __future__ import annotations

import ctypes

import numpy as np

from .build import build_cellverlet
from .oracle import LJParams

_LIB = None
_D, _I64, _P = ctypes.c_double, ctypes.c_int64, ctypes.c_void_p


def lib():
    global _LIB
    if _LIB is None:
        L = ctypes.CDLL(build_cellverlet())
        L.cv_run.restype = ctypes.c_int
        L.cv_run.argtypes = [_I64, _P, _P, _D, _D, _D, _D, _D, _D, _D, _D, _I64, _P, _P, _P, _P, _P, _P, _P]
        _LIB = L
    return _LIB


def run(x, v, L: float, dt: float, nsteps: int, margin: float, p: LJParams = LJParams()):
    """nsteps of velocity-Verlet over the Verlet list.  Returns a dict: x (unwrapped), v, f (id
    order), pe, ke, vir, rebuilds, pairs (half-list pairs of the last construction), seconds (the
    nsteps only)."""
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3).copy()
    v = np.zeros_like(x) if v is None else np.ascontiguousarray(v, dtype=np.float64).reshape(-1, 3).copy()
    f = np.empty_like(x)
    pe, ke, vir, sec = _D(), _D(), _D(), _D()
    reb, pairs = _I64(), _I64()
    eps, sigma, rc, c2, c0 = p.args()
    r = lib().cv_run(x.shape[0], x.ctypes.data_as(_P), v.ctypes.data_as(_P), float(L), rc, float(margin), eps,
                     sigma, c2, c0, float(dt), int(nsteps), f.ctypes.data_as(_P), ctypes.byref(pe),
                     ctypes.byref(ke), ctypes.byref(vir), ctypes.byref(reb), ctypes.byref(pairs), ctypes.byref(sec))
    if r != 0:
        raise RuntimeError("cv_run failed (%d)" % r)
    return dict(x=x, v=v, f=f, pe=pe.value, ke=ke.value, vir=vir.value, rebuilds=reb.value, pairs=pairs.value,
                seconds=sec.value)
