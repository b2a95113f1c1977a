"""FP64 CPU oracle for the volume potential (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The product path (the CUDA library and
its binding) never does. See ``vp_oracle.cpp`` for what is computed and how.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "vp_oracle.cpp")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle (g++ -O2 -fopenmp) into oracle/_build/liboracle.so."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared",
                               _SRC, "-o", tmp])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        d = ctypes.POINTER(ctypes.c_double)
        i32 = ctypes.POINTER(ctypes.c_int32)
        lib.ora_volume_potential.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                             ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                             ctypes.c_int, i32, i32, i32, d, ctypes.c_int, d, d,
                                             d, d, d, ctypes.c_int]
        lib.ora_gauss_legendre.argtypes = [ctypes.c_int, d, d]
        lib.ora_kernel.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int, d, d, d]
        lib.ora_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def num_threads() -> int:
    return int(_load().ora_num_threads())


def gauss_legendre(n: int):
    x = np.zeros(n); w = np.zeros(n)
    if _load().ora_gauss_legendre(n, _dp(x), _dp(w)) != 0:
        raise ValueError("bad order")
    return x, w


def kernel(kind: int, alpha: float, r):
    r = np.ascontiguousarray(r, np.float64)
    g = np.zeros_like(r); dg = np.zeros_like(r)
    if _load().ora_kernel(kind, alpha, r.size, _dp(r), _dp(g), _dp(dg)) != 0:
        raise ValueError("bad kernel arguments")
    return g, dg


def volume_potential(kind: int, alpha: float, p: int, tree, f, tx, ty, nthreads: int = 0):
    """u, du/dx, du/dy at the targets (tx, ty) for nodal source values f on `tree`."""
    lv = np.ascontiguousarray(tree.level, np.int32)
    ix = np.ascontiguousarray(tree.ix, np.int32)
    iy = np.ascontiguousarray(tree.iy, np.int32)
    f = np.ascontiguousarray(f, np.float64)
    tx = np.ascontiguousarray(tx, np.float64)
    ty = np.ascontiguousarray(ty, np.float64)
    assert f.size == lv.size * p * p and tx.size == ty.size
    u = np.zeros(tx.size); ux = np.zeros(tx.size); uy = np.zeros(tx.size)
    rc = _load().ora_volume_potential(int(kind), float(alpha), int(p), float(tree.cx), float(tree.cy),
                                      float(tree.side), int(lv.size), _ip(lv), _ip(ix), _ip(iy), _dp(f),
                                      int(tx.size), _dp(tx), _dp(ty), _dp(u), _dp(ux), _dp(uy),
                                      int(nthreads))
    if rc == -2:
        raise ValueError("a target lies on a leaf boundary")
    if rc != 0:
        raise ValueError(f"oracle rejected its arguments (status {rc})")
    return u, ux, uy
