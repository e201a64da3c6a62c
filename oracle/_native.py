"""Loader for the oracle's plain-C potentials (``potentials.c``).

TEST INFRASTRUCTURE ONLY: imported by ``oracle`` and nothing in the product.
The shared object is built with gcc on first use (``build()``), on x86 and on
Arm alike; it depends on libc/libm only.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "potentials.c")
_SO = os.path.join(_HERE, "_oracle_potentials.so")
_lib = None


def build(force=False):
    """Compile potentials.c into a shared object next to it (gcc -O2)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC",
                               "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        L.oracle_lj.argtypes = [ctypes.c_int, dp, dp, ctypes.c_double, ctypes.c_double,
                                ctypes.c_double, ctypes.c_int, dp, dp, dp]
        L.oracle_tersoff.argtypes = [ctypes.c_int, dp, dp, dp, dp, dp, dp]
        L.oracle_tersoff_sampled.argtypes = [ctypes.c_int, dp, dp, dp, ctypes.c_int, ip, dp]
        L.oracle_lj_sampled.argtypes = [ctypes.c_int, dp, dp, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_double, ctypes.c_int, ip, dp]
        L.oracle_count_neighbours.argtypes = [ctypes.c_int, dp, dp, ctypes.c_double, ctypes.c_int]
        for f in (L.oracle_lj, L.oracle_tersoff, L.oracle_tersoff_sampled, L.oracle_lj_sampled,
                  L.oracle_count_neighbours):
            f.restype = ctypes.c_int
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def lj(R, h, eps, sigma, rc, shift):
    R = _f64(R, (-1, 3))
    h = _f64(h, (3, 3))
    n = R.shape[0]
    e = np.zeros(n)
    F = np.zeros((n, 3))
    V = np.zeros((3, 3))
    lib().oracle_lj(n, _dp(R), _dp(h), eps, sigma, rc, int(shift), _dp(e), _dp(F), _dp(V))
    return e, F, V


def tersoff(R, h, par):
    R = _f64(R, (-1, 3))
    h = _f64(h, (3, 3))
    p = _f64(par)
    n = R.shape[0]
    e = np.zeros(n)
    F = np.zeros((n, 3))
    V = np.zeros((3, 3))
    st = lib().oracle_tersoff(n, _dp(R), _dp(h), _dp(p), _dp(e), _dp(F), _dp(V))
    if st != 0:
        raise RuntimeError("oracle_tersoff: reverse neighbour entry missing")
    return e, F, V


def tersoff_sampled(R, h, par, idx):
    R = _f64(R, (-1, 3))
    h = _f64(h, (3, 3))
    p = _f64(par)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    F = np.zeros((len(idx), 3))
    st = lib().oracle_tersoff_sampled(R.shape[0], _dp(R), _dp(h), _dp(p), len(idx), _ip(idx),
                                      _dp(F))
    if st != 0:
        raise RuntimeError("oracle_tersoff_sampled: reverse neighbour entry missing")
    return F


def lj_sampled(R, h, eps, sigma, rc, idx):
    R = _f64(R, (-1, 3))
    h = _f64(h, (3, 3))
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    F = np.zeros((len(idx), 3))
    lib().oracle_lj_sampled(R.shape[0], _dp(R), _dp(h), eps, sigma, rc, len(idx), _ip(idx), _dp(F))
    return F


def count_neighbours(R, h, rc, i):
    R = _f64(R, (-1, 3))
    h = _f64(h, (3, 3))
    return lib().oracle_count_neighbours(R.shape[0], _dp(R), _dp(h), rc, int(i))
