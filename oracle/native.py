"""ctypes wrapper of the plain-C FP64 oracle (``oracle/csrc/grf_oracle.c``).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).  Same definitions as
``oracle.field.synth`` and ``oracle.field.mode_sums``; built with gcc and
OpenMP, no fast-math, so it can evaluate sizes that numpy cannot finish in
seconds and serve as the timed CPU baseline.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "csrc", "grf_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force=False):
    """Compile the C oracle with gcc (portable flags: runs on x86-64 and Arm)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        L.oracle_synth.argtypes = [ctypes.c_int64, ctypes.c_int, dp, ctypes.c_int64, dp, dp, dp,
                                   ctypes.c_double, dp]
        L.oracle_synth.restype = ctypes.c_int
        L.oracle_mode_sums.argtypes = [ctypes.c_int64, ctypes.c_int, dp, dp, ctypes.c_int64, dp, dp,
                                       dp, dp, dp]
        L.oracle_mode_sums.restype = ctypes.c_int
        L.oracle_threads.restype = ctypes.c_int
        L.oracle_set_threads.argtypes = [ctypes.c_int]
        _lib = L
    return _lib


def _p(arr):
    return arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _cells(cells):
    c = np.asarray(cells)
    if c.ndim == 1:
        c = c[:, None]
    return np.ascontiguousarray(c, dtype=np.float64)


def threads():
    return lib().oracle_threads()


def set_threads(n):
    lib().oracle_set_threads(int(n))


def synth(a, amp, psi, mu, cells):
    x = _cells(cells)
    amp = np.ascontiguousarray(amp, dtype=np.float64)
    psi = np.ascontiguousarray(psi, dtype=np.float64)
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(len(amp), x.shape[1]))
    y = np.empty(x.shape[0], dtype=np.float64)
    rc = lib().oracle_synth(x.shape[0], x.shape[1], _p(x), len(amp), _p(a), _p(amp), _p(psi),
                            float(mu), _p(y))
    if rc != 0:
        raise ValueError("oracle_synth rejected its arguments")
    return y


def mode_sums(a, psi, cells, g):
    x = _cells(cells)
    psi = np.ascontiguousarray(psi, dtype=np.float64)
    n, d = len(psi), x.shape[1]
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(n, d))
    g = np.ascontiguousarray(g, dtype=np.float64)
    s_cos = np.empty(n)
    s_sin = np.empty(n)
    s_sinx = np.empty((n, d))
    rc = lib().oracle_mode_sums(x.shape[0], d, _p(x), _p(g), n, _p(a), _p(psi), _p(s_cos),
                                _p(s_sin), _p(s_sinx))
    if rc != 0:
        raise ValueError("oracle_mode_sums rejected its arguments")
    return s_cos, s_sin, s_sinx
