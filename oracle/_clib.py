"""Loader for the oracle's C part (joseph_fp64.c: the parallel-, fan- and cone-beam Joseph
projectors), compiled with gcc on demand.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "joseph_fp64.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_OUT = os.path.join(_OUT_DIR, "liboracle_joseph.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle's C file into a shared library (gcc, OpenMP, -O2, no
    fast-math so FP64 semantics are kept).  Returns the library path."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    stale = (not os.path.exists(_OUT)) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC)
    if force or stale:
        tmp = _OUT + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c99", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _OUT)
    return _OUT


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            for name in ("oracle_joseph_forward", "oracle_joseph_transpose"):
                f = getattr(L, name)
                f.restype = None
                f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, ip,
                              ctypes.c_double, ctypes.c_double, dp, dp]
            for name in ("oracle_joseph_forward_rays", "oracle_joseph_transpose_rays"):
                f = getattr(L, name)
                f.restype = None
                f.argtypes = [ctypes.c_int, ctypes.c_long, dp, dp, dp, ip, dp, dp]
            for name in ("oracle_cone_forward", "oracle_cone_transpose"):
                f = getattr(L, name)
                f.restype = None
                f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_long, dp, dp, dp, dp, dp, dp, ip, dp, dp]
            _lib = L
    return _lib
