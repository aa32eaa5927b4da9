"""Builds and loads the oracle's C library (plain gcc, -O2, no fast-math).

Test infrastructure only: see the package docstring.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_build/liboracle.so (idempotent)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if (not force and os.path.exists(_OUT)
            and os.path.getmtime(_OUT) >= os.path.getmtime(_SRC)):
        return _OUT
    tmp = _OUT + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                           "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _OUT)
    return _OUT


_D = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_L, _I, _F = ctypes.c_long, ctypes.c_int, ctypes.c_double

_SIGS = {
    "or_blur_decimate": [_D, _L, _L, _D, _I, _I, _D],
    "or_blur_decimate_adj": [_D, _L, _L, _D, _I, _I, _D],
    "or_laplacian": [_D, _L, _L, _D],
    "or_pan_stats": [_D, _L, _L, _I, _F, _D, _D, _D, _D],
    "or_matting_apply": [_D, _D, _D, _D, _L, _L, _I, _D],
    "or_guided_filter": [_D, _D, _D, _D, _L, _L, _I, _D],
    "or_apply_system": [_L, _L, _I, _D, _I, _D, _D, _D, _I, _F, _I, _D, _D],
    "or_cg": [_L, _L, _I, _D, _I, _D, _D, _D, _I, _F, _I, _D, _D, _F, _I,
              ctypes.POINTER(ctypes.c_double)],
    "or_box_filter": [_D, _L, _L, _I, _D],
    "or_kernel_normal_eq": [_D, _L, _L, _I, _I, _D, _D, _D],
}


def lib():
    global _lib
    with _lock:
        if _lib is None:
            handle = ctypes.CDLL(build())
            for name, args in _SIGS.items():
                fn = getattr(handle, name)
                fn.argtypes = args
                fn.restype = ctypes.c_int if name == "or_cg" else None
            _lib = handle
    return _lib
