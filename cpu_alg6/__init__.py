"""The paper's blocked CPU spin summation (Algorithms 5a/5b and 6) and the
algorithm it is measured against (Algorithm 2, the NCC code's) as a native
host library, a comparison point for the GPU library on the same machine's
host cores. The GPU package never imports it.

``spinsum_alg6.h`` declares the C entry point; this module builds it with the
host compiler (``build()``) and marshals numpy arrays (argument marshalling
only). Tensors are the paper's dense N^d arrays in column-major order.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libspinsum_alg6.so")


def build(verbose: bool = False) -> str:
    """Compile the library: C++17, no fused multiply-add (each product and sum
    rounds once, in the order the source states), no host-specific flags."""
    os.makedirs(_BUILD, exist_ok=True)
    cmd = ["g++", "-O3", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-pthread",
           "-o", _SO, os.path.join(_HERE, "alg6.cpp"), os.path.join(_HERE, "alg2.cpp")]
    if verbose:
        print(" ".join(cmd))
    subprocess.check_call(cmd)
    return _SO


_lib = None


def _load():
    global _lib
    if _lib is None:
        if not os.path.exists(_SO):
            build()
        lib = ctypes.CDLL(_SO)
        P = ctypes.c_void_p
        lib.spinsum_alg6.argtypes = [ctypes.c_int, ctypes.c_int64, P, P, P, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int]
        lib.spinsum_alg6.restype = ctypes.c_int
        lib.spinsum_alg2.argtypes = [ctypes.c_int, ctypes.c_int64, P, P, P, ctypes.c_int, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_int]
        lib.spinsum_alg2.restype = ctypes.c_int
        _lib = lib
    return _lib


def spinsum_alg6(A: np.ndarray, coef, factorized: bool = False, alpha: float = 1.0, beta: float = 0.0,
                 out: np.ndarray | None = None, inplace: bool = False, bl: int = 0, threads: int = 0) -> np.ndarray:
    """B = alpha * S(A) + beta * B on a dense column-major N^d float64 array
    (d = A.ndim in 2..4). ``coef``: [nfactors, d!] (or [d!]) in lexicographic
    permutation order. Returns B (``A`` itself when ``inplace``)."""
    d = A.ndim
    if A.dtype != np.float64 or not A.flags.f_contiguous or len(set(A.shape)) != 1:
        raise ValueError("A must be a column-major float64 N^d array")
    c = np.ascontiguousarray(np.asarray(coef, dtype=np.float64))
    if c.ndim == 1:
        c = c[None, :]
    if c.ndim != 2 or c.shape[1] != math.factorial(d):
        raise ValueError("coefficient chain must have d! columns")
    if inplace:
        B = A
    elif out is None:
        B = np.zeros(A.shape, dtype=np.float64, order="F")
    else:
        B = out
        if B.shape != A.shape or B.dtype != np.float64 or not B.flags.f_contiguous:
            raise ValueError("out must be a column-major float64 array of A's shape")
    rc = _load().spinsum_alg6(d, A.shape[0], A.ctypes.data, B.ctypes.data, c.ctypes.data, c.shape[0],
                              int(bool(factorized)), float(alpha), float(beta), int(bl), int(threads))
    if rc != 0:
        raise ValueError(f"spinsum_alg6 failed ({rc})")
    return B


def spinsum_alg2(A: np.ndarray, coef, alpha: float = 1.0, beta: float = 0.0, out: np.ndarray | None = None,
                 inplace: bool = False, threads: int = 0) -> np.ndarray:
    """The paper's Algorithm 2 (the NCC code's spin summation) on a dense
    column-major N^d float64 array; a chain is applied as its expanded
    product. Returns B (``A`` itself when ``inplace``)."""
    d = A.ndim
    if A.dtype != np.float64 or not A.flags.f_contiguous or len(set(A.shape)) != 1:
        raise ValueError("A must be a column-major float64 N^d array")
    c = np.ascontiguousarray(np.asarray(coef, dtype=np.float64))
    if c.ndim == 1:
        c = c[None, :]
    if c.ndim != 2 or c.shape[1] != math.factorial(d):
        raise ValueError("coefficient chain must have d! columns")
    if inplace:
        B = A
    elif out is None:
        B = np.zeros(A.shape, dtype=np.float64, order="F")
    else:
        B = out
        if B.shape != A.shape or B.dtype != np.float64 or not B.flags.f_contiguous:
            raise ValueError("out must be a column-major float64 array of A's shape")
    rc = _load().spinsum_alg2(d, A.shape[0], A.ctypes.data, B.ctypes.data, c.ctypes.data, c.shape[0],
                              float(alpha), float(beta), int(threads))
    if rc != 0:
        raise ValueError(f"spinsum_alg2 failed ({rc})")
    return B
