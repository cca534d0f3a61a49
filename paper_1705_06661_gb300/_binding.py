"""ctypes binding of the C-ABI in include/spinsum.h.

Argument marshalling only: every function here forwards to the entry point
of the same name in _build/libspinsum.so and turns a negative status into a
SpinsumError carrying spinsum_last_error(). There is no fallback: if the
library is missing, importing this module raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

SPINSUM_OK = 0
SPINSUM_ERR_ARG = -1
SPINSUM_ERR_ALIAS = -2
SPINSUM_ERR_UNSUPPORTED = -3
SPINSUM_ERR_CUDA = -4
SPINSUM_ERR_TIMEOUT = -5
SPINSUM_ERR_DEVICE = -6

SPINSUM_F64 = 0
SPINSUM_F32 = 1

SPINSUM_EXPANDED = 0
SPINSUM_FACTORIZED = 1
SPINSUM_ADJOINT = 2
SPINSUM_STRICT = 4
SPINSUM_TMA = 8
SPINSUM_STATIC_MAX_PROBLEMS = 64

_STATUS_NAMES = {
    -1: "SPINSUM_ERR_ARG", -2: "SPINSUM_ERR_ALIAS", -3: "SPINSUM_ERR_UNSUPPORTED", -4: "SPINSUM_ERR_CUDA",
    -5: "SPINSUM_ERR_TIMEOUT", -6: "SPINSUM_ERR_DEVICE",
}


class SpinsumError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_I64P = ctypes.POINTER(ctypes.c_int64)
_VP = ctypes.c_void_p


class spinsum_problem(ctypes.Structure):
    _fields_ = [
        ("d", ctypes.c_int),
        ("ext", ctypes.c_int64 * 8),
        ("A", _VP),
        ("lda", ctypes.c_int64 * 8),
        ("B", _VP),
        ("ldb", ctypes.c_int64 * 8),
        ("coef", _VP),
        ("nfactors", ctypes.c_int),
        ("mode", ctypes.c_int),
        ("alpha", ctypes.c_double),
        ("beta", ctypes.c_double),
        ("inplace", ctypes.c_int),
    ]


def _load() -> ctypes.CDLL:
    path = _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"spinsum CUDA library not built ({path}); run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    sig = [ctypes.c_int, _I64P, _VP, _I64P, _VP, _I64P, _VP, ctypes.c_int, ctypes.c_int, ctypes.c_double,
           ctypes.c_double, ctypes.c_int, _VP]
    for name in ("spinsum_2d", "spinsum_3d", "spinsum_4d"):
        f = getattr(lib, name)
        f.argtypes = sig
        f.restype = ctypes.c_int
    hsig = sig[:-1] + [_VP, ctypes.c_size_t, _VP]
    for name in ("spinsum_2d_host", "spinsum_3d_host", "spinsum_4d_host"):
        f = getattr(lib, name)
        f.argtypes = hsig
        f.restype = ctypes.c_int
    lib.spinsum_plan_create.argtypes = [ctypes.POINTER(_VP), ctypes.POINTER(spinsum_problem), ctypes.c_int,
                                        ctypes.c_int, ctypes.c_int, _VP]
    lib.spinsum_plan_create.restype = ctypes.c_int
    lib.spinsum_plan_execute.argtypes = [_VP, _VP]
    lib.spinsum_plan_execute.restype = ctypes.c_int
    lib.spinsum_plan_destroy.argtypes = [_VP]
    lib.spinsum_plan_destroy.restype = ctypes.c_int
    lib.spinsum_plan_describe.argtypes = [_VP]
    lib.spinsum_plan_describe.restype = ctypes.c_char_p
    lib.spinsum_batch_static.argtypes = [ctypes.POINTER(spinsum_problem), ctypes.c_int, ctypes.c_int, _VP]
    lib.spinsum_batch_static.restype = ctypes.c_int
    lib.spinsum_check_status.argtypes = [_VP]
    lib.spinsum_check_status.restype = ctypes.c_int
    lib.spinsum_last_error.argtypes = []
    lib.spinsum_last_error.restype = ctypes.c_char_p
    lib.spinsum_launch_count.argtypes = [ctypes.c_int]
    lib.spinsum_launch_count.restype = ctypes.c_int64
    lib.spinsum_version.argtypes = []
    lib.spinsum_version.restype = ctypes.c_char_p
    lib.spinsum_unpack.argtypes = [ctypes.c_int, ctypes.c_int, _I64P, _VP, _I64P, _VP, _I64P, _VP]
    lib.spinsum_unpack.restype = ctypes.c_int
    lib.spinsum_pack.argtypes = [ctypes.c_int, ctypes.c_int, _I64P, _VP, _I64P, _VP, _I64P, _VP]
    lib.spinsum_pack.restype = ctypes.c_int
    lib.spinsum_contract.argtypes = [ctypes.c_int, _I64P, _VP, _VP, ctypes.c_int, ctypes.c_int, _VP, ctypes.c_int64,
                                     ctypes.c_int64, _VP, ctypes.c_int64, _VP]
    lib.spinsum_contract.restype = ctypes.c_int
    return lib


lib = _load()
LIBRARY_PATH = _build.LIB


def spinsum_last_error() -> str:
    return lib.spinsum_last_error().decode()


def _check(status: int) -> int:
    if status != SPINSUM_OK:
        raise SpinsumError(status, spinsum_last_error())
    return status


def _i64(a) -> ctypes.Array:
    a = [int(x) for x in a]
    return (ctypes.c_int64 * len(a))(*a)


def _coef(coef) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(coef, dtype=np.float64))


def _call(fn, n, dtype, ext, A, lda, B, ldb, coef, nfactors, mode, alpha, beta, inplace, stream):
    if len(ext) != n or len(lda) != n or len(ldb) != n:
        raise ValueError(f"expected {n} extents and strides")
    c = _coef(coef)
    return _check(fn(int(dtype), _i64(ext), _VP(A), _i64(lda), _VP(B), _i64(ldb), _VP(c.ctypes.data),
                     int(nfactors), int(mode), float(alpha), float(beta), int(inplace), _VP(stream)))


def spinsum_unpack(d, dtype, ext, P, ldp, B, ldb, stream) -> int:
    """spinsum_unpack of the C-ABI; P, B and stream are integer addresses."""
    if len(ext) != 2 * d or len(ldb) != 2 * d or len(ldp) != d + 1:
        raise ValueError("expected 2d extents and B strides, d + 1 P strides")
    return _check(lib.spinsum_unpack(int(d), int(dtype), _i64(ext), _VP(P), _i64(ldp), _VP(B), _i64(ldb),
                                     _VP(stream)))


def spinsum_pack(d, dtype, ext, B, ldb, P, ldp, stream) -> int:
    """spinsum_pack of the C-ABI; B, P and stream are integer addresses."""
    if len(ext) != 2 * d or len(ldb) != 2 * d or len(ldp) != d + 1:
        raise ValueError("expected 2d extents and B strides, d + 1 P strides")
    return _check(lib.spinsum_pack(int(d), int(dtype), _i64(ext), _VP(B), _i64(ldb), _VP(P), _i64(ldp),
                                   _VP(stream)))


def spinsum_contract(d, ext, A, coef, nfactors, mode, W, Y, ldw, C, ldc, stream) -> int:
    """spinsum_contract of the C-ABI; A, W, C and stream are integer addresses;
    coef None contracts A itself."""
    if len(ext) != 2 * d:
        raise ValueError("expected 2d extents")
    c = None if coef is None else _coef(coef)
    return _check(lib.spinsum_contract(int(d), _i64(ext), _VP(A), _VP(None if c is None else c.ctypes.data),
                                       int(nfactors), int(mode), _VP(W), int(Y), int(ldw), _VP(C), int(ldc),
                                       _VP(stream)))


def spinsum_2d(dtype, ext, A, lda, B, ldb, coef, nfactors, mode, alpha, beta, inplace, stream) -> int:
    """spinsum_2d of the C-ABI; A, B and stream are integer addresses."""
    return _call(lib.spinsum_2d, 4, dtype, ext, A, lda, B, ldb, coef, nfactors, mode, alpha, beta, inplace, stream)


def spinsum_3d(dtype, ext, A, lda, B, ldb, coef, nfactors, mode, alpha, beta, inplace, stream) -> int:
    """spinsum_3d of the C-ABI; A, B and stream are integer addresses."""
    return _call(lib.spinsum_3d, 6, dtype, ext, A, lda, B, ldb, coef, nfactors, mode, alpha, beta, inplace, stream)


def spinsum_4d(dtype, ext, A, lda, B, ldb, coef, nfactors, mode, alpha, beta, inplace, stream) -> int:
    """spinsum_4d of the C-ABI; A, B and stream are integer addresses."""
    return _call(lib.spinsum_4d, 8, dtype, ext, A, lda, B, ldb, coef, nfactors, mode, alpha, beta, inplace, stream)


def _call_host(fn, n, dtype, ext, A, lda, B, ldb, coef, nfactors, mode, alpha, beta, inplace, ws, ws_bytes,
               stream):
    if len(ext) != n or len(lda) != n or len(ldb) != n:
        raise ValueError(f"expected {n} extents and strides")
    c = _coef(coef)
    return _check(fn(int(dtype), _i64(ext), _VP(A), _i64(lda), _VP(B), _i64(ldb), _VP(c.ctypes.data),
                     int(nfactors), int(mode), float(alpha), float(beta), int(inplace), _VP(ws),
                     ctypes.c_size_t(int(ws_bytes)), _VP(stream)))


def spinsum_2d_host(dtype, ext, A, lda, B, ldb, coef, nfactors, mode, alpha, beta, inplace, workspace,
                    workspace_bytes, stream) -> int:
    """spinsum_2d_host of the C-ABI; A and B are host addresses, workspace a device address."""
    return _call_host(lib.spinsum_2d_host, 4, dtype, ext, A, lda, B, ldb, coef, nfactors, mode, alpha, beta,
                      inplace, workspace, workspace_bytes, stream)


def spinsum_3d_host(dtype, ext, A, lda, B, ldb, coef, nfactors, mode, alpha, beta, inplace, workspace,
                    workspace_bytes, stream) -> int:
    """spinsum_3d_host of the C-ABI; A and B are host addresses, workspace a device address."""
    return _call_host(lib.spinsum_3d_host, 6, dtype, ext, A, lda, B, ldb, coef, nfactors, mode, alpha, beta,
                      inplace, workspace, workspace_bytes, stream)


def spinsum_4d_host(dtype, ext, A, lda, B, ldb, coef, nfactors, mode, alpha, beta, inplace, workspace,
                    workspace_bytes, stream) -> int:
    """spinsum_4d_host of the C-ABI; A and B are host addresses, workspace a device address."""
    return _call_host(lib.spinsum_4d_host, 8, dtype, ext, A, lda, B, ldb, coef, nfactors, mode, alpha, beta,
                      inplace, workspace, workspace_bytes, stream)


def spinsum_check_status(stream) -> int:
    return _check(lib.spinsum_check_status(_VP(stream)))


def spinsum_launch_count(reset: bool = False) -> int:
    return int(lib.spinsum_launch_count(int(bool(reset))))


def spinsum_version() -> str:
    return lib.spinsum_version().decode()


def spinsum_plan_create(problems, dtype, allow_tuning_runs, stream):
    """problems: list of spinsum_problem; returns an opaque plan handle."""
    arr = (spinsum_problem * len(problems))(*problems)
    h = _VP()
    _check(lib.spinsum_plan_create(ctypes.byref(h), arr, len(problems), int(dtype), int(allow_tuning_runs),
                                   _VP(stream)))
    return h


def spinsum_batch_static(problems, dtype, stream) -> int:
    """problems: list of spinsum_problem; runs the batch without allocating device memory."""
    arr = (spinsum_problem * len(problems))(*problems)
    return _check(lib.spinsum_batch_static(arr, len(problems), int(dtype), _VP(stream)))


def spinsum_plan_execute(plan, stream) -> int:
    return _check(lib.spinsum_plan_execute(plan, _VP(stream)))


def spinsum_plan_destroy(plan) -> int:
    return _check(lib.spinsum_plan_destroy(plan))


def spinsum_plan_describe(plan) -> str:
    return lib.spinsum_plan_describe(plan).decode()
