"""ORACLE -- test infrastructure only.

Python wrapper around the plain C oracle in ``spinsum_oracle.c`` (see the
header there for the definitions it follows: Def. 1-4, Eq. 1-6, Algorithms 1
and 3 and Sec. 4.6.5 of the paper). Only the tests, ``__graft_entry__.smoke``
and the CPU-baseline leg of ``bench.py`` may use it; the library's GPU path
never imports it.

Tensors are numpy float64 arrays of any strides; the last ``d`` axes are the
permuted index group, the leading axes are spectators. Coefficient chains are
arrays of shape [nfactors, d!] in lexicographic permutation order, meaning
B = F_1(F_2(...F_k(A))).

Packed antisymmetric storage (``unpack`` / ``pack``) is written here in numpy
from its definition: one value per strictly increasing tuple, indexed by its
colex rank (the combinatorial number system), signs from the inversion count.

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
(copy / single-permutation transposes against numpy's transpose, the paper's
Eq. 7 = Eq. 8 factorization, the Sec. 4.6.2 regularization identity, the
Fig. 1a update formulas, the closed-shell expansion of Table II row 1, brute
force against a dense permutation matrix, invariants of the symmetrizer and
antisymmetrizer, adjoint and composition identities).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")


def build(verbose: bool = False) -> str:
    os.makedirs(_BUILD, exist_ok=True)
    src = os.path.join(_HERE, "spinsum_oracle.c")
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
           "-o", _SO, src]
    if verbose:
        print(" ".join(cmd))
    subprocess.check_call(cmd)
    return _SO


_lib = None
_P = ctypes.c_void_p


def _load():
    global _lib
    if _lib is None:
        if not os.path.exists(_SO):
            build()
        lib = ctypes.CDLL(_SO)
        lib.oracle_perms.argtypes = [ctypes.c_int, _P]
        lib.oracle_perms.restype = ctypes.c_int
        lib.oracle_expand.argtypes = [ctypes.c_int, _P, ctypes.c_int, _P]
        lib.oracle_expand.restype = ctypes.c_int
        lib.oracle_spinsum.argtypes = [ctypes.c_int, ctypes.c_int, _P, _P, _P, _P, _P, _P, ctypes.c_int,
                                       ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int]
        lib.oracle_spinsum.restype = ctypes.c_int
        lib.oracle_spinsum_transpose.argtypes = [ctypes.c_int, ctypes.c_int, _P, _P, _P, _P, ctypes.c_int,
                                                 ctypes.c_double]
        lib.oracle_spinsum_transpose.restype = ctypes.c_int
        lib.oracle_num_threads.argtypes = []
        lib.oracle_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def perms(d: int) -> np.ndarray:
    """S_d in the oracle's lexicographic order, 0-based images, shape [d!, d]."""
    n = math.factorial(d)
    out = np.zeros(n * d, dtype=np.int32)
    _load().oracle_perms(d, out.ctypes.data)
    return out.reshape(n, d)


def _chain(d: int, coef) -> np.ndarray:
    c = np.ascontiguousarray(np.asarray(coef, dtype=np.float64))
    if c.ndim == 1:
        c = c[None, :]
    if c.shape[1] != math.factorial(d):
        raise ValueError("coefficient chain must have d! columns")
    return c


def expand(d: int, coef) -> np.ndarray:
    """Product-rule expansion of a factor chain into one d!-vector."""
    c = _chain(d, coef)
    out = np.zeros(math.factorial(d), dtype=np.float64)
    _load().oracle_expand(d, c.ctypes.data, c.shape[0], out.ctypes.data)
    return out


def _elem_strides(a: np.ndarray) -> np.ndarray:
    return np.array([s // a.itemsize for s in a.strides], dtype=np.int64)


def spinsum(A: np.ndarray, d: int, coef, factorized: bool = False, alpha: float = 1.0, beta: float = 0.0,
            B: np.ndarray | None = None, inplace: bool = False) -> np.ndarray:
    """B = alpha * S(A) + beta * B (or A in place). Returns the output array."""
    if A.dtype != np.float64:
        raise TypeError("oracle works in float64")
    c = _chain(d, coef)
    ext = np.array(A.shape, dtype=np.int64)
    nspec = A.ndim - d
    if inplace:
        B = A
    elif B is None:
        B = np.zeros(A.shape, dtype=np.float64, order="F")
    lda, ldb = _elem_strides(A), _elem_strides(B)
    rc = _load().oracle_spinsum(d, nspec, ext.ctypes.data, A.ctypes.data, lda.ctypes.data, B.ctypes.data,
                                ldb.ctypes.data, c.ctypes.data, c.shape[0], int(bool(factorized)),
                                float(alpha), float(beta), int(bool(inplace)))
    if rc != 0:
        raise ValueError(f"oracle_spinsum failed ({rc})")
    return B


def spinsum_transpose(Y: np.ndarray, d: int, coef, alpha: float = 1.0) -> np.ndarray:
    """X = alpha * S^T(Y) by literal scatter-transposition, dense column-major."""
    c = _chain(d, coef)
    Yf = np.asfortranarray(Y, dtype=np.float64)
    X = np.zeros(Y.shape, dtype=np.float64, order="F")
    ext = np.array(Y.shape, dtype=np.int64)
    rc = _load().oracle_spinsum_transpose(d, Y.ndim - d, ext.ctypes.data, Yf.ctypes.data, X.ctypes.data,
                                          c.ctypes.data, c.shape[0], float(alpha))
    if rc != 0:
        raise ValueError(f"oracle_spinsum_transpose failed ({rc})")
    return X


def colex_rank(t) -> int:
    """Rank of the strictly increasing tuple t among all such tuples in colex
    order: sum_k C(t_k, k + 1) (the combinatorial number system)."""
    return int(sum(math.comb(int(x), k + 1) for k, x in enumerate(t)))


def _inversions(t) -> int:
    return sum(1 for a in range(len(t)) for b in range(a + 1, len(t)) if t[a] > t[b])


def unpack(P: np.ndarray, d: int, O: int) -> np.ndarray:
    """Antisymmetric tensor from its packed form: B[s, t] = (-1)^inv(t) *
    P[s, rank(sorted t)] for t without repeated entries, else 0. P has the
    spectator axes then one packed axis of length C(O, d)."""
    import itertools
    spec = P.shape[:-1]
    B = np.zeros(spec + (O,) * d)
    for t in itertools.product(range(O), repeat=d):
        if len(set(t)) < d:
            continue
        sign = -1.0 if _inversions(t) % 2 else 1.0
        B[(Ellipsis,) + t] = sign * P[..., colex_rank(sorted(t))]
    return B


def pack(B: np.ndarray, d: int) -> np.ndarray:
    """Packed form: P[s, rank(t0)] = B[s, t0] for every strictly increasing t0."""
    import itertools
    O = B.shape[-1]
    spec = B.shape[:-d]
    P = np.zeros(spec + (math.comb(O, d),))
    for t0 in itertools.combinations(range(O), d):
        P[..., colex_rank(t0)] = B[(Ellipsis,) + t0]
    return P


def contract(A: np.ndarray, d: int, coef, W: np.ndarray, factorized: bool = False) -> np.ndarray:
    """Contraction over the permuted index group of the spin-summed tensor:
    C[s, y] = sum_t S(A)[s, t] * W[y, t], the use the summation feeds
    (Sec. 1, Sec. 6); coef None contracts A itself. t is the column-major
    index of the permuted tuple (first permuted index fastest), s that of the
    spectator positions. W has shape (Y, O**d). Returns C with the spectator
    axes then one axis of length Y. Written as the spin summation above
    followed by one matrix product (numpy)."""
    nspec = A.ndim - d
    spec = A.shape[:nspec]
    T = int(np.prod(A.shape[nspec:])) if d else 1
    B = A if coef is None else spinsum(A, d, coef, factorized=factorized)
    S = int(np.prod(spec)) if nspec else 1
    Bm = np.asarray(B).reshape((S, T), order="F")
    C = Bm @ np.asarray(W, dtype=np.float64).T
    return C.reshape(tuple(spec) + (W.shape[0],), order="F")
