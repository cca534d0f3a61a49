"""Seeded synthetic workloads shared by the oracle side and the GPU side.

This package holds no part of the spin-summation arithmetic: it produces input
tensors, coefficient vectors (the operators of the paper's Table II as data,
and seeded random sets) and the shapes of the benchmark configurations.

Generator: SplitMix64 (Steele, Lea & Flood 2014) used counter-based, draw i of
seed s = mix64(s + (i + 1) * 0x9E3779B97F4A7C15), one draw per tensor element
in column-major linear order.
  uniform  : (x >> 11) * 2^-53 * 2 - 1          in [-1, 1)
  integer  : ((x >> 32) mod 7) - 3               in {-3, ..., 3}
  coef     : [-2, -1, 1, 2, 4][(x >> 32) mod 5]  one draw per permutation, lex order

Coefficient vectors are indexed by the permutations of S_d in lexicographic
one-line order (id first), the order in which the paper enumerates S_3
(Algorithms 2 and 4). Python's itertools.permutations yields exactly this order.
"""
from __future__ import annotations

import ctypes
import itertools
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libwlrng.so")

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


# ----------------------------------------------------------------------------
# generator
# ----------------------------------------------------------------------------
def build(verbose: bool = False) -> str:
    """Compile the C generator (OpenMP) into workloads/_build/libwlrng.so."""
    os.makedirs(_BUILD, exist_ok=True)
    src = os.path.join(_HERE, "splitmix.c")
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", _SO, src]
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
        for name, ptr in (("wl_draw_u64", ctypes.c_void_p), ("wl_uniform_f64", ctypes.c_void_p),
                          ("wl_int7_f64", ctypes.c_void_p)):
            fn = getattr(lib, name)
            fn.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64, ptr]
            fn.restype = None
        _lib = lib
    return _lib


def draws_numpy(seed: int, n: int, start: int = 0) -> np.ndarray:
    """Reference numpy implementation of the counter-based SplitMix64 draws."""
    with np.errstate(over="ignore"):
        i = np.arange(start + 1, start + n + 1, dtype=np.uint64)
        z = np.uint64(seed) + i * GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def draws(seed: int, n: int, start: int = 0) -> np.ndarray:
    out = np.empty(n, dtype=np.uint64)
    _load().wl_draw_u64(seed, start, n, out.ctypes.data)
    return out


def _shape_n(shape) -> int:
    n = 1
    for s in shape:
        n *= int(s)
    return n


def uniform(seed: int, shape, start: int = 0) -> np.ndarray:
    """Column-major (Fortran-order) float64 tensor, uniform in [-1, 1)."""
    n = _shape_n(shape)
    flat = np.empty(n, dtype=np.float64)
    if n:
        _load().wl_uniform_f64(seed, start, n, flat.ctypes.data)
    return flat.reshape(tuple(shape), order="F")


def integers(seed: int, shape, start: int = 0) -> np.ndarray:
    """Column-major float64 tensor of integers in {-3..3}."""
    n = _shape_n(shape)
    flat = np.empty(n, dtype=np.float64)
    if n:
        _load().wl_int7_f64(seed, start, n, flat.ctypes.data)
    return flat.reshape(tuple(shape), order="F")


def uniform_numpy(seed: int, n: int, start: int = 0) -> np.ndarray:
    x = draws_numpy(seed, n, start)
    return (x >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0) * 2.0 - 1.0


def integers_numpy(seed: int, n: int, start: int = 0) -> np.ndarray:
    x = draws_numpy(seed, n, start)
    return ((x >> np.uint64(32)) % np.uint64(7)).astype(np.int64).astype(np.float64) - 3.0


# ----------------------------------------------------------------------------
# coefficient vectors (operators as data)
# ----------------------------------------------------------------------------
def perms(d: int):
    """S_d in lexicographic one-line order, 1-based tuples, id first."""
    return list(itertools.permutations(range(1, d + 1)))


def perm_name(p) -> str:
    return "".join(str(x) for x in p)


def coef_vector(d: int, terms) -> np.ndarray:
    """terms: iterable of (coefficient, one-line name like '213'); returns a
    length-d! float64 vector in lexicographic order. Repeated names add up."""
    idx = {perm_name(p): k for k, p in enumerate(perms(d))}
    v = np.zeros(len(idx), dtype=np.float64)
    for c, name in terms:
        v[idx[name]] += c
    return v


def _two_minus(d: int, names) -> list:
    ident = "".join(str(i) for i in range(1, d + 1))
    return [(2.0, ident)] + [(-1.0, n) for n in names]


# Table II of the paper (Sec. 5.1): each row is a factor chain [F_1, ..., F_k]
# with B = F_1(F_2(...F_k(A))); "2" is twice the identity. Rows 8-11, 16 and 17
# are garbled in the extracted text. TABLE2 holds the reading in which every
# inner factor is "2 minus the transpositions that involve one index" and every
# outer factor is "2 minus a pair of transpositions of the remaining indices";
# TABLE2_PRINTED holds the rows exactly as printed, as extra coefficient sets.
_T2 = {
    1: [["213"], ["321", "132"]],
    2: [["321", "132"]],
    3: [["213", "132"]],
    4: [["213", "321"]],
    5: [["2134"], ["3214", "1324"], ["4231", "1432", "1243"]],
    6: [["3214", "1324"], ["4231", "1432", "1243"]],
    7: [["2134", "1324"], ["4231", "1432", "1243"]],
    8: [["2134", "3214"], ["4231", "1432", "1243"]],
    9: [["4231", "1432"], ["3214", "1324", "1243"]],
    10: [["2134", "1432"], ["3214", "1324", "1243"]],
    11: [["2134", "4231"], ["3214", "1324", "1243"]],
    12: [["4231", "1243"], ["2134", "1324", "1432"]],
    13: [["3214", "1243"], ["2134", "1324", "1432"]],
    14: [["3214", "4231"], ["2134", "1324", "1432"]],
    15: [["1432", "1243"], ["2134", "3214", "4231"]],
    16: [["1324", "1243"], ["2134", "3214", "4231"]],
    17: [["1324", "1432"], ["2134", "3214", "4231"]],
    18: [["4231", "1432", "1243"]],
    19: [["3214", "1324", "1243"]],
    20: [["2134", "1324", "1432"]],
    21: [["2134", "3214", "4231"]],
}
# rows whose printed text differs from the reading above
_T2_PRINTED = {
    8: [["2134", "3214"], ["4231", "1432", "4231"]],
    9: [["4231", "1432"], ["3214", "1324", "4231"]],
    10: [["2134", "1432"], ["3214", "1324", "4231"]],
    11: [["2134", "4231"], ["3214", "1324", "1234"]],
    16: [["1432", "1243"], ["2134", "3214", "4231"]],
    17: [["1432", "1432"], ["2134", "3214", "4231"]],
}


def table2_dim(row: int) -> int:
    return 3 if row <= 4 else 4


def table2(row: int, printed: bool = False) -> np.ndarray:
    """Factor chain of Table II row `row` as an array [nfactors, d!]."""
    d = table2_dim(row)
    spec = _T2_PRINTED[row] if (printed and row in _T2_PRINTED) else _T2[row]
    return np.stack([coef_vector(d, _two_minus(d, f)) for f in spec])


TABLE2_ROWS = list(range(1, 22))
TABLE2_GARBLED = sorted(_T2_PRINTED)

COEF_VALUES = np.array([-2.0, -1.0, 1.0, 2.0, 4.0])


def random_coef(d: int, seed: int) -> np.ndarray:
    """Seeded random coefficient set, one value from {-2,-1,1,2,4} per
    permutation in lex order; shape [1, d!]."""
    n = len(perms(d))
    x = draws(seed, n)
    return COEF_VALUES[((x >> np.uint64(32)) % np.uint64(5)).astype(np.int64)][None, :].copy()


# ----------------------------------------------------------------------------
# benchmark configurations
# ----------------------------------------------------------------------------
@dataclass
class Problem:
    """One spin summation: spectator extents (fastest first) then d permuted
    extents; column-major dense storage; data seed; coefficient chain."""
    d: int
    spec: tuple
    O: int
    seed: int
    coef: np.ndarray
    name: str = ""

    @property
    def shape(self):
        return tuple(self.spec) + (self.O,) * self.d

    @property
    def n(self) -> int:
        return _shape_n(self.shape)


@dataclass
class Config:
    name: str
    d: int
    spec: tuple
    O: int
    seed: int
    sets: dict = field(default_factory=dict)


def config1() -> Config:
    """3D, all six extents 8, uniform seed 0 (+ an integer copy)."""
    sets = {f"row{r}": table2(r) for r in (1, 2, 3, 4)}
    sets["random"] = random_coef(3, 101)
    return Config("3d-8^6", 3, (8, 8, 8), 8, 0, sets)


def config2() -> Config:
    """3D, spectators 48^3, permuted 16^3 (453M doubles, 3.6 GB)."""
    sets = {f"row{r}": table2(r) for r in (1, 2, 3, 4)}
    sets["random"] = random_coef(3, 102)
    return Config("3d-48^3x16^3", 3, (48, 48, 48), 16, 1, sets)


def config3() -> Config:
    """4D, all eight extents 12 (430M doubles, 3.4 GB)."""
    sets = {f"row{r}": table2(r) for r in range(5, 22)}
    sets["random"] = random_coef(4, 103)
    return Config("4d-12^8", 4, (12, 12, 12, 12), 12, 2, sets)


def config4_blocks(nblocks: int = 64):
    """64 independent 3D blocks: V = 16 + (r mod 25) for a,b,c and
    O = 6 + (r mod 9) for i,j,k, r = draws of seed 3; block data seed 1000+b;
    coefficient sets cycle rows 1-4 and a random set (seed 200+b)."""
    x = draws(3, 2 * nblocks) >> np.uint64(32)
    out = []
    for b in range(nblocks):
        V = 16 + int(x[2 * b] % np.uint64(25))
        O = 6 + int(x[2 * b + 1] % np.uint64(9))
        k = b % 5
        coef = table2(k + 1) if k < 4 else random_coef(3, 200 + b)
        out.append(Problem(3, (V, V, V), O, 1000 + b, coef, f"block{b}"))
    return out


def config5() -> Config:
    """4D differentiable case, all extents 10; A seed 4, cotangent seed 5."""
    sets = {"random": random_coef(4, 105), "row5": table2(5)}
    return Config("4d-10^8", 4, (10, 10, 10, 10), 10, 4, sets)


COTANGENT_SEED_CFG5 = 5
