"""The Klein four-group transform of the 4D orbit operators (host tables and
weights), checked on the CPU against the orbit operator's definition.

For a 4D orbit with canonical label tuple t0, output member u of the
summation is sum_sigma a_sigma x[u o sigma] (Def. 2-3): the dense operator
M[u][v] = sum of a_sigma over sigma with t_u o sigma = t_v. The library
applies it on the freely transformable patterns as x^ = T x (4-point
Walsh-Hadamard transforms over the V-orbits), y^ = W x^ with W sparse, and
y = T^T y^ / 4. Here T and the sparsity come from the library's tables, W
from the planner, and M is built independently from the definition, and
T^T W T = 4 M must hold exactly for Table II rows and random integer sets.
The row 1-norms of W stay within sum|a| (the bound behind the limb widths).
"""
import ctypes
import itertools
import math

import numpy as np
import pytest

import workloads as wl

LABELS = [(0, 1, 2, 3), (0, 0, 1, 2), (0, 1, 1, 2), (0, 1, 2, 2), (0, 0, 1, 1), (0, 0, 0, 1), (0, 1, 1, 1),
          (0, 0, 0, 0)]
PERMS = list(itertools.permutations(range(4)))
KF_WHT = 8
WH_TOTAL = 326


@pytest.fixture(scope="module")
def lib():
    from paper_1705_06661_gb300 import _binding
    return _binding._load()


def members(P):
    out = []
    for p in PERMS:
        t = tuple(LABELS[P][p[m]] for m in range(4))
        if t not in out:
            out.append(t)
    return out


def dense_operator(P, a):
    mem = members(P)
    M = np.zeros((len(mem), len(mem)), dtype=np.int64)
    for u, t in enumerate(mem):
        for s, p in enumerate(PERMS):
            M[u, mem.index(tuple(t[p[m]] for m in range(4)))] += int(a[s])
    return M


def tables(lib, P):
    out = np.zeros(223, dtype=np.int32)
    f = lib.ss_debug_wht_tables
    f.argtypes = [ctypes.c_int, ctypes.c_void_p]
    f.restype = ctypes.c_int
    assert f(P, out.ctypes.data) == 0
    ok, m, nb = out[0], out[1], out[2]
    orb = out[3:27].reshape(6, 4)
    nnz = out[27:51]
    col = out[51:195].reshape(24, 6)
    woff = out[195:220]
    return bool(ok), int(m), int(nb), orb, nnz, col, woff


def plan_wh(lib, coef, alpha=1.0, mode=0):
    coef = np.ascontiguousarray(np.atleast_2d(np.asarray(coef, dtype=np.float64)))
    info = np.zeros(4, dtype=np.int64)
    wh = np.zeros(WH_TOTAL, dtype=np.int32)
    f = lib.ss_debug_plan_wh
    P = ctypes.c_void_p
    f.argtypes = [ctypes.c_int, ctypes.c_int, P, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, P, P]
    f.restype = ctypes.c_int
    assert f(6, 4, coef.ctypes.data, coef.shape[0], mode, alpha, 0.0, info.ctypes.data, wh.ctypes.data) == 0
    return {"flags": int(info[0]), "W": int(info[1]), "kdrop": int(info[2]), "arith": int(info[3])}, wh


def chi(k, vi):
    return -1 if bin(k & vi).count("1") % 2 else 1


def test_transformable_patterns(lib):
    want = {0: (True, 24), 1: (True, 12), 2: (True, 12), 3: (True, 12), 4: (False, 6), 5: (True, 4), 6: (True, 4),
            7: (False, 1)}
    for P in range(8):
        ok, m, nb, orb, nnz, col, woff = tables(lib, P)
        assert (ok, m) == want[P]
        if not ok:
            continue
        assert nb * 4 == m
        # the V-orbits partition the members; member orb[o][vi] is orb[o][0] o v_vi
        assert sorted(orb[:nb].ravel().tolist()) == list(range(m))
        mem = members(P)
        klein = [(0, 1, 2, 3), (1, 0, 3, 2), (2, 3, 0, 1), (3, 2, 1, 0)]
        for o in range(nb):
            t = mem[orb[o][0]]
            for vi, v in enumerate(klein):
                assert mem[orb[o][vi]] == tuple(t[v[k]] for k in range(4))
        assert int(woff[m]) == int(nnz[:m].sum())
        assert max(nnz[:m]) <= 6


def _check(lib, coef, P_list=range(8)):
    import oracle
    a = oracle.expand(4, coef)
    info, wh = plan_wh(lib, coef)
    lx = np.abs(a).sum()
    scale = 1
    while not np.all(np.equal(np.mod(a * scale, 1), 0)):
        scale *= 2
    ai = np.round(a * scale).astype(np.int64)
    assert info["arith"] == 0
    if np.abs(ai).sum() > 63:
        assert not info["flags"] & KF_WHT
        return False
    assert info["flags"] & KF_WHT and info["W"] == 24
    off = 0
    for P in P_list:
        ok, m, nb, orb, nnz, col, woff = tables(lib, P)
        if not ok:
            continue
        T = np.zeros((m, m), dtype=np.int64)
        for o in range(nb):
            for k in range(4):
                for vi in range(4):
                    T[4 * o + k, orb[o][vi]] = chi(k, vi)
        Wm = np.zeros((m, m), dtype=np.int64)
        for i in range(m):
            for q in range(nnz[i]):
                Wm[i, col[i][q]] += wh[off + woff[i] + q]
        np.testing.assert_array_equal(T.T @ Wm @ T, 4 * dense_operator(P, ai), err_msg=f"pattern {P}")
        assert np.abs(Wm).sum(axis=1).max() <= np.abs(ai).sum()
        off += int(woff[m])
    assert lx * scale == np.abs(ai).sum()
    return True


@pytest.mark.parametrize("row", range(5, 22))
def test_table2_rows(lib, row):
    assert _check(lib, wl.table2(row))


def test_random_sets(lib):
    used = 0
    for seed in range(100, 140):
        used += _check(lib, wl.random_coef(4, seed))
    assert used >= 30     # most {-2,-1,1,2,4} sets have sum |a| <= 63


def test_eligibility(lib):
    big = np.full((1, 24), 3.0)                  # sum |a| = 72 > 63: the dense core
    info, _ = plan_wh(lib, big)
    assert info["arith"] == 0 and not info["flags"] & KF_WHT
    info, _ = plan_wh(lib, wl.table2(5), alpha=0.3)     # alpha not a power of two
    assert not info["flags"] & KF_WHT
    info, _ = plan_wh(lib, wl.table2(5), alpha=-0.25)   # a negative power of two folds into the weights
    assert info["flags"] & KF_WHT
    info, _ = plan_wh(lib, wl.table2(5), mode=4)        # strict FP64
    assert info["arith"] == 1 and not info["flags"] & KF_WHT


def test_dense_core_switch_keeps_the_grid(lib, monkeypatch):
    monkeypatch.setenv("SPINSUM_4D_DENSE_CORE", "1")
    info, _ = plan_wh(lib, wl.table2(5))
    assert info["arith"] == 0 and not info["flags"] & KF_WHT and info["W"] == 24
    monkeypatch.delenv("SPINSUM_4D_DENSE_CORE")
    info, _ = plan_wh(lib, wl.table2(5))
    assert info["flags"] & KF_WHT and info["W"] == 24
