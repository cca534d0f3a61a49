"""CPU-only checks of the C-ABI library: it loads, exports every function
that include/spinsum.h declares, rejects bad arguments before touching the
GPU, and its host planner (product rule, orbit counts, choice of arithmetic)
agrees with the oracle and with closed forms. Nothing here launches a kernel."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "_spinsum_build", os.path.join(ROOT, "paper_1705_06661_gb300", "_build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    path = mod.build()
    return ctypes.CDLL(path)


def header_functions():
    txt = open(os.path.join(ROOT, "include", "spinsum.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(spinsum_[a-z0-9_]+)\s*\(", txt)))


def test_exports_every_declared_function(lib):
    names = header_functions()
    assert "spinsum_2d" in names and "spinsum_3d" in names and "spinsum_4d" in names
    assert "spinsum_plan_create" in names
    for n in names:
        assert hasattr(lib, n), n


def test_binding_has_same_names(lib):
    import paper_1705_06661_gb300 as ss
    for n in header_functions():
        assert hasattr(ss, n), n


@pytest.fixture(scope="module")
def ss():
    import paper_1705_06661_gb300 as m
    return m


FAKE_A = 0x7F0000000000
FAKE_B = 0x7F8000000000


def _dense(ext):
    ld, s = [], 1
    for e in ext:
        ld.append(s)
        s *= e
    return ld


@pytest.mark.parametrize("case,code", [
    ("bad_dtype", "ERR_ARG"), ("unequal_extents", "ERR_ARG"), ("negative_extent", "ERR_ARG"),
    ("nan_coef", "ERR_ARG"), ("zero_factors", "ERR_ARG"), ("bad_mode", "ERR_ARG"), ("overlap", "ERR_ALIAS"),
    ("inplace_distinct", "ERR_ALIAS"), ("inplace_strides", "ERR_ALIAS"), ("misaligned", "ERR_ARG"),
    ("strict_f32", "ERR_ARG"), ("null_ptr", "ERR_ARG"), ("negative_stride", "ERR_UNSUPPORTED"),
])
def test_argument_errors_need_no_gpu(ss, case, code):
    ext = [4, 4, 4, 5, 5, 5]
    lda = _dense(ext)
    ldb = list(lda)
    coef = wl.table2(2)
    a, b = FAKE_A, FAKE_B
    dtype, nf, mode, inplace = ss.SPINSUM_F64, 1, 0, 0
    if case == "bad_dtype":
        dtype = 9
    elif case == "unequal_extents":
        ext[5] = 4
    elif case == "negative_extent":
        ext[0] = -1
    elif case == "nan_coef":
        coef = np.array([[np.nan, 0, 0, 0, 0, 0]])
    elif case == "zero_factors":
        nf = 0
    elif case == "bad_mode":
        mode = 64
    elif case == "overlap":
        b = a + 8 * 100
    elif case == "inplace_distinct":
        inplace = 1
    elif case == "inplace_strides":
        inplace, b = 1, a
        ldb[0] = 2
    elif case == "misaligned":
        a += 3
    elif case == "strict_f32":
        dtype, mode = ss.SPINSUM_F32, ss.SPINSUM_STRICT
    elif case == "null_ptr":
        a = 0
    elif case == "negative_stride":
        lda[3] = -lda[3]
    with pytest.raises(ss.SpinsumError, match=code):
        ss.spinsum_3d(dtype, ext, a, lda, b, ldb, coef, nf, mode, 1.0, 0.0, inplace, 0)
    assert ss.spinsum_last_error()


def test_empty_problem_launches_nothing(ss):
    before = ss.spinsum_launch_count()
    ext = [0, 4, 4, 5, 5, 5]
    assert ss.spinsum_3d(ss.SPINSUM_F64, ext, 0, _dense(ext), 0, _dense(ext), wl.table2(1), 2, 1, 1.0, 0.0, 0,
                         0) == 0
    assert ss.spinsum_launch_count() == before


def debug_plan(lib, d, O, V, coef, mode=0, alpha=1.0, beta=0.0):
    coef = np.ascontiguousarray(np.atleast_2d(np.asarray(coef, dtype=np.float64)))
    n = math.factorial(d)
    ex = np.zeros(n)
    info = np.zeros(32, dtype=np.int64)
    ci = np.zeros(8 * 24, dtype=np.int32)
    mp = np.zeros(501, dtype=np.int32)
    f = lib.ss_debug_plan
    f.restype = ctypes.c_int
    P = ctypes.c_void_p
    f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, P, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                  ctypes.c_double, P, P, P, P]
    rc = f(d, O, V, coef.ctypes.data, coef.shape[0], mode, alpha, beta, ex.ctypes.data, info.ctypes.data,
           ci.ctypes.data, mp.ctypes.data)
    assert rc == 0
    keys = ["arith", "W", "kdrop", "nstage", "kernel", "vec", "flags", "cexp", "emin", "emax"]
    out = dict(zip(keys, info[:10].tolist()))
    out["norb"] = info[10:18].tolist()
    out["blocks"] = int(info[18])
    out["k2lf"] = int(info[19])
    return ex, out, ci.reshape(8, 24), mp


@pytest.mark.parametrize("row", wl.TABLE2_ROWS)
def test_host_product_rule_matches_oracle(lib, row):
    import oracle
    d = wl.table2_dim(row)
    ex, info, _, _ = debug_plan(lib, d, 4, 4, wl.table2(row))
    np.testing.assert_array_equal(ex, oracle.expand(d, wl.table2(row)))
    assert info["arith"] == 0          # exact core for every Table II operator
    assert info["W"] >= 24 and info["W"] <= 26


def test_host_product_rule_random_chains(lib):
    import oracle
    for d in (2, 3, 4):
        chain = np.concatenate([wl.random_coef(d, 300 + d), wl.random_coef(d, 310 + d), wl.uniform(320, (1, math.factorial(d)))])
        ex, info, _, _ = debug_plan(lib, d, 4, 4, chain, mode=1)
        np.testing.assert_array_equal(ex, oracle.expand(d, chain))
        assert info["arith"] == 1          # real coefficients: strict core
        assert info["nstage"] == 3


@pytest.mark.parametrize("d,O", [(2, 1), (2, 7), (2, 64), (3, 1), (3, 2), (3, 5), (3, 16), (4, 1), (4, 3), (4, 5),
                                 (4, 12), (4, 40)])
def test_orbit_counts(lib, d, O):
    """orbits per equality pattern are the choices of distinct values; the
    orbit members cover the O^d tuples exactly once."""
    _, info, _, _ = debug_plan(lib, d, O, 8, wl.random_coef(d, 1))
    norb = info["norb"]
    sizes = {2: [2, 1], 3: [6, 3, 3, 1], 4: [24, 12, 12, 12, 6, 4, 4, 1]}[d]
    assert sum(n * m for n, m in zip(norb, sizes)) == O ** d
    # canonical tuples i <= j <= k (<= l): C(O + d - 1, d)
    assert sum(norb[:len(sizes)]) == math.comb(O + d - 1, d)
    if d == 4 and O == 5:
        assert sum(norb) == 70   # the 70 tetrahedral tasks of a 40^4 tensor with 8^4 blocks (Sec. 4.5)


def test_orbit_matrices(lib):
    """rows of every degenerate pattern's orbit matrix sum to sum(alpha);
    the 1-member pattern's matrix is exactly sum(alpha)."""
    for d in (2, 3, 4):
        a = wl.random_coef(d, 400 + d)
        _, info, ci, mp = debug_plan(lib, d, 6, 8, a)
        np.testing.assert_array_equal(ci[0, :math.factorial(d)], a[0].astype(np.int32))
        sizes = {2: [2, 1], 3: [6, 3, 3, 1], 4: [24, 12, 12, 12, 6, 4, 4, 1]}[d]
        off = 0
        for m in sizes[1:]:
            M = mp[off:off + m * m].reshape(m, m)
            assert (M.sum(axis=1) == a.sum()).all()
            off += m * m
        assert mp[off - 1] == a.sum()


def test_exact_path_parameters(lib):
    _, info, ci, _ = debug_plan(lib, 3, 16, 48, wl.table2(1), mode=1, alpha=-0.5)
    assert info["arith"] == 0 and info["nstage"] == 2
    # L = |2 - pi213|_1 * |2 - pi321 - pi132|_1 = 3 * 4 = 12 -> W = 26, then rounding to < 2^50
    assert info["W"] == 26 and info["kdrop"] >= 1
    # sign of alpha folded into the last-applied stage (the outer factor 2 - pi213)
    assert ci[1, 0] == -2 and ci[0, 0] == 2
    _, info, _, _ = debug_plan(lib, 3, 16, 48, wl.table2(1), alpha=3.0)
    assert info["flags"] & 2                  # alpha not a power of two: multiplied at the end
    big = np.arange(1.0, 25.0)[None, :]       # |alpha|_1 = 300 > 127: strict core
    _, info, _, _ = debug_plan(lib, 4, 4, 4, big)
    assert info["arith"] == 1
    _, info, _, _ = debug_plan(lib, 4, 4, 4, wl.table2(5), mode=4)
    assert info["arith"] == 1                 # SPINSUM_STRICT


def test_launch_shape(lib):
    # aligned dense spectator blocks: the register orbit stream (kernel 0) with 16-byte vectors for 3D
    _, info, _, _ = debug_plan(lib, 3, 16, 48, wl.table2(1))
    assert info["kernel"] == 0 and info["vec"] == 2
    _, info, _, _ = debug_plan(lib, 4, 12, 12, wl.table2(5))
    assert info["kernel"] == 0 and info["vec"] == 1
    # SPINSUM_TMA (8) selects the TMA-staged orbit stream (kernel 2) for 3D, not for 4D or strict
    _, info, _, _ = debug_plan(lib, 3, 16, 48, wl.table2(1), mode=8)
    assert info["kernel"] == 2
    _, info, _, _ = debug_plan(lib, 4, 12, 12, wl.table2(5), mode=8)
    assert info["kernel"] == 0
    _, info, _, _ = debug_plan(lib, 3, 16, 48, wl.table2(1), mode=8 | 4)
    assert info["kernel"] == 0
    # odd spectator block (S = 27 * 27 * 27 is odd): no 16-byte runs, scalar register path
    _, info, _, _ = debug_plan(lib, 3, 8, 27, wl.table2(1))
    assert info["kernel"] == 0 and info["vec"] == 1
    _, info, _, _ = debug_plan(lib, 3, 16, 3, wl.table2(1))   # 27 spectators: general kernel
    assert info["kernel"] == 1
    # the paper's N^d layout (no spectators, first permuted index at stride 1): tiled kernel
    # CTAs: F^d per sorted tuple of coarse blocks (F tiles per coarse edge)
    for d, N, bl in ((2, 1000, 32), (3, 344, 8), (4, 80, 4)):
        coef = {2: np.array([[2.0, -1.0]]), 3: wl.table2(1), 4: wl.table2(5)}[d]
        _, info, _, _ = debug_plan(lib, d, N, 1, coef)
        F = 1 << info["k2lf"]
        nc = -(-(-(-N // bl)) // F)
        assert info["kernel"] == 3 and info["blocks"] == math.comb(nc + d - 1, d) * F ** d


@pytest.mark.parametrize("case,code", [("bad_d", -1), ("bad_dtype", -1), ("unequal_extents", -1),
                                       ("sparse_spectators", -3), ("short_packed_stride", -1),
                                       ("overlap", -2), ("extent_too_large", -3)])
def test_pack_argument_errors_need_no_gpu(ss, case, code):
    """spinsum_unpack / spinsum_pack validate before touching a device."""
    d = 3
    ext = [3, 3, 3, 6, 6, 6]
    ldb = _dense(ext)
    S = 27
    ldp = [1, 3, 9, S]
    P, B = FAKE_A, FAKE_B
    dtype = ss.SPINSUM_F64
    if case == "bad_d":
        d, ext, ldb, ldp = 5, ext + [6, 6, 6, 6], _dense(ext + [6, 6, 6, 6]), ldp + [1, 1]
    elif case == "bad_dtype":
        dtype = 7
    elif case == "unequal_extents":
        ext[5] = 5
    elif case == "sparse_spectators":
        ldb[1] = 4
    elif case == "short_packed_stride":
        ldp[3] = S - 1
    elif case == "overlap":
        B = P + 8 * 10
    elif case == "extent_too_large":
        ext[3] = ext[4] = ext[5] = 5000
        ldb = _dense(ext)
    for fn in (lambda: ss.spinsum_unpack(d, dtype, ext, P, ldp, B, ldb, 0),
               lambda: ss.spinsum_pack(d, dtype, ext, B, ldb, P, ldp, 0)):
        with pytest.raises(ss.SpinsumError) as e:
            fn()
        assert e.value.status == code, (case, e.value)


@pytest.mark.parametrize("case,code", [("bad_d", "ERR_ARG"), ("neg_y", "ERR_ARG"), ("ldw", "ERR_ARG"),
                                       ("ldc", "ERR_ARG"), ("mode", "ERR_ARG"), ("alias_a", "ERR_ALIAS"),
                                       ("alias_w", "ERR_ALIAS"), ("null", "ERR_ARG"), ("misaligned", "ERR_ARG")])
def test_contract_argument_errors(ss, case, code):
    """spinsum_contract rejects bad arguments on the host, before any launch."""
    d, ext = 3, [4, 4, 4, 5, 5, 5]
    S, T, Y = 64, 125, 6
    A, W, C = FAKE_A, FAKE_B, FAKE_B + 1 << 20
    ldw, ldc, mode, dd = Y, S, 1, d
    if case == "bad_d":
        dd, ext = 5, ext + [5, 5, 5, 5]
    elif case == "neg_y":
        Y = -1
    elif case == "ldw":
        ldw = Y - 1
    elif case == "ldc":
        ldc = S - 1
    elif case == "mode":
        mode = 1 | ss.SPINSUM_TMA
    elif case == "alias_a":
        C = A + 8 * 100
    elif case == "alias_w":
        C = W + 8 * 10
    elif case == "null":
        W = 0
    elif case == "misaligned":
        C += 4
    with pytest.raises(ss.SpinsumError, match=code):
        ss.spinsum_contract(dd, ext, A, wl.table2(1), 2, mode, W, Y, ldw, C, ldc, 0)
    assert ss.spinsum_last_error()


def test_contract_empty_launches_nothing(ss):
    before = ss.spinsum_launch_count()
    ss.spinsum_contract(3, [0, 4, 4, 5, 5, 5], FAKE_A, wl.table2(1), 2, 1, FAKE_B, 3, 3, FAKE_B + (1 << 20), 1, 0)
    ss.spinsum_contract(3, [4, 4, 4, 5, 5, 5], FAKE_A, wl.table2(1), 2, 1, FAKE_B, 0, 1, FAKE_B + (1 << 20), 64, 0)
    assert ss.spinsum_launch_count() == before
