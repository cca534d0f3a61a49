"""Pins for the oracle: checks against what the paper and the mathematics fix,
never against the oracle itself. CPU only.

- element-level update statements printed in the paper (tests/golden/updates.txt)
- single-permutation operators against numpy's transpose (a library routine)
- Eq. 7 = Eq. 8 and the Sec. 4.6.2 regularization identity (Eq. 9-10)
- Table II row 1 expanded: the closed-shell weighting
- brute force against a dense matrix built from Def. 2 independently
- invariants: symmetrizer, antisymmetrizer, linearity, adjoint, composition
- cross-mode equalities: in place = out of place, factorized = expanded
"""
import itertools
import math
import os
import re

import numpy as np
import pytest

import workloads as wl

GOLD = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------
# helpers that use only numpy and the paper's definitions
# ---------------------------------------------------------------------------
def lex(d):
    return list(itertools.permutations(range(d)))


def np_permute(A, d, phi):
    """pi_phi(A) per Def. 2: B[..., t] = A[..., t_phi(1), ..., t_phi(d)]; in
    numpy terms the permuted axes are transposed by phi^{-1} (0-based phi)."""
    nspec = A.ndim - d
    inv = list(np.argsort(phi))
    return np.transpose(A, list(range(nspec)) + [nspec + k for k in inv])


def vec(d, mapping):
    """coefficient vector from {one-line-name: coef}"""
    return wl.coef_vector(d, [(c, n) for n, c in mapping.items()])


def int_tensor(seed, shape):
    return wl.integers(seed, shape)


def uni_tensor(seed, shape):
    return wl.uniform(seed, shape)


# ---------------------------------------------------------------------------
# the permutation order
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("d", [2, 3, 4])
def test_perms_are_lexicographic(oracle_mod, d):
    assert [tuple(p) for p in oracle_mod.perms(d)] == lex(d)
    assert [tuple(x - 1 for x in p) for p in wl.perms(d)] == lex(d)


# ---------------------------------------------------------------------------
# golden update statements
# ---------------------------------------------------------------------------
_TERM = re.compile(r"([+-]?)\s*(?:(\d+(?:\.\d+)?)\s*\*\s*)?([AT])\[([^\]]+)\]")


def _parse_cases():
    cases, cur = [], None
    for line in open(os.path.join(GOLD, "updates.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        m = re.match(r"\[case (.+)\]", line)
        if m:
            cur = {"name": m.group(1), "lines": []}
            cases.append(cur)
        elif line.startswith("cite:"):
            cur["cite"] = line[5:].strip()
        elif line.startswith("d:"):
            cur["d"] = int(line[2:])
        elif line.startswith("chain:"):
            facs = []
            for f in line[6:].split("|"):
                facs.append({n: float(c) for n, c in (t.split(":") for t in f.split())})
            cur["chain"] = facs
        else:
            lhs, rhs = line.split("=")
            lm = re.match(r"([BT])\[([^\]]+)\]", lhs.strip())
            terms = []
            for sgn, c, arr, idx in _TERM.findall(rhs):
                coef = float(c) if c else 1.0
                terms.append(((-coef) if sgn == "-" else coef, arr, [s.strip() for s in idx.split(",")]))
            cur["lines"].append((lm.group(1), [s.strip() for s in lm.group(2).split(",")], terms))
    return cases


CASES = _parse_cases()


def _eval_line(d, O, nspec, src, lhs_idx, terms, out):
    grids = np.indices((O,) * d)
    g = {f"i{k + 1}": grids[k] for k in range(d)}
    sl = (slice(None),) * nspec
    acc = 0.0
    for coef, arr, idx in terms:
        acc = acc + coef * src[arr][sl + tuple(g[n] for n in idx)]
    out[sl + tuple(g[n] for n in lhs_idx)] = acc


@pytest.mark.parametrize("case", CASES, ids=[c["name"] for c in CASES])
@pytest.mark.parametrize("spec", [(), (3,), (2, 3)])
def test_golden_updates(oracle_mod, case, spec):
    d = case["d"]
    O = 4
    A = int_tensor(11, tuple(spec) + (O,) * d)
    chain = np.stack([vec(d, f) for f in case["chain"]])
    B = oracle_mod.spinsum(A, d, chain, factorized=True)
    Bx = oracle_mod.spinsum(A, d, chain, factorized=False)
    np.testing.assert_array_equal(B, Bx)
    arrays = {"A": A}
    for arr, lhs, terms in case["lines"]:
        if arr == "T":
            T = np.full(A.shape, np.nan, order="F")
            _eval_line(d, O, len(spec), arrays, lhs, terms, T)
            arrays["T"] = T
        else:
            want = np.full(A.shape, np.nan, order="F")
            _eval_line(d, O, len(spec), arrays, lhs, terms, want)
            assert not np.isnan(want).any()
            np.testing.assert_array_equal(B, want, err_msg=case["cite"])


# ---------------------------------------------------------------------------
# single permutations against numpy's transpose
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("d,spec,O", [(2, (3,), 5), (3, (2, 3), 4), (4, (3,), 3)])
def test_single_permutation_is_transpose(oracle_mod, d, spec, O):
    A = uni_tensor(5, tuple(spec) + (O,) * d)
    n = math.factorial(d)
    for k, phi in enumerate(lex(d)):
        e = np.zeros(n)
        e[k] = 1.0
        B = oracle_mod.spinsum(A, d, e)
        np.testing.assert_array_equal(B, np_permute(A, d, phi), err_msg=str(phi))
    e = np.zeros(n)
    e[0] = 1.0
    np.testing.assert_array_equal(oracle_mod.spinsum(A, d, e), A)


def test_three_cycles_are_told_apart(oracle_mod):
    """pi_231 and pi_312 are inverse to each other; a gather/scatter mix-up
    swaps them. Def. 2: pi_231(A)[i1,i2,i3] = A[i2,i3,i1]."""
    A = uni_tensor(9, (4, 4, 4))
    B = oracle_mod.spinsum(A, 3, vec(3, {"231": 1.0}))
    for i1, i2, i3 in itertools.product(range(4), repeat=3):
        assert B[i1, i2, i3] == A[i2, i3, i1]
    assert not np.array_equal(B, oracle_mod.spinsum(A, 3, vec(3, {"312": 1.0})))


# ---------------------------------------------------------------------------
# Eq. 7 = Eq. 8, Sec. 4.6.2, Table II row 1
# ---------------------------------------------------------------------------
def _read_rows(name):
    rows = []
    for line in open(os.path.join(GOLD, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append(line.split())
    return rows


def test_eq7_equals_eq8(oracle_mod):
    rows = _read_rows("eq7_eq8.txt")
    outer, inner, full = (np.array([float(x) for x in r]) for r in rows)
    np.testing.assert_array_equal(oracle_mod.expand(3, np.stack([outer, inner])), full)
    A = int_tensor(3, (3, 5, 5, 5))
    B7 = oracle_mod.spinsum(A, 3, full)
    B8 = oracle_mod.spinsum(A, 3, np.stack([outer, inner]), factorized=True)
    np.testing.assert_array_equal(B7, B8)


def test_sec462_regularization_identity(oracle_mod):
    rows = _read_rows("sec462_regularization.txt")
    left, pre, right = (np.array([float(x) for x in r]) for r in rows[:3])
    names = [wl.perm_name(p) for p in wl.perms(3)]
    a = {"123": 2.0, "213": -1.0, "321": 3.0}      # a1, a2, a3
    lv = vec(3, a)
    rv = np.zeros(6)
    for lname, rname in rows[3:]:
        rv[names.index(rname)] = a[lname]
    assert np.array_equal(lv != 0, left != 0) and np.array_equal(rv != 0, right != 0)
    A = int_tensor(4, (2, 5, 5, 5))
    T = np.asfortranarray(np_permute(A, 3, (1, 0, 2)))          # pi213(A) by numpy
    np.testing.assert_array_equal(oracle_mod.spinsum(A, 3, lv), oracle_mod.spinsum(T, 3, rv))
    # and with the oracle doing the pre-transposition as a stage
    np.testing.assert_array_equal(oracle_mod.spinsum(A, 3, lv),
                                  oracle_mod.spinsum(A, 3, np.stack([rv, pre]), factorized=True))


def test_table2_row1_closed_shell_weighting(oracle_mod):
    want = np.array([float(x) for x in _read_rows("table2_row1_expanded.txt")[0]])
    np.testing.assert_array_equal(oracle_mod.expand(3, wl.table2(1)), want)


def test_table2_row5_expansion_has_no_cancellation(oracle_mod):
    """Row 5 factors have 1-norms 3, 4, 5; the product of the 24 terms of
    the 2*3*4 products hits every permutation once, so |alpha|_1 = 60."""
    full = oracle_mod.expand(4, wl.table2(5))
    assert np.count_nonzero(full) == 24
    assert np.abs(full).sum() == 60.0


# ---------------------------------------------------------------------------
# brute force: dense operator matrix from Def. 2, built with numpy only
# ---------------------------------------------------------------------------
def dense_operator(shape, d, alpha):
    N = int(np.prod(shape))
    lin = np.arange(N).reshape(shape, order="F")
    M = np.zeros((N, N))
    for a, phi in zip(alpha, lex(d)):
        if a == 0:
            continue
        src = np.asarray(np_permute(lin, d, phi)).reshape(-1, order="F")
        M[np.arange(N), src] += a
    return M


@pytest.mark.parametrize("d,shape", [(2, (2, 3, 3)), (3, (2, 3, 3, 3)), (3, (4, 4, 4)), (4, (2, 3, 3, 3, 3)),
                                     (4, (2, 2, 2, 2))])
def test_brute_force_dense_matrix(oracle_mod, d, shape):
    n = math.factorial(d)
    alpha = wl.COEF_VALUES[(wl.draws(7 + d, n) >> np.uint64(32)) % np.uint64(5)]
    M = dense_operator(shape, d, alpha)
    for A in (int_tensor(1, shape), uni_tensor(2, shape)):
        want = (M @ A.reshape(-1, order="F")).reshape(shape, order="F")
        got = oracle_mod.spinsum(A, d, alpha)
        L = np.abs(alpha).sum()
        assert np.max(np.abs(got - want)) <= 1e-15 * L * max(1.0, np.abs(A).max())
    A = int_tensor(1, shape)
    np.testing.assert_array_equal(oracle_mod.spinsum(A, d, alpha),
                                  (M @ A.reshape(-1, order="F")).reshape(shape, order="F"))


# ---------------------------------------------------------------------------
# invariants
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("d", [3, 4])
def test_symmetrizer(oracle_mod, d):
    O = 4
    n = math.factorial(d)
    A = int_tensor(21, (2,) + (O,) * d)
    B = oracle_mod.spinsum(A, d, np.ones(n))
    for phi in lex(d):
        np.testing.assert_array_equal(np_permute(B, d, phi), B)
    # on a symmetric tensor the symmetrizer multiplies by d!
    np.testing.assert_array_equal(oracle_mod.spinsum(B, d, np.ones(n)), n * B)


def _sign(p):
    s = 1
    for a in range(len(p)):
        for b in range(a + 1, len(p)):
            if p[a] > p[b]:
                s = -s
    return s


@pytest.mark.parametrize("d", [3, 4])
def test_antisymmetrizer(oracle_mod, d):
    O = 4
    A = int_tensor(22, (3,) + (O,) * d)
    sg = np.array([float(_sign(p)) for p in lex(d)])
    B = oracle_mod.spinsum(A, d, sg)
    for phi, s in zip(lex(d), sg):
        np.testing.assert_array_equal(np_permute(B, d, phi), s * B)
    # zero wherever two permuted indices coincide
    idx = np.indices((O,) * d)
    rep = np.zeros((O,) * d, dtype=bool)
    for a in range(d):
        for b in range(a + 1, d):
            rep |= idx[a] == idx[b]
    assert np.all(B[:, rep] == 0)


def test_linearity(oracle_mod):
    x = int_tensor(31, (3, 4, 4, 4))
    y = int_tensor(32, (3, 4, 4, 4))
    al = wl.random_coef(3, 5)
    lhs = oracle_mod.spinsum(np.asfortranarray(3 * x - 2 * y), 3, al)
    rhs = 3 * oracle_mod.spinsum(x, 3, al) - 2 * oracle_mod.spinsum(y, 3, al)
    np.testing.assert_array_equal(lhs, rhs)


def _inverse_coefs(d, alpha):
    P = lex(d)
    out = np.zeros_like(alpha)
    for k, phi in enumerate(P):
        out[P.index(tuple(np.argsort(phi)))] = alpha[k]
    return out


@pytest.mark.parametrize("d,spec,O", [(3, (3, 2), 5), (4, (2,), 4)])
def test_adjoint(oracle_mod, d, spec, O):
    """<S x, y> = <x, S^T y>; S^T by literal scatter equals the operator with
    coefficients alpha_{sigma^{-1}} (exact on integer data)."""
    shape = tuple(spec) + (O,) * d
    x, y = int_tensor(41, shape), int_tensor(42, shape)
    for chain in (wl.random_coef(d, 43), np.concatenate([wl.random_coef(d, 44), wl.random_coef(d, 45)])):
        Sx = oracle_mod.spinsum(x, d, chain, factorized=True)
        STy = oracle_mod.spinsum_transpose(y, d, chain)
        assert np.sum(Sx * y) == np.sum(x * STy)
        full = oracle_mod.expand(d, chain)
        np.testing.assert_array_equal(STy, oracle_mod.spinsum(y, d, _inverse_coefs(d, full)))


@pytest.mark.parametrize("d", [3, 4])
def test_composition(oracle_mod, d):
    """S_a(S_b(x)) = S_{a*b}(x) for non-self-adjoint random sets; pins the
    product rule's composition order against stage-by-stage application."""
    x = int_tensor(51, (2,) + (3,) * d)
    a, b = wl.random_coef(d, 52)[0], wl.random_coef(d, 53)[0]
    ab = oracle_mod.expand(d, np.stack([a, b]))
    np.testing.assert_array_equal(oracle_mod.spinsum(oracle_mod.spinsum(x, d, b), d, a),
                                  oracle_mod.spinsum(x, d, ab))
    ba = oracle_mod.expand(d, np.stack([b, a]))
    assert not np.array_equal(ab, ba)


# ---------------------------------------------------------------------------
# modes, alpha/beta, strides
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("row", [1, 5, 6, 12])
def test_inplace_equals_out_of_place(oracle_mod, row):
    d = wl.table2_dim(row)
    A = uni_tensor(61, (2, 3) + (4,) * d)
    for fac in (False, True):
        B = oracle_mod.spinsum(A, d, wl.table2(row), factorized=fac, alpha=0.5, beta=0.25,
                               B=np.asfortranarray(A.copy()))
        A2 = np.asfortranarray(A.copy())
        oracle_mod.spinsum(A2, d, wl.table2(row), factorized=fac, alpha=0.5, beta=0.25, inplace=True)
        np.testing.assert_array_equal(A2, B)


@pytest.mark.parametrize("row", list(range(1, 22)))
def test_factorized_equals_expanded_on_integers(oracle_mod, row):
    d = wl.table2_dim(row)
    A = int_tensor(62, (2,) + (4,) * d)
    np.testing.assert_array_equal(oracle_mod.spinsum(A, d, wl.table2(row), factorized=True),
                                  oracle_mod.spinsum(A, d, wl.table2(row), factorized=False))


def test_alpha_beta(oracle_mod):
    A = int_tensor(71, (3, 4, 4, 4))
    B0 = int_tensor(72, (3, 4, 4, 4))
    al = wl.table2(1)
    S = oracle_mod.spinsum(A, 3, al)
    B = oracle_mod.spinsum(A, 3, al, alpha=-2.0, beta=3.0, B=np.asfortranarray(B0.copy()))
    np.testing.assert_array_equal(B, -2 * S + 3 * B0)
    Bn = np.full(A.shape, np.nan, order="F")
    np.testing.assert_array_equal(oracle_mod.spinsum(A, 3, al, beta=0.0, B=Bn), S)


def test_strided_layouts(oracle_mod):
    """The paper's layout (no spectators, permuted group at stride 1) and an
    arbitrary strided view agree with a dense copy."""
    A = uni_tensor(81, (6, 6, 6))
    al = wl.random_coef(3, 82)
    want = oracle_mod.spinsum(np.asfortranarray(A), 3, al)
    big = np.zeros((3, 5, 6, 6, 6), order="F")
    view = big[1, 2]
    view[...] = A
    np.testing.assert_array_equal(oracle_mod.spinsum(view, 3, al), want)
    C = np.ascontiguousarray(A)                                    # row-major strides
    np.testing.assert_array_equal(oracle_mod.spinsum(C, 3, al), want)


def test_empty_and_degenerate(oracle_mod):
    A = np.zeros((0, 3, 3, 3), order="F")
    assert oracle_mod.spinsum(A, 3, np.ones(6)).shape == A.shape
    A = uni_tensor(91, (2, 1, 1, 1))
    # extent 1: every orbit has one member, the operator is multiplication by sum(alpha)
    al = wl.random_coef(3, 92)
    np.testing.assert_array_equal(oracle_mod.spinsum(A, 3, al), al.sum() * A)


def test_transpose_of_factor_chain_reverses_order(oracle_mod):
    d = 3
    y = int_tensor(93, (2, 4, 4, 4))
    F1, F2 = wl.random_coef(d, 94)[0], wl.random_coef(d, 95)[0]
    st = oracle_mod.spinsum_transpose(y, d, np.stack([F1, F2]))
    want = oracle_mod.spinsum(oracle_mod.spinsum(y, d, _inverse_coefs(d, F1)), d, _inverse_coefs(d, F2))
    np.testing.assert_array_equal(st, want)


def test_table2_flop_reduction_factors(oracle_mod):
    """Sec. 5: factorization reduces the FLOP count of test cases 1, 2-4, 5,
    6-17 and 18-21 by 2x, 1x, 4x, 2x and 1x, and cases 6-17 all need the same
    number of operations. Counting the additions per output element (terms - 1
    expanded against the sum of terms - 1 over the factors) and rounding gives
    these factors exactly under the repaired reading of Table II, including the
    garbled rows 8-11, 16 and 17; a wrong sign or a missing term in any factor
    changes a count."""
    want = {1: 2, 5: 4}
    want.update({r: 1 for r in (2, 3, 4, 18, 19, 20, 21)})
    want.update({r: 2 for r in range(6, 18)})
    counts = {}
    for row in wl.TABLE2_ROWS:
        d = wl.table2_dim(row)
        chain = np.atleast_2d(wl.table2(row))
        expanded = oracle_mod.expand(d, chain)
        adds_exp = int(np.count_nonzero(expanded)) - 1
        adds_fac = int(sum(np.count_nonzero(f) - 1 for f in chain))
        assert round(adds_exp / adds_fac) == want[row], (row, adds_exp, adds_fac)
        counts[row] = (adds_exp, adds_fac)
    assert len({counts[r] for r in range(6, 18)}) == 1
    assert max(counts, key=lambda r: counts[r][0] / counts[r][1]) == 5


def test_d2_is_a_weighted_transpose(oracle_mod):
    """d = 2 (Def. 3 with the two permutations of (i, j)): B = a_12 A +
    a_21 A^T over the permuted pair, against numpy's transpose, with
    spectators and on the plain N^2 matrix; a two-factor chain equals its
    product (the group algebra of S_2: (a + b t)(c + e t) = (ac + be) + (ae + bc) t)."""
    A = wl.uniform(61, (3, 4, 6, 6))
    for coef in ([1.0, 1.0], [1.0, -1.0], [2.0, -1.0], [0.0, 1.0]):
        want = coef[0] * A + coef[1] * A.transpose(0, 1, 3, 2)
        np.testing.assert_array_equal(oracle_mod.spinsum(A, 2, np.array([coef])), want)
    M = wl.uniform(62, (9, 9))
    np.testing.assert_array_equal(oracle_mod.spinsum(M, 2, np.array([[3.0, -2.0]])), 3.0 * M - 2.0 * M.T)
    chain = np.array([[2.0, -1.0], [1.0, 3.0]])
    a, b, c, e = 2.0, -1.0, 1.0, 3.0
    np.testing.assert_array_equal(oracle_mod.expand(2, chain), [a * c + b * e, a * e + b * c])
    Ai = wl.integers(63, (5, 5, 7, 7))
    np.testing.assert_array_equal(oracle_mod.spinsum(Ai, 2, chain, factorized=True),
                                  oracle_mod.spinsum(Ai, 2, chain, factorized=False))


@pytest.mark.parametrize("d,O", [(2, 7), (3, 6), (4, 6)])
def test_packed_antisymmetric_storage(oracle_mod, d, O):
    """unpack gives an antisymmetric tensor (any transposition of two permuted
    axes negates it, equal indices give 0), pack inverts it, and the packed
    axis has C(O, d) entries in colex order: for d = 2 the pair i < j sits at
    i + j (j - 1) / 2 (C(i, 1) + C(j, 2), written out)."""
    P = wl.uniform(90 + d, (3, 2, math.comb(O, d)))
    B = oracle_mod.unpack(P, d, O)
    nspec = B.ndim - d
    for a, b in itertools.combinations(range(d), 2):
        axes = list(range(B.ndim))
        axes[nspec + a], axes[nspec + b] = axes[nspec + b], axes[nspec + a]
        np.testing.assert_array_equal(B.transpose(axes), -B)
    np.testing.assert_array_equal(oracle_mod.pack(B, d), P)
    assert sorted(oracle_mod.colex_rank(t) for t in itertools.combinations(range(O), d)) == list(range(math.comb(O, d)))
    if d == 2:
        for i in range(O):
            assert np.all(B[..., i, i] == 0)
            for j in range(i + 1, O):
                np.testing.assert_array_equal(B[..., i, j], P[..., i + j * (j - 1) // 2])
                np.testing.assert_array_equal(B[..., j, i], -P[..., i + j * (j - 1) // 2])


# ---------------------------------------------------------------------------
# contraction over the permuted group (the fused consumer of the summation)
# ---------------------------------------------------------------------------
def test_contract_brute_force(oracle_mod):
    """C[s, y] = sum over permuted tuples t of B[s, t] W[y, t], with the tuple
    index t = i_1 + O i_2 + O^2 i_3 written out here by explicit loops."""
    d, O, spec, Y = 3, 3, (2, 3), 4
    A = wl.integers(40, spec + (O,) * d)
    W = wl.integers(41, (Y, O ** d))
    coef = wl.table2(1)
    B = oracle_mod.spinsum(A, d, coef, factorized=True)
    C = oracle_mod.contract(A, d, coef, W, factorized=True)
    assert C.shape == spec + (Y,)
    for s in itertools.product(*[range(n) for n in spec]):
        for y in range(Y):
            acc = 0.0
            for t in itertools.product(range(O), repeat=d):
                tl = t[0] + O * t[1] + O * O * t[2]
                acc += B[s + t] * W[y, tl]
            assert C[s + (y,)] == acc


def test_contract_with_unit_rows_is_the_summation(oracle_mod):
    """W = identity (Y = O^d): the contraction returns S(A) itself."""
    d, O, spec = 4, 3, (2,)
    A = wl.integers(42, spec + (O,) * d)
    coef = wl.random_coef(4, 43)
    C = oracle_mod.contract(A, d, coef, np.eye(O ** d))
    B = oracle_mod.spinsum(A, d, coef)
    np.testing.assert_array_equal(C, B.reshape(spec + (O ** d,), order="F"))


def test_contract_plain_matches_tensordot(oracle_mod):
    """coef None: the contraction alone equals numpy's tensordot over the
    permuted axes (W reshaped column-major to one axis per index)."""
    d, O, spec, Y = 3, 4, (3, 2), 5
    A = wl.uniform(44, spec + (O,) * d)
    W = wl.uniform(45, (Y, O ** d))
    Wt = W.reshape((Y,) + (O,) * d, order="F")
    want = np.tensordot(A, Wt, axes=([2, 3, 4], [1, 2, 3]))
    np.testing.assert_allclose(oracle_mod.contract(A, d, None, W), want, rtol=0, atol=1e-13)
