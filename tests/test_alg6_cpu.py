"""The paper's blocked CPU algorithm (Algorithms 5a/5b and 6, host library
``cpu_alg6``) against the oracle. Both add a row's terms in lexicographic
order of sigma with one rounding per product and sum, so every case is
compared for equality: expanded and factorized chains, in place, alpha and
beta, tiles cut by the tensor's edge, one and several threads."""
import math

import numpy as np
import pytest

import cpu_alg6
import oracle
import workloads as wl

CASES = [(2, 13, 4), (2, 70, 0), (2, 5, 1), (3, 9, 4), (3, 10, 3), (3, 17, 16), (3, 33, 0), (4, 7, 3), (4, 9, 4),
         (4, 5, 8), (4, 11, 0)]


def _uniform(rng, d, N):
    return np.asfortranarray(rng.uniform(-1.0, 1.0, (N,) * d))


@pytest.mark.parametrize("d,N,bl", CASES)
def test_alg6_equals_oracle(d, N, bl):
    rng = np.random.default_rng(100 * d + N + bl)
    n = math.factorial(d)
    A = _uniform(rng, d, N)
    chains = [(rng.uniform(-1.0, 1.0, (1, n)), False),
              (rng.integers(-2, 3, (3, n)).astype(np.float64), True),
              (rng.uniform(-1.0, 1.0, (2, n)), False),
              (rng.uniform(-1.0, 1.0, (2, n)), True)]
    for coef, fac in chains:
        for alpha, beta in ((1.0, 0.0), (0.37, -1.25)):
            B0 = _uniform(rng, d, N)
            want = oracle.spinsum(A, d, coef, factorized=fac, alpha=alpha, beta=beta, B=B0.copy(order="F"))
            got = cpu_alg6.spinsum_alg6(A, coef, factorized=fac, alpha=alpha, beta=beta, out=B0.copy(order="F"),
                                        bl=bl, threads=3)
            assert np.array_equal(got, want), (d, N, bl, fac, alpha, beta)


@pytest.mark.parametrize("d,N,bl", [(3, 10, 3), (4, 9, 4), (2, 13, 4)])
def test_alg6_in_place(d, N, bl):
    rng = np.random.default_rng(7 + d)
    n = math.factorial(d)
    A = _uniform(rng, d, N)
    for coef, fac in ((rng.uniform(-1.0, 1.0, (2, n)), True), (rng.uniform(-1.0, 1.0, (1, n)), False)):
        for alpha, beta in ((1.0, 0.0), (2.0, 0.5)):
            mine = A.copy(order="F")
            cpu_alg6.spinsum_alg6(mine, coef, factorized=fac, alpha=alpha, beta=beta, inplace=True, bl=bl, threads=2)
            ref = A.copy(order="F")
            oracle.spinsum(ref, d, coef, factorized=fac, alpha=alpha, beta=beta, inplace=True)
            assert np.array_equal(mine, ref)


@pytest.mark.parametrize("row", [1, 2, 4, 5, 6, 8, 12, 18, 21])
def test_alg6_table2_rows(row):
    d = wl.table2_dim(row)
    N = 11 if d == 3 else 6
    A = np.asfortranarray(wl.uniform(row, (N,) * d))
    coef = wl.table2(row)
    for fac in (False, True):
        want = oracle.spinsum(A, d, coef, factorized=fac)
        got = cpu_alg6.spinsum_alg6(A, coef, factorized=fac, bl=4, threads=4)
        assert np.array_equal(got, want)


def test_alg6_thread_count_does_not_change_result():
    rng = np.random.default_rng(3)
    A = _uniform(rng, 3, 21)
    coef = rng.uniform(-1.0, 1.0, (2, 6))
    r1 = cpu_alg6.spinsum_alg6(A, coef, factorized=True, bl=4, threads=1)
    r5 = cpu_alg6.spinsum_alg6(A, coef, factorized=True, bl=4, threads=5)
    assert np.array_equal(r1, r5)


def test_alg6_arguments():
    lib = cpu_alg6._load()
    A = np.zeros((4, 4, 4), order="F")
    B = np.zeros_like(A, order="F")
    c = np.ones(6)
    P = lambda a: a.ctypes.data  # noqa: E731
    assert lib.spinsum_alg6(5, 4, P(A), P(B), P(c), 1, 0, 1.0, 0.0, 0, 1) == -1   # d
    assert lib.spinsum_alg6(3, -1, P(A), P(B), P(c), 1, 0, 1.0, 0.0, 0, 1) == -1  # N
    assert lib.spinsum_alg6(3, 4, P(A), P(B), P(c), 0, 0, 1.0, 0.0, 0, 1) == -1   # no factor
    assert lib.spinsum_alg6(3, 4, P(A), P(B), P(c), 9, 0, 1.0, 0.0, 0, 1) == -1   # too many factors
    assert lib.spinsum_alg6(3, 4, P(A), P(B), P(c), 1, 2, 1.0, 0.0, 0, 1) == -1   # factorized flag
    assert lib.spinsum_alg6(3, 4, P(A), P(B), P(c), 1, 0, 1.0, 0.0, 65, 1) == -1  # tile edge
    assert lib.spinsum_alg6(3, 4, P(A), P(B), P(c), 1, 0, 1.0, 0.0, 0, -1) == -1  # threads
    assert lib.spinsum_alg6(3, 4, None, P(B), P(c), 1, 0, 1.0, 0.0, 0, 1) == -1   # null input
    assert lib.spinsum_alg6(3, 0, None, None, P(c), 1, 0, 1.0, 0.0, 0, 1) == 0    # empty tensor
    with pytest.raises(ValueError):
        cpu_alg6.spinsum_alg6(np.zeros((4, 4, 5), order="F"), c)
    with pytest.raises(ValueError):
        cpu_alg6.spinsum_alg6(A, np.ones(5))


# ---------------------------------------------------------------------------
# Algorithm 2 (the NCC code's spin summation)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("d,N", [(2, 9), (2, 1), (3, 7), (3, 12), (4, 5), (4, 6)])
def test_alg2_equals_oracle(d, N):
    """Same rounding order as the oracle (lexicographic sigma, multiply then
    add): equal for real single-factor sets and for integer chains (whose
    expansion is exact)."""
    rng = np.random.default_rng(300 + 10 * d + N)
    n = math.factorial(d)
    A = _uniform(rng, d, N)
    for coef in (rng.uniform(-1.0, 1.0, (1, n)), rng.integers(-2, 3, (3, n)).astype(np.float64)):
        for alpha, beta in ((1.0, 0.0), (0.37, -1.25)):
            B0 = _uniform(rng, d, N)
            want = oracle.spinsum(A, d, coef, alpha=alpha, beta=beta, B=B0.copy(order="F"))
            for threads in (1, 3):
                got = cpu_alg6.spinsum_alg2(A, coef, alpha=alpha, beta=beta, out=B0.copy(order="F"),
                                            threads=threads)
                assert np.array_equal(got, want), (d, N, alpha, beta, threads)


@pytest.mark.parametrize("row", [1, 3, 5, 6, 18])
def test_alg2_in_place_table2(row):
    d = wl.table2_dim(row)
    N = 9 if d == 3 else 5
    A = np.asfortranarray(wl.integers(row + 50, (N,) * d))
    coef = wl.table2(row)
    mine = A.copy(order="F")
    cpu_alg6.spinsum_alg2(mine, coef, inplace=True, threads=2)
    assert np.array_equal(mine, oracle.spinsum(A, d, coef, factorized=True))
