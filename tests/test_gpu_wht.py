"""The d = 4 orbit-stream kernel through the Klein four-group transform
(operators with sum|a| <= 63 and a power-of-two alpha) against the dense
fixed-point core and the oracle.

The transformed path computes the same integer sums on the same 48-bit grid
as the dense core, so its results must be bit-identical to the same kernel
with the dense orbit matrices (SPINSUM_4D_DENSE_CORE=1 selects them) on any
input, and within the FP64 tolerance of the oracle; integer-valued inputs are
exact.
Covered: Table II rows 5, 6, 12, 18, 21 and random sets, expanded and
factorized, out of place and in place (several spectator chunks per CTA),
beta, negative power-of-two alpha, every orbit pattern (O = 1..7), a set
with sum|a| > 63 (dense core on the same kernel), zeros, tiny and huge
values."""
import numpy as np
import pytest

import workloads as wl
from tests.gpu_helpers import assert_bitexact, assert_within, fp64_tol, gpu_run

pytestmark = pytest.mark.gpu

SETS = [("row5", wl.table2(5), True), ("row6", wl.table2(6), True), ("row12", wl.table2(12), False),
        ("row18", wl.table2(18), False), ("row21", wl.table2(21), True), ("random103", wl.random_coef(4, 103), False),
        ("random105", wl.random_coef(4, 105), False), ("dense72", np.full((1, 24), 3.0), False)]


def _dense(monkeypatch, *a, **kw):
    monkeypatch.setenv("SPINSUM_4D_DENSE_CORE", "1")
    try:
        return gpu_run(*a, **kw)
    finally:
        monkeypatch.delenv("SPINSUM_4D_DENSE_CORE")


@pytest.mark.parametrize("shape", [(3, 3, 3, 3, 7, 7, 7, 7), (8, 8, 8, 8, 6, 6, 6, 6), (6, 5, 7, 4, 5, 5, 5, 5)])
def test_transform_equals_dense_core(monkeypatch, shape):
    import oracle
    A = wl.uniform(30, shape)
    for name, coef, fac in SETS:
        want = oracle.spinsum(A, 4, coef, factorized=fac)
        k1 = gpu_run(A, 4, coef, factorized=fac)
        dense = _dense(monkeypatch, A, 4, coef, factorized=fac)
        assert_bitexact(k1, dense, f"{name} transformed vs dense")
        assert_within(k1, want, fp64_tol(4, coef, fac, A), f"{name} vs oracle")
        ip = gpu_run(A, 4, coef, factorized=fac, inplace=True)
        assert_bitexact(ip, k1, f"{name} in place")


@pytest.mark.parametrize("O", [1, 2, 3, 4, 5, 7])
def test_all_patterns_integer_exact(O):
    import oracle
    shape = (4, 4, 4, 4) + (O,) * 4
    A = wl.integers(31, shape)
    for name, coef, fac in SETS:
        want = oracle.spinsum(A, 4, coef, factorized=fac)
        assert_bitexact(gpu_run(A, 4, coef, factorized=fac), want, f"O={O} {name}")
        assert_bitexact(gpu_run(A, 4, coef, factorized=fac, inplace=True), want, f"O={O} {name} in place")


@pytest.mark.parametrize("alpha,beta", [(1.0, 1.0), (-0.25, 0.0), (2.0, -1.5), (-1.0, 3.0)])
def test_alpha_beta_in_and_out_of_place(alpha, beta):
    import oracle
    shape = (8, 8, 4, 4, 5, 5, 5, 5)
    coef = wl.random_coef(4, 103)
    A = wl.integers(32, shape)
    B0 = wl.integers(33, shape)
    want = oracle.spinsum(A, 4, coef, alpha=alpha, beta=beta, B=np.asfortranarray(B0.copy()))
    assert_bitexact(gpu_run(A, 4, coef, alpha=alpha, beta=beta, B0=B0), want, f"alpha={alpha} beta={beta}")
    want_ip = oracle.spinsum(A, 4, coef, alpha=alpha, beta=beta, B=np.asfortranarray(A.copy()))
    assert_bitexact(gpu_run(A, 4, coef, alpha=alpha, beta=beta, inplace=True), want_ip, "in place")


def test_out_of_range_groups_take_the_strict_core(monkeypatch):
    """Zero groups stay on the fixed-point path; groups with tiny, huge or
    non-finite members take the strict core, which matches the oracle bit
    for bit."""
    import oracle
    shape = (4, 4, 4, 4, 6, 6, 6, 6)
    A = wl.uniform(34, shape)
    flat = A.reshape(-1, order="F")
    n = flat.size
    flat[: n // 10] = 0.0
    flat[n // 10: n // 5] *= 1e-310
    flat[n // 5: n // 4] *= 1e300
    flat[n // 3] = np.inf
    flat[n // 2] = np.nan
    A = flat.reshape(shape, order="F")
    coef = wl.table2(5)
    want = oracle.spinsum(A, 4, coef)
    got = gpu_run(A, 4, coef)
    dense = _dense(monkeypatch, A, 4, coef)
    assert np.array_equal(np.isnan(got), np.isnan(want))
    fin = np.isfinite(want)
    assert np.array_equal(got[~fin & ~np.isnan(want)], want[~fin & ~np.isnan(want)])
    assert np.abs(got[fin] - want[fin]).max() <= 1e-14 * 60 * np.abs(A[np.isfinite(A)]).max()
    assert_bitexact(got, dense, "transformed vs dense on special values")
