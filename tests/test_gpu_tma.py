"""Parity of the TMA-staged orbit kernel (the SPINSUM_TMA mode: a producer
warp copies each orbit member run into a shared-memory ring with bulk copies,
consumer warps apply the operator) with the oracle, element by element.

3D, exact FP64 and FP32 storage; integer-valued inputs bit-exact, uniform
inputs within the tolerances of the register-streaming kernel; out of place
and in place, with beta; and a spectator block of 32^3 positions, so that every
persistent CTA takes about 25 (orbit, chunk) tiles and its 4-stage ring wraps
several times. That the planner selects this kernel for these shapes is
checked on the CPU (tests/test_abi_cpu.py)."""
import numpy as np
import pytest

import workloads as wl
from tests.gpu_helpers import assert_bitexact, assert_within, fp32_tol, fp64_tol, gpu_run

pytestmark = pytest.mark.gpu

SHAPES = [(8, 8, 8, 8, 8, 8), (32, 32, 32, 8, 8, 8), (16, 8, 8, 5, 5, 5)]


def _sets():
    return [("row1", wl.table2(1), True), ("row2", wl.table2(2), False), ("random", wl.random_coef(3, 101), False)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("inplace", [False, True])
def test_tma_exact_fp64(shape, inplace):
    import oracle
    for name, coef, fac in _sets():
        for kind in ("int", "uni"):
            A = wl.integers(20, shape) if kind == "int" else wl.uniform(20, shape)
            want = oracle.spinsum(A, 3, coef, factorized=fac)
            got = gpu_run(A, 3, coef, factorized=fac, inplace=inplace, tma=True)
            msg = f"tma {shape} {name} {kind} ip={inplace}"
            if kind == "int":
                assert_bitexact(got, want, msg)
            else:
                assert_within(got, want, fp64_tol(3, coef, fac, A), msg)


@pytest.mark.parametrize("shape", SHAPES[:2])
def test_tma_fp32(shape):
    import oracle
    for name, coef, fac in _sets():
        A = wl.uniform(21, shape).astype(np.float32).astype(np.float64)
        want = oracle.spinsum(A, 3, coef, factorized=fac)
        got = gpu_run(A, 3, coef, factorized=fac, dtype="f32", tma=True)
        assert_within(got, want, fp32_tol(3, coef, fac, A), f"tma f32 {shape} {name}")


def test_tma_beta_and_alpha():
    import oracle
    shape = SHAPES[1]
    coef = wl.table2(1)
    A = wl.integers(22, shape)
    B0 = wl.integers(23, shape)
    want = oracle.spinsum(A, 3, coef, alpha=0.5, beta=-2.0, B=np.asfortranarray(B0.copy()))
    got = gpu_run(A, 3, coef, alpha=0.5, beta=-2.0, B0=B0, tma=True)
    assert_bitexact(got, want, "tma alpha/beta")
