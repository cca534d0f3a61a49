"""Parity of the CUDA path (through the C-ABI) with the oracle, element by
element, on seeded inputs: every Table II set, the printed-as-is variants,
random sets; expanded and factorized; out of place and in place; exact and
strict FP64 cores; plus FP32 storage and the edge cases.

Bars: strict FP64 is bit-identical to the oracle on all inputs; the exact
FP64 core is bit-identical on integer-valued inputs and within
1e-14 * L * max|A| on uniform inputs; FP32 is within (terms + 2) 2^-24 L max|A|.
"""
import numpy as np
import pytest

import workloads as wl
from tests.gpu_helpers import (assert_bitexact, assert_within, fp32_tol, fp64_tol, gpu_run)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def orc():
    import oracle
    return oracle


def _sets(d):
    rows = [1, 2, 3, 4] if d == 3 else list(range(5, 22))
    out = [(f"row{r}", wl.table2(r)) for r in rows]
    out += [(f"row{r}-printed", wl.table2(r, printed=True)) for r in wl.TABLE2_GARBLED if wl.table2_dim(r) == d]
    out += [("random", wl.random_coef(d, 101 if d == 3 else 103)),
            ("random2", np.concatenate([wl.random_coef(d, 111), wl.random_coef(d, 112)]))]
    return out


SHAPES = {3: (8, 8, 8, 8, 8, 8), 4: (3, 3, 3, 3, 5, 5, 5, 5)}


@pytest.mark.parametrize("d", [3, 4])
@pytest.mark.parametrize("inplace", [False, True])
@pytest.mark.parametrize("factorized", [False, True])
def test_sets_exact_core(orc, d, inplace, factorized):
    shape = SHAPES[d]
    for name, coef in _sets(d):
        for kind in ("int", "uni"):
            A = wl.integers(0, shape) if kind == "int" else wl.uniform(0, shape)
            want = orc.spinsum(A, d, coef, factorized=factorized)
            got = gpu_run(A, d, coef, factorized=factorized, inplace=inplace)
            msg = f"d={d} {name} {kind} fac={factorized} ip={inplace}"
            if kind == "int":
                assert_bitexact(got, want, msg)
            else:
                assert_within(got, want, fp64_tol(d, coef, factorized, A), msg)


@pytest.mark.parametrize("d", [3, 4])
@pytest.mark.parametrize("inplace", [False, True])
@pytest.mark.parametrize("factorized", [False, True])
def test_sets_strict_core_bitexact(orc, d, inplace, factorized):
    shape = SHAPES[d]
    for name, coef in _sets(d):
        A = wl.uniform(1, shape)
        want = orc.spinsum(A, d, coef, factorized=factorized)
        got = gpu_run(A, d, coef, factorized=factorized, strict=True, inplace=inplace)
        assert_bitexact(got, want, f"strict d={d} {name} fac={factorized} ip={inplace}")


@pytest.mark.parametrize("d", [3, 4])
def test_non_integer_coefficients_take_strict_core(orc, d):
    shape = SHAPES[d]
    coef = wl.uniform(5, (1, 6 if d == 3 else 24))[0]
    A = wl.uniform(2, shape)
    assert_bitexact(gpu_run(A, d, coef), orc.spinsum(A, d, coef), "real coefficients")


@pytest.mark.parametrize("O", [1, 2, 3, 4, 7])
@pytest.mark.parametrize("d", [3, 4])
def test_small_and_degenerate_extents(orc, d, O):
    spec = (4, 4, 5) if d == 3 else (4, 4, 2, 2)
    shape = spec + (O,) * d
    coef = wl.random_coef(d, 7)
    for A in (wl.integers(3, shape), wl.uniform(3, shape)):
        want = orc.spinsum(A, d, coef)
        got = gpu_run(A, d, coef)
        assert_within(got, want, fp64_tol(d, coef, False, A), f"O={O}")
        assert_bitexact(gpu_run(A, d, coef, strict=True), want, f"strict O={O}")


@pytest.mark.parametrize("spec", [(9, 10, 11), (3, 3, 3), (1, 1, 1), (5, 1, 7), (2, 3, 5)])
def test_ragged_and_short_spectator_blocks(orc, spec):
    """ragged tails, odd blocks (scalar path), blocks too short for the
    streaming kernel (general kernel), spectator extents of 1."""
    shape = tuple(spec) + (6, 6, 6)
    coef = wl.table2(1)
    A = wl.uniform(4, shape)
    want = orc.spinsum(A, 3, coef)
    assert_within(gpu_run(A, 3, coef), want, fp64_tol(3, coef, False, A), str(spec))
    assert_bitexact(gpu_run(A, 3, coef, strict=True), want, f"strict {spec}")
    Ai = wl.integers(4, shape)
    assert_bitexact(gpu_run(Ai, 3, coef, factorized=True, inplace=True), orc.spinsum(Ai, 3, coef), str(spec))


@pytest.mark.parametrize("layout", ["rowmajor", "sliced", "offset"])
@pytest.mark.parametrize("d", [3, 4])
def test_other_layouts(orc, d, layout):
    shape = SHAPES[d]
    coef = wl.random_coef(d, 9)
    A = wl.uniform(6, shape)
    want = orc.spinsum(A, d, coef)
    kw = {"layout": "colmajor", "offset": 1} if layout == "offset" else {"layout": layout}
    assert_within(gpu_run(A, d, coef, **kw), want, fp64_tol(d, coef, False, A), layout)
    assert_bitexact(gpu_run(A, d, coef, strict=True, **kw), want, layout)


@pytest.mark.parametrize("d", [3, 4])
def test_paper_layout(orc, d):
    """The paper's own N^d tensor (Sec. 3.1): no spectators, the permuted group
    column-major with the first permuted index at stride 1."""
    import torch
    from tests.gpu_helpers import ss
    N = 20 if d == 3 else 9
    A = wl.uniform(8, (N,) * d)
    coef = wl.table2(1 if d == 3 else 6)
    want = orc.spinsum(A, d, coef, factorized=True)
    m = ss()
    At = m.to_colmajor(torch.from_numpy(A).cuda())
    for strict in (False, True):
        B = m.spinsum(At, coef, d=d, factorized=True, strict=strict).cpu().numpy()
        if strict:
            assert_bitexact(B, want, "paper layout strict")
        else:
            assert_within(B, want, fp64_tol(d, coef, True, A), "paper layout")


@pytest.mark.parametrize("alpha,beta", [(1.0, 0.0), (0.5, 0.0), (-2.0, 0.0), (3.0, 0.0), (1.0, 1.0), (0.25, -1.5),
                                        (-3.0, 2.0)])
@pytest.mark.parametrize("d", [3, 4])
def test_alpha_beta(orc, d, alpha, beta):
    shape = SHAPES[d]
    coef = wl.table2(1 if d == 3 else 5)
    A = wl.integers(10, shape)
    B0 = wl.integers(11, shape)
    want = orc.spinsum(A, d, coef, alpha=alpha, beta=beta, B=np.asfortranarray(B0.copy()))
    got = gpu_run(A, d, coef, alpha=alpha, beta=beta, B0=B0)
    assert_bitexact(got, want, f"alpha={alpha} beta={beta}")
    got = gpu_run(A, d, coef, alpha=alpha, beta=beta, B0=B0, strict=True)
    assert_bitexact(got, want, f"strict alpha={alpha} beta={beta}")
    # in place: B_old is A
    want_ip = orc.spinsum(A, d, coef, alpha=alpha, beta=beta, B=np.asfortranarray(A.copy()))
    assert_bitexact(gpu_run(A, d, coef, alpha=alpha, beta=beta, inplace=True), want_ip, "in place")


def test_beta_zero_never_reads_b(orc):
    A = wl.uniform(12, SHAPES[3])
    B0 = np.full(A.shape, np.nan, order="F")
    coef = wl.table2(2)
    got = gpu_run(A, 3, coef, B0=B0)
    assert np.isfinite(got).all()
    assert_within(got, orc.spinsum(A, 3, coef), fp64_tol(3, coef, False, A), "beta=0")


@pytest.mark.parametrize("d", [3, 4])
def test_special_values_match_oracle(orc, d):
    """Zero orbits, tiny and huge magnitudes, signed zeros, infinities and
    NaNs leave the fixed-point range; those element groups take the strict
    core, so they match the oracle exactly."""
    shape = SHAPES[d]
    A = wl.uniform(13, shape)
    flat = A.reshape(-1, order="F")
    n = flat.size
    flat[: n // 8] = 0.0
    flat[n // 8: n // 4] *= 1e-310
    flat[n // 4: n // 3] *= 1e300
    flat[n // 3: n // 3 + 50] = -0.0
    flat[n // 2] = np.inf
    flat[n // 2 + 7] = -np.inf
    flat[n // 2 + 99] = np.nan
    A = flat.reshape(shape, order="F")
    coef = wl.random_coef(d, 14)
    want = orc.spinsum(A, d, coef)
    got = gpu_run(A, d, coef)
    finite = np.isfinite(want)
    assert np.array_equal(np.isnan(got), np.isnan(want))
    assert np.array_equal(got[~finite & ~np.isnan(want)], want[~finite & ~np.isnan(want)])
    # scale-aware check on the finite part: per element the bound uses its own orbit scale,
    # so compare relative to the largest input
    err = np.abs(got[finite] - want[finite])
    assert err.max() <= 1e-14 * np.abs(coef).sum() * np.abs(A[np.isfinite(A)]).max()
    assert_bitexact(gpu_run(A, d, coef, strict=True), want, "strict special values")


def test_empty_tensor():
    import torch
    from tests.gpu_helpers import ss
    m = ss()
    A = m.colmajor_empty((0, 4, 4, 3, 3, 3))
    m.spinsum(A, wl.table2(1), d=3)
    torch.cuda.synchronize()


@pytest.mark.parametrize("d", [3, 4])
@pytest.mark.parametrize("factorized", [False, True])
def test_fp32_storage(orc, d, factorized):
    shape = SHAPES[d]
    rows = [1, "random"] if d == 3 else [5, 6, "random"]
    for r in rows:
        coef = wl.table2(r) if r != "random" else wl.random_coef(d, 15)
        A32 = wl.uniform(16, shape).astype(np.float32)
        A = np.asfortranarray(A32.astype(np.float64))
        want = orc.spinsum(A, d, coef, factorized=factorized)
        got = gpu_run(A, d, coef, factorized=factorized, dtype="f32")
        assert_within(got, want, fp32_tol(d, coef, factorized, A), f"fp32 {r}")
        got = gpu_run(A, d, coef, factorized=factorized, dtype="f32", inplace=True)
        assert_within(got, want, fp32_tol(d, coef, factorized, A), f"fp32 ip {r}")


def test_argument_errors():
    import torch
    from tests.gpu_helpers import ss
    m = ss()
    A = m.colmajor_empty((4, 4, 4, 5, 5, 5))
    A.zero_()
    B = m.colmajor_like(A)
    st = torch.cuda.current_stream().cuda_stream
    ext = list(A.shape)
    ld = list(A.stride())
    coef = wl.table2(2)
    with pytest.raises(m.SpinsumError, match="ERR_ARG"):
        m.spinsum_3d(m.SPINSUM_F64, ext[:5] + [4], A.data_ptr(), ld, B.data_ptr(), ld, coef, 1, 0, 1.0, 0.0, 0, st)
    with pytest.raises(m.SpinsumError, match="ERR_ALIAS"):
        m.spinsum_3d(m.SPINSUM_F64, ext, A.data_ptr(), ld, A.data_ptr() + 8, ld, coef, 1, 0, 1.0, 0.0, 0, st)
    with pytest.raises(m.SpinsumError, match="ERR_ALIAS"):
        m.spinsum_3d(m.SPINSUM_F64, ext, A.data_ptr(), ld, B.data_ptr(), ld, coef, 1, 0, 1.0, 0.0, 1, st)
    with pytest.raises(m.SpinsumError, match="ERR_ARG"):
        m.spinsum_3d(7, ext, A.data_ptr(), ld, B.data_ptr(), ld, coef, 1, 0, 1.0, 0.0, 0, st)
    with pytest.raises(m.SpinsumError, match="ERR_ARG"):
        m.spinsum_3d(m.SPINSUM_F64, ext, A.data_ptr(), ld, B.data_ptr(), ld, np.array([np.nan] * 6), 1, 0, 1.0,
                     0.0, 0, st)
    with pytest.raises(m.SpinsumError, match="ERR_ARG"):
        m.spinsum_3d(m.SPINSUM_F32, ext, A.data_ptr(), ld, B.data_ptr(), ld, coef, 1, m.SPINSUM_STRICT, 1.0,
                     0.0, 0, st)
    m.spinsum_check_status(st)
