"""The paper's own layout (Sec. 3.1): dense N^d tensors whose permuted group
includes the stride-1 index, run by the tiled block-orbit kernel. Parity with
the oracle for every Table II set, ragged N (not a multiple of the tile edge),
in place, alpha/beta, strict and FP32."""
import numpy as np
import pytest

import workloads as wl
from tests.gpu_helpers import assert_bitexact, assert_within, fp32_tol, fp64_tol

pytestmark = pytest.mark.gpu


def _run(A_np, d, coef, **kw):
    import torch
    import paper_1705_06661_gb300 as ss
    dt = kw.pop("dtype", torch.float64)
    A = ss.to_colmajor(torch.from_numpy(A_np).to("cuda", dt))
    B0 = kw.pop("B0", None)
    if kw.get("inplace"):
        out = None
    elif B0 is not None:
        out = ss.to_colmajor(torch.from_numpy(B0).to("cuda", dt))
    else:
        out = ss.colmajor_like(A)
    r = ss.spinsum(A, coef, d=d, out=out, **kw)
    ss.spinsum_check_status(torch.cuda.current_stream().cuda_stream)
    return r.double().cpu().numpy()


SETS3 = [("row%d" % r, wl.table2(r)) for r in (1, 2, 3, 4)] + [("random", wl.random_coef(3, 601))]
SETS4 = [("row%d" % r, wl.table2(r)) for r in (5, 6, 9, 13, 17, 18, 21)] + [("random", wl.random_coef(4, 602))]


@pytest.mark.parametrize("N", [1, 2, 7, 8, 13, 20, 33])
def test_k2_3d(N):
    import oracle
    for name, coef in SETS3:
        for fac in (False, True):
            Ai = wl.integers(610 + N, (N, N, N))
            assert_bitexact(_run(Ai, 3, coef, factorized=fac), oracle.spinsum(Ai, 3, coef, factorized=fac),
                            f"N={N} {name}")
            Au = wl.uniform(620 + N, (N, N, N))
            want = oracle.spinsum(Au, 3, coef, factorized=fac)
            assert_within(_run(Au, 3, coef, factorized=fac), want, fp64_tol(3, coef, fac, Au), f"N={N} {name}")
            assert_bitexact(_run(Au, 3, coef, factorized=fac, strict=True), want, f"strict N={N} {name}")


@pytest.mark.parametrize("N", [1, 3, 4, 6, 9, 10])
def test_k2_4d(N):
    import oracle
    for name, coef in SETS4:
        fac = coef.shape[0] > 1
        Ai = wl.integers(630 + N, (N,) * 4)
        assert_bitexact(_run(Ai, 4, coef, factorized=fac), oracle.spinsum(Ai, 4, coef, factorized=fac),
                        f"N={N} {name}")
        Au = wl.uniform(640 + N, (N,) * 4)
        want = oracle.spinsum(Au, 4, coef, factorized=fac)
        assert_within(_run(Au, 4, coef, factorized=fac), want, fp64_tol(4, coef, fac, Au), f"N={N} {name}")
        assert_bitexact(_run(Au, 4, coef, factorized=fac, strict=True), want, f"strict N={N} {name}")


@pytest.mark.parametrize("d,N", [(3, 21), (4, 7)])
def test_k2_inplace_alpha_beta_fp32(d, N):
    import torch
    import oracle
    coef = wl.table2(1 if d == 3 else 5)
    A = wl.integers(650, (N,) * d)
    B0 = wl.integers(651, (N,) * d)
    for alpha, beta in ((1.0, 0.0), (-0.5, 2.0), (3.0, 1.0)):
        want = oracle.spinsum(A, d, coef, alpha=alpha, beta=beta, B=np.asfortranarray(B0.copy()))
        assert_bitexact(_run(A, d, coef, alpha=alpha, beta=beta, B0=B0), want, f"alpha={alpha} beta={beta}")
        want_ip = oracle.spinsum(A, d, coef, alpha=alpha, beta=beta, B=np.asfortranarray(A.copy()))
        assert_bitexact(_run(A, d, coef, alpha=alpha, beta=beta, inplace=True), want_ip, "in place")
    Au = np.asfortranarray(wl.uniform(652, (N,) * d).astype(np.float32).astype(np.float64))
    want = oracle.spinsum(Au, d, coef, factorized=True)
    got = _run(Au, d, coef, factorized=True, dtype=torch.float32)
    assert_within(got, want, fp32_tol(d, coef, True, Au), "fp32")
