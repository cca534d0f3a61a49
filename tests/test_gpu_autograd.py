"""Differentiation: the backward pass is the adjoint sum a_sigma pi_{sigma^-1}
(chains reversed), run by the same orbit kernels. Checked by the inner-product
identity (exact on integer data), against the oracle's literal transpose, and
by torch.autograd.gradcheck (full on a 2^8 tensor, fast mode on 4^8)."""
import numpy as np
import pytest

import workloads as wl
from tests.gpu_helpers import assert_bitexact, assert_within, fp64_tol, gpu_run

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("d,shape", [(3, (4, 3, 5, 6, 6, 6)), (4, (3, 2, 2, 3, 5, 5, 5, 5))])
@pytest.mark.parametrize("factorized", [False, True])
def test_adjoint_matches_oracle_transpose(d, shape, factorized):
    import oracle
    chain = np.concatenate([wl.random_coef(d, 501), wl.random_coef(d, 502)])
    for kind in ("int", "uni"):
        Y = (wl.integers if kind == "int" else wl.uniform)(503, shape)
        want = oracle.spinsum_transpose(Y, d, chain)
        got = gpu_run(Y, d, chain, factorized=factorized, adjoint=True)
        if kind == "int":
            assert_bitexact(got, want, "adjoint")
        else:
            assert_within(got, want, fp64_tol(d, chain, factorized, Y), "adjoint")
        # strict core: same operator, reference order of the adjoint chain
        got = gpu_run(Y, d, chain, factorized=factorized, adjoint=True, strict=True)
        assert_within(got, want, fp64_tol(d, chain, factorized, Y), "adjoint strict")


@pytest.mark.parametrize("d", [3, 4])
def test_inner_product_identity(d):
    shape = (3,) * d + (5,) * d
    x, y = wl.integers(511, shape), wl.integers(512, shape)
    a = wl.random_coef(d, 513)
    Sx = gpu_run(x, d, a)
    STy = gpu_run(y, d, a, adjoint=True)
    assert np.sum(Sx * y) == np.sum(x * STy)


def _gradcheck(d, n, fast, coef, factorized):
    import torch
    import paper_1705_06661_gb300 as ss
    A = ss.to_colmajor(torch.from_numpy(wl.uniform(521, (n,) * (2 * d))).cuda()).requires_grad_(True)
    fn = lambda x: ss.spinsum_autograd(x, coef, d=d, factorized=factorized, alpha=0.5)  # noqa: E731
    assert torch.autograd.gradcheck(fn, (A,), eps=1e-6, atol=1e-9, rtol=1e-7, fast_mode=fast)


def test_gradcheck_full_2_8():
    _gradcheck(4, 2, False, wl.random_coef(4, 522), False)
    _gradcheck(4, 2, False, np.concatenate([wl.random_coef(4, 523), wl.random_coef(4, 524)]), True)


def test_gradcheck_fast_4_8():
    _gradcheck(4, 4, True, wl.random_coef(4, 525), False)
    _gradcheck(4, 4, True, wl.table2(5), True)


def test_backward_matches_oracle_on_config5_shape_scaled():
    """forward and backward through autograd on a 10^4 x 6^4 tensor with the
    config-5 coefficient sets; the gradient equals the oracle's transpose of
    the cotangent."""
    import torch
    import oracle
    import paper_1705_06661_gb300 as ss
    shape = (10, 10, 10, 10, 6, 6, 6, 6)
    A_np = wl.uniform(4, shape)
    G_np = wl.uniform(5, shape)
    for coef, fac in ((wl.random_coef(4, 105), False), (wl.table2(5), True)):
        A = ss.to_colmajor(torch.from_numpy(A_np).cuda()).requires_grad_(True)
        B = ss.spinsum_autograd(A, coef, d=4, factorized=fac)
        G = ss.to_colmajor(torch.from_numpy(G_np).cuda())
        B.backward(G)
        want_B = oracle.spinsum(A_np, 4, coef, factorized=fac)
        assert_within(B.detach().cpu().numpy(), want_B, fp64_tol(4, coef, fac, A_np), "forward")
        want_g = oracle.spinsum_transpose(G_np, 4, coef)
        assert_within(A.grad.cpu().numpy(), want_g, fp64_tol(4, coef, fac, G_np), "backward")
