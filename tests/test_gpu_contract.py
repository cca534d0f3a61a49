"""The spin summation fused into a contraction over the permuted group
(spinsum_contract) against the oracle: C[s, y] = sum_t S(A)[s, t] W[y, t], the
oracle's summation followed by one matrix product.

Tolerance. The summed values carry the summation's error, at most
1e-14 * L * max|A| each; the FP64 accumulation over the T = O^d tuples adds
at most T * 2^-53 of sum_t |S(A)[s, t] W[y, t]| on each side (kernel and
oracle, in different orders). With sum_t |W[y, t]| <= w1 and |S(A)| <= L max|A|:
|dC| <= (1e-14 + 2 T 2^-53) * L * max|A| * w1. Integer-valued A and W keep
every product and partial sum exact, so those results are bit-exact."""
import numpy as np
import pytest

import workloads as wl
from tests.gpu_helpers import assert_bitexact, assert_within, chain_norm

pytestmark = pytest.mark.gpu


def _tol(d, coef, fac, A, W):
    L = 1.0 if coef is None else chain_norm(d, coef, fac)
    T = W.shape[1]
    return (1e-14 + 2 * T * 2.0 ** -53) * L * float(np.abs(A).max()) * float(np.abs(W).sum(axis=1).max())


def _run(A_np, d, coef, W_np, fac=False, strict=False, adjoint=False, pad_w=0, pad_c=0):
    import torch
    import paper_1705_06661_gb300 as ss
    A = ss.to_colmajor(torch.from_numpy(A_np).cuda())
    Y, T = W_np.shape
    Wb = ss.colmajor_empty((Y + pad_w, T))
    Wb.fill_(float("nan"))
    W = Wb[:Y]
    W.copy_(torch.from_numpy(W_np))
    spec = A_np.shape[:d]
    S = int(np.prod(spec))
    ldc = S + pad_c
    base = torch.full((ldc * Y,), -7.0, dtype=torch.float64, device="cuda")
    strides = [int(np.prod(spec[:k])) for k in range(d)] + [ldc]
    out = base.as_strided(spec + (Y,), strides, 0)
    C = ss.contract(A, coef, W, d=d, out=out, factorized=fac, strict=strict, adjoint=adjoint)
    torch.cuda.synchronize()
    ss.spinsum_check_status(torch.cuda.current_stream().cuda_stream)
    if pad_c:
        gaps = base.view(Y, ldc)[:, S:].cpu().numpy()
        assert np.all(gaps == -7.0), "C padding written"
    return C.cpu().numpy()


CASES = [(3, (5, 6, 7), 6, wl.table2(1), True), (3, (8, 8, 4), 5, wl.random_coef(3, 101), False),
         (4, (3, 5, 2, 3), 4, wl.table2(5), True), (4, (2, 2, 17, 1), 5, wl.random_coef(4, 103), False),
         (2, (33, 7), 9, np.array([[2.0, -1.0]]), False)]


@pytest.mark.parametrize("Y", [1, 3, 4, 5, 8, 9, 16, 17, 33])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_fused_against_oracle(case, Y):
    import oracle
    d, spec, O, coef, fac = CASES[case]
    shape = spec + (O,) * d
    A = wl.uniform(50 + case, shape)
    W = wl.uniform(60 + Y, (Y, O ** d))
    want = oracle.contract(A, d, coef, W, factorized=fac)
    got = _run(A, d, coef, W, fac=fac)
    assert_within(got, want, _tol(d, coef, fac, A, W), f"case {case} Y={Y}")
    plain = _run(A, d, None, W)
    assert_within(plain, oracle.contract(A, d, None, W), _tol(d, None, False, A, W), f"plain case {case} Y={Y}")


@pytest.mark.parametrize("case", range(len(CASES)))
def test_integer_inputs_bit_exact(case):
    import oracle
    d, spec, O, coef, fac = CASES[case]
    shape = spec + (O,) * d
    A = wl.integers(70 + case, shape)
    W = wl.integers(80 + case, (7, O ** d))
    assert_bitexact(_run(A, d, coef, W, fac=fac), oracle.contract(A, d, coef, W, factorized=fac), f"case {case}")
    assert_bitexact(_run(A, d, coef, W, fac=fac, strict=True), oracle.contract(A, d, coef, W, factorized=fac),
                    f"strict case {case}")
    assert_bitexact(_run(A, d, None, W), oracle.contract(A, d, None, W), f"plain case {case}")


def test_adjoint_strict_and_padding():
    import oracle
    d, spec, O = 3, (4, 4, 5), 6
    A = wl.uniform(90, spec + (O,) * d)
    W = wl.uniform(91, (10, O ** d))
    coef = np.concatenate([wl.random_coef(3, 92), wl.random_coef(3, 93)])
    # the adjoint of a chain is the chain of transposed factors in reverse order
    g = oracle.perms(3)
    inv = [int(np.where((g == np.argsort(p)).all(axis=1))[0][0]) for p in g]
    adj = np.stack([coef[1][inv], coef[0][inv]])
    want = oracle.contract(A, d, adj, W, factorized=True)
    got = _run(A, d, coef, W, fac=True, adjoint=True, pad_w=3, pad_c=5)
    assert_within(got, want, _tol(d, coef, True, A, W), "adjoint, padded W and C")
    want = oracle.contract(A, d, coef, W, factorized=True)
    got = _run(A, d, coef, W, fac=True, strict=True)
    assert_within(got, want, (2 * O ** d * 2.0 ** -53) * chain_norm(d, coef, True) * np.abs(A).max()
                  * np.abs(W).sum(axis=1).max(), "strict")


def test_fused_equals_unfused_pair():
    """The fused call against the summation stored by spinsum followed by the
    contraction alone: the same summed values, multiplied in the same orbit
    order, so bit-identical."""
    import torch
    import paper_1705_06661_gb300 as ss
    d, spec, O = 4, (4, 4, 4, 4), 6
    A_np = wl.uniform(94, spec + (O,) * d)
    W_np = wl.uniform(95, (12, O ** d))
    coef = wl.table2(6)
    A = ss.to_colmajor(torch.from_numpy(A_np).cuda())
    W = ss.colmajor_empty(W_np.shape)
    W.copy_(torch.from_numpy(W_np))
    fused = ss.contract(A, coef, W, factorized=True)
    B = ss.spinsum(A, coef, d=4, factorized=True)
    pair = ss.contract(B, None, W)
    torch.cuda.synchronize()
    assert_bitexact(fused.cpu().numpy(), pair.cpu().numpy(), "fused vs unfused")


def test_empty_permuted_group_gives_zeros():
    import torch
    import paper_1705_06661_gb300 as ss
    A = ss.colmajor_empty((4, 4, 4, 0, 0, 0))
    W = ss.colmajor_empty((3, 0))
    C = ss.colmajor_empty((4, 4, 4, 3))
    C.fill_(5.0)
    ss.contract(A, wl.table2(1), W, out=C)
    torch.cuda.synchronize()
    assert torch.all(C == 0)
