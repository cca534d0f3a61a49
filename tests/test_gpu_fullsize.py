"""Parity at the benchmark sizes, in the launch configuration bench.py times:
the whole output compared element by element with the oracle (plain C,
OpenMP over the host cores).

- 3D, A[48,48,48,16,16,16] (453M doubles): Table II row 1 factorized, out of
  place (the benchmark step) and in place; an integer-valued copy bit-exact.
- 4D, A[12]^8 (430M doubles): Table II rows 5 and 6 factorized and a random
  24-term set expanded, out of place and in place; an integer-valued copy in
  place bit-exact.
- 64 uneven 3D blocks (V in [16,40], O in [6,14]) in one batched plan, FP64
  and FP32 storage; per-block errors against the FP64 oracle.
- 4D, A[10]^8 through autograd: forward and backward against the oracle and
  its literal transpose.
- The paper's layout (tiled kernel): 3D A[544]^3 and 4D A[112]^4, out of place
  and, integer-valued, in place.
"""
import numpy as np
import pytest

import workloads as wl
from tests.gpu_helpers import assert_bitexact, assert_within, chain_norm, fp32_tol, fp64_tol

pytestmark = pytest.mark.gpu


def _dev(A_np):
    """column-major numpy -> CUDA tensor with the same (column-major) strides"""
    import torch
    t = torch.from_numpy(A_np).to("cuda")
    assert t.stride()[0] == 1
    return t


def _host(t):
    return t.cpu().numpy()


def test_config2_3d_full():
    import oracle
    import paper_1705_06661_gb300 as ss
    shape = (48, 48, 48, 16, 16, 16)
    coef = wl.table2(1)
    A_np = wl.uniform(1, shape)
    want = oracle.spinsum(A_np, 3, coef, factorized=True)
    A = _dev(A_np)
    B = ss.colmajor_like(A)
    ss.spinsum(A, coef, d=3, out=B, factorized=True)
    assert_within(_host(B), want, fp64_tol(3, coef, True, A_np), "config 2 out of place")
    del B
    ss.spinsum(A, coef, d=3, inplace=True, factorized=True)
    assert_within(_host(A), want, fp64_tol(3, coef, True, A_np), "config 2 in place")
    del A, want
    Ai_np = wl.integers(1, shape)
    Ai = _dev(Ai_np)
    Bi = ss.colmajor_like(Ai)
    ss.spinsum(Ai, coef, d=3, out=Bi)
    assert_bitexact(_host(Bi), oracle.spinsum(Ai_np, 3, coef), "config 2 integer copy")


def test_config3_4d_full():
    """A[12]^8 in the benchmark's launch configuration: Table II row 5
    factorized (the benchmark's operator), row 6 factorized and the random
    24-term set expanded, each out of place and in place over the whole
    output; an integer-valued copy in place, bit-exact, for row 5 and the
    random set."""
    import oracle
    import paper_1705_06661_gb300 as ss
    shape = (12,) * 8
    A_np = wl.uniform(2, shape)
    A = _dev(A_np)
    B = ss.colmajor_like(A)
    sets = ((wl.table2(5), True), (wl.table2(6), True), (wl.random_coef(4, 103), False))
    for k, (coef, fac) in enumerate(sets):
        want = oracle.spinsum(A_np, 4, coef, factorized=fac)
        ss.spinsum(A, coef, d=4, out=B, factorized=fac)
        assert_within(_host(B), want, fp64_tol(4, coef, fac, A_np), f"config 3 set {k} out of place")
        B.copy_(A)
        ss.spinsum(B, coef, d=4, inplace=True, factorized=fac)
        assert_within(_host(B), want, fp64_tol(4, coef, fac, A_np), f"config 3 set {k} in place")
        del want
    del A
    Ai_np = wl.integers(2, shape)
    Ai = _dev(Ai_np)
    for k, (coef, fac) in enumerate((sets[0], sets[2])):
        B.copy_(Ai)
        ss.spinsum(B, coef, d=4, inplace=True, factorized=fac)
        assert_bitexact(_host(B), oracle.spinsum(Ai_np, 4, coef, factorized=fac), f"config 3 integer set {k} in place")


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_config4_batched_full(dtype):
    import torch
    import oracle
    import paper_1705_06661_gb300 as ss
    blocks = wl.config4_blocks()
    tdt = torch.float64 if dtype == "f64" else torch.float32
    devA, devB, specs = [], [], []
    for pr in blocks:
        A_np = wl.uniform(pr.seed, pr.shape)
        a = _dev(A_np).to(tdt)
        b = ss.colmajor_like(a)
        devA.append(a)
        devB.append(b)
        specs.append({"A": a, "B": b, "coef": pr.coef, "d": 3, "factorized": True})
    plan = ss.Plan(specs, tune=False)
    plan.execute()
    torch.cuda.synchronize()
    worst = 0.0
    for pr, a, b in zip(blocks, devA, devB):
        A_np = a.double().cpu().numpy()       # the values the kernel saw (FP32-rounded for f32)
        want = oracle.spinsum(A_np, 3, pr.coef, factorized=True)
        got = b.double().cpu().numpy()
        if dtype == "f64":
            assert_within(got, want, fp64_tol(3, pr.coef, True, A_np), pr.name)
        else:
            err = assert_within(got, want, fp32_tol(3, pr.coef, True, A_np), pr.name)
            worst = max(worst, err / (chain_norm(3, pr.coef, True) * np.abs(A_np).max()))
    plan.close()
    if dtype == "f32":
        assert worst < 2.0 ** -19


def test_config5_autograd_full():
    import torch
    import oracle
    import paper_1705_06661_gb300 as ss
    shape = (10,) * 8
    A_np = wl.uniform(4, shape)
    G_np = wl.uniform(5, shape)
    coef = wl.random_coef(4, 105)
    A = _dev(A_np).requires_grad_(True)
    B = ss.spinsum_autograd(A, coef, d=4)
    B.backward(_dev(G_np))
    assert_within(B.detach().cpu().numpy(), oracle.spinsum(A_np, 4, coef), fp64_tol(4, coef, False, A_np),
                  "config 5 forward")
    assert_within(A.grad.cpu().numpy(), oracle.spinsum_transpose(G_np, 4, coef), fp64_tol(4, coef, False, G_np),
                  "config 5 backward")


@pytest.mark.parametrize("d,N,row", [(3, 544, 1), (4, 112, 5)])
def test_paper_layout_full(d, N, row):
    """The paper-layout benchmark tensors (tiled kernel): 3D A[544]^3 and 4D
    A[112]^4, Table II row 1 / row 5 factorized out of place against the
    oracle over the whole output; an integer-valued copy in place, bit-exact."""
    import oracle
    import paper_1705_06661_gb300 as ss
    shape = (N,) * d
    coef = wl.table2(row)
    A_np = wl.uniform(3, shape)
    want = oracle.spinsum(A_np, d, coef, factorized=True)
    A = _dev(A_np)
    B = ss.colmajor_like(A)
    ss.spinsum(A, coef, d=d, out=B, factorized=True)
    assert_within(_host(B), want, fp64_tol(d, coef, True, A_np), f"paper layout {d}d N={N}")
    del A, B, want
    Ai_np = wl.integers(3, shape)
    Ai = _dev(Ai_np)
    ss.spinsum(Ai, coef, d=d, inplace=True, factorized=True)
    assert_bitexact(_host(Ai), oracle.spinsum(Ai_np, d, coef, factorized=True), f"paper layout {d}d N={N} integer")
